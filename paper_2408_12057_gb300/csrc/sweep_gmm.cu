// Gaussian-mixture family (fp32 state, fp64 log-weights): sweep kernel instantiations.
#include "internal.h"
#include <cmath>

namespace oais {

template <int D>
static cudaError_t go(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s)
{
    GmmTarget<float, D> tg;
    tg.means = static_cast<const float*>(t.X);
    tg.d = t.d;
    tg.K = t.n;
    tg.inv_v = (float)(1.0 / t.p0);
    tg.inv_s2 = (float)(1.0 / (t.ref_scale * t.ref_scale));
    const double two_pi = 6.283185307179586;
    tg.log_const = (float)(-0.5 * t.d * std::log(two_pi * t.p0) - std::log((double)t.n)
                           + 0.5 * t.d * std::log(two_pi * t.ref_scale * t.ref_scale));
    const size_t smem = GmmTarget<float, D>::smem_bytes(t.n);
    switch (move) {
    case kRwmh: return launch_one<GmmTarget<float, D>, kRwmh, D, float>(tg, smem, P, s);
    case kMala: return launch_one<GmmTarget<float, D>, kMala, D, float>(tg, smem, P, s);
    case kHmc:  return launch_one<GmmTarget<float, D>, kHmc, D, float>(tg, smem, P, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_gmm(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s)
{
    switch (t.D) {
    case 2: return go<2>(t, move, P, s);
    case 4: return go<4>(t, move, P, s);
    case 8: return go<8>(t, move, P, s);
    case 16: return go<16>(t, move, P, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace oais
