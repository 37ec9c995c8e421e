// Conjugate-Gaussian family (fp64 throughout): sweep kernel instantiations.
#include "internal.h"

namespace oais {

template <int D>
static cudaError_t go(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s)
{
    GaussTarget<double, D> tg;
    tg.mu = static_cast<const double*>(t.X);
    tg.d = t.d;
    tg.inv_sig2 = 1.0 / (t.p0 * t.p0);
    switch (move) {
    case kRwmh: return launch_one<GaussTarget<double, D>, kRwmh, D, double>(tg, 0, P, s);
    case kMala: return launch_one<GaussTarget<double, D>, kMala, D, double>(tg, 0, P, s);
    case kHmc:  return launch_one<GaussTarget<double, D>, kHmc, D, double>(tg, 0, P, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_gauss(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s)
{
    switch (t.D) {
    case 1: return go<1>(t, move, P, s);
    case 2: return go<2>(t, move, P, s);
    case 4: return go<4>(t, move, P, s);
    case 8: return go<8>(t, move, P, s);
    case 16: return go<16>(t, move, P, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace oais
