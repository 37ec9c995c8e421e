// Bayesian logistic-regression family (fp32 state and data, fp64 log-weights): sweep kernel instantiations.
#include "internal.h"
#include <cmath>

namespace oais {

template <int D>
static cudaError_t go(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s)
{
    RowsTarget<D, true> tg;
    tg.X = static_cast<const float*>(t.X);
    tg.y = static_cast<const float*>(t.y);
    tg.d = t.d;
    tg.n = t.n;
    tg.inv_sig2 = (float)(1.0 / (t.p0 * t.p0));
    tg.lin_const = (float)(-0.5 * t.n * std::log(6.283185307179586 * t.p0 * t.p0));
    tg.xs = nullptr;
    tg.ys = nullptr;
    const size_t smem = RowsTarget<D, true>::smem_bytes(0);
    switch (move) {
    case kRwmh: return launch_one<RowsTarget<D, true>, kRwmh, D, float>(tg, smem, P, s);
    case kMala: return launch_one<RowsTarget<D, true>, kMala, D, float>(tg, smem, P, s);
    case kHmc:  return launch_one<RowsTarget<D, true>, kHmc, D, float>(tg, smem, P, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_logreg(const DevTarget& t, int move, const SweepParams& P, cudaStream_t s)
{
    switch (t.D) {
    case 2: return go<2>(t, move, P, s);
    case 4: return go<4>(t, move, P, s);
    case 8: return go<8>(t, move, P, s);
    case 16: return go<16>(t, move, P, s);
    case 32: return go<32>(t, move, P, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace oais
