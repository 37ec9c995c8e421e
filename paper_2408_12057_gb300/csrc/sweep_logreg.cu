// Bayesian logistic-regression family (fp32 state and data, fp64 log-weights): sweep and ASMC kernel instantiations.
#include "internal.h"
#include <cmath>

namespace oais {

template <int D>
static RowsTarget<D, true> make_logreg(const DevTarget& t, size_t* smem)
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
    *smem = RowsTarget<D, true>::smem_bytes(0);
    return tg;
}

OAIS_FAMILY_DISPATCH(logreg, make_logreg, float,
                     OAIS_WIDTH(2) OAIS_WIDTH(4) OAIS_WIDTH(8) OAIS_WIDTH(16) OAIS_WIDTH(32))

} // namespace oais
