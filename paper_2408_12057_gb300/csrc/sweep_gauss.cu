// Conjugate-Gaussian family (fp64 throughout): sweep and ASMC kernel instantiations.
#include "internal.h"

namespace oais {

template <int D>
static GaussTarget<double, D> make_gauss(const DevTarget& t, size_t* smem)
{
    GaussTarget<double, D> tg;
    tg.mu = static_cast<const double*>(t.X);
    tg.d = t.d;
    tg.inv_sig2 = 1.0 / (t.p0 * t.p0);
    *smem = 0;
    return tg;
}

OAIS_FAMILY_DISPATCH(gauss, make_gauss, double,
                     OAIS_WIDTH(1) OAIS_WIDTH(2) OAIS_WIDTH(4) OAIS_WIDTH(8) OAIS_WIDTH(16))

} // namespace oais
