// Unidentifiable product family (fp64 throughout): sweep, ASMC and potential kernel
// instantiations.  The device array X holds (m, k, b, c0).
#include "internal.h"

namespace oais {

template <int D>
static UnidTarget<double, D> make_unid(const DevTarget& t, size_t* smem)
{
    UnidTarget<double, D> tg;
    tg.par = static_cast<const double*>(t.X);
    tg.d = t.d;
    *smem = 0;
    return tg;
}

OAIS_FAMILY_DISPATCH(unid, make_unid, double, OAIS_WIDTH(2))

} // namespace oais
