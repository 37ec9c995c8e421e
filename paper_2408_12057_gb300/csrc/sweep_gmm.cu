// Gaussian-mixture family (fp32 state, fp64 log-weights): sweep and ASMC kernel instantiations.
#include "internal.h"
#include <cmath>

namespace oais {

template <int D>
static GmmTarget<float, D> make_gmm(const DevTarget& t, size_t* smem)
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
    tg.sm = nullptr;
    tg.fsched = t.fsched;
    tg.c2 = (float)(-0.5 / t.p0 * 1.4426950408889634);
    tg.rks = RngKS{};
    *smem = GmmTarget<float, D>::smem_bytes(t.n);
    return tg;
}

OAIS_FAMILY_DISPATCH(gmm, make_gmm, float, OAIS_WIDTH(2) OAIS_WIDTH(4) OAIS_WIDTH(8) OAIS_WIDTH(16))

} // namespace oais
