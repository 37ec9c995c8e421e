"""The final reweighting of the tensor-core forms from the rounded data X~ to the data X
(oais_set_exact_data): one more target in the annealing sequence, gamma(.; X) after
gamma(.; X~) at beta = 1, reached without a move, so each particle's log w gains
log L(x_T; X) - log L(x_T; X~).

  per particle: the corrected log w equals the oracle's log w on X~ plus the oracle's fp64
    log L(x_T; X) - log L(x_T; X~) at the oracle's final state, within the fp32 bar (1e-5
    relative), for the particles whose MH decisions all clear the tie bound;
  whole run: on the logistic workload's data the corrected bf16 form's log Z_hat and the plain
    FP32 form's (which samples X) agree within 3 standard errors of their difference (pooled
    replicates), while the uncorrected bf16 form sits at the quantisation shift from them.
"""
import numpy as np
import pytest
from mcse import pooled

import oracle as o
from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")


def bf16(X):
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("contraction", ["resident", "stream"])
def test_reweighting_matches_the_oracle_per_particle(contraction):
    pr = W.logistic(n=500, d=16, seed=3)
    N, T = 300, 8
    beta = W.linear_schedule(T) ** 3
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    c = oais.CONTRACT_BF16_TC if contraction == "resident" else oais.CONTRACT_BF16_TC_STREAM
    Xt = bf16(pr.X).astype(np.float64)
    if contraction == "stream":
        Xt = Xt.astype(np.float16).astype(np.float64)
    run = oais.OAIS(pr, oais.MALA, N, beta, eps=eps, seed=11, contraction=c, exact_data=True)
    res = run.round(T)
    logw, ell, x = (t.cpu().numpy().astype(np.float64) for t in run.particles())
    run.close()
    ref = o.asmc(o.Target(pr.kind, Xt, pr.y, pr.ref_scale, pr.p0), o.MALA, N, beta, eps, seed=11)
    tg_x = o.Target(pr.kind, np.asarray(pr.X, dtype=np.float64), pr.y, pr.ref_scale, pr.p0)
    tg_t = o.Target(pr.kind, Xt, pr.y, pr.ref_scale, pr.p0)
    clean = ref["margin"] > 2e-3
    assert clean.mean() > 0.9
    for n in np.flatnonzero(clean):
        want = ref["logw"][n] + tg_x.log_lik(ref["x"][n]) - tg_t.log_lik(ref["x"][n])
        assert logw[n] == pytest.approx(want, rel=1e-5, abs=1e-4), n
        assert ell[n] == pytest.approx(tg_x.log_lik(ref["x"][n]), rel=1e-5, abs=1e-4), n
    lw = torch.from_numpy(logw)
    assert res["logZ"] == pytest.approx(torch.logsumexp(lw, 0).item() - np.log(N), rel=1e-12)


def test_corrected_bf16_estimates_the_log_Z_of_X():
    pr = W.logistic()
    N, T = 1 << 15, 256
    beta = W.linear_schedule(T) ** 4
    eps = oais.default_step_sizes(pr, beta, oais.MALA)
    runs = {"exact": [], "bf16": [], "fp32": []}
    for k in range(4):
        for key, c, ex in [("exact", oais.CONTRACT_BF16_TC, True), ("bf16", oais.CONTRACT_BF16_TC, False),
                           ("fp32", oais.CONTRACT_FP32, False)]:
            r = oais.OAIS(pr, oais.MALA, N, beta, eps=eps, seed=300 + k, contraction=c, exact_data=ex)
            runs[key].append(r.round(T))
            r.close()
    est = {k: pooled([r["logZ"] for r in v], [r["se"] for r in v]) for k, v in runs.items()}
    (ze, se_e), (zf, se_f), (zb, se_b) = est["exact"], est["fp32"], est["bf16"]
    assert abs(ze - zf) < 3 * np.hypot(se_e, se_f), est
    # the uncorrected form estimates log Z of X~: its gap to the fp32 form is the shift (~0.017)
    assert abs((zf - zb) - (zf - ze)) > 0.005, est


def test_exact_data_is_refused_where_it_does_not_apply():
    pr = W.logistic(n=100, d=8, seed=1)
    r = oais.OAIS(pr, oais.MALA, 128, W.linear_schedule(4), contraction=oais.CONTRACT_FP32)
    with pytest.raises(oais.OAISError) as err:
        r.set_exact_data(True)
    assert err.value.status == 6
    r.close()
