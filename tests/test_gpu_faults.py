"""Failure paths of a round, driven without a GPU fault (host-side faults armed through
oais_arm_fault), and the anytime property they must keep (Sec. 1: every completed round
leaves a valid estimate and schedule; a failed round changes neither).

  NaN data    element 0 of the context's device copies of X becomes NaN for one round: every
              log-likelihood is NaN, the status check reports OAIS_ENONFINITE.
  withheld    a tensor-core sweep that runs as a persistent grid raises no hand-off flag, so
  hand-off    each resumed tile's bounded wait (50 ms here) gives up: OAIS_ETIMEOUT, with the
              GPU still answering.

In each case the last round's log Z_hat, statistics, ELBO terms and the next schedule are
unchanged by the failed round, the round counter does not advance, and the following round is
bit-identical to the same round of an undisturbed run.
"""
import numpy as np
import pytest

from paper_2408_12057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
oais = pytest.importorskip("paper_2408_12057_gb300.oais")


def snapshot(r):
    b, e = r.schedule()
    st = r.stats()
    return {"logZ": r.logZ(), "beta_next": b, "eps_next": e, "elbo": r.elbo_terms(), **st}


def assert_same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        np.testing.assert_array_equal(np.asarray(a[k]), np.asarray(b[k]), err_msg=k)


CASES = {
    # CUDA-core fp32 form, fp64 form, resident tensor-core form, streamed tensor-core form
    "fp32_logreg": lambda: (W.logistic(n=300, d=8, seed=3), oais.MALA, 4096, 12,
                            dict(contraction=oais.CONTRACT_FP32)),
    "fp64_gauss": lambda: (W.gauss_conj(), oais.RWMH, 2048, 12, dict()),
    "tc_resident": lambda: (W.logistic(), oais.MALA, 2048, 6, dict(contraction=oais.CONTRACT_BF16_TC)),
    "tc_stream": lambda: (W.linreg(n=500, d=16, seed=4), oais.HMC, 1024, 6,
                          dict(contraction=oais.CONTRACT_BF16_TC_STREAM, leapfrog=3)),
}


def make(case, N=None):
    pr, move, N0, T, kw = CASES[case]()
    N = N or N0
    beta = W.linear_schedule(T) ** 2
    eps = oais.default_step_sizes(pr, beta, move)
    return (lambda: oais.OAIS(pr, move, N, beta, eps=eps, seed=31, **kw)), T


@pytest.mark.parametrize("case", list(CASES))
def test_nan_data_fails_the_round_and_keeps_the_last_one(case):
    new, T = make(case)
    r = new()
    r.round(T)
    before = snapshot(r)
    r.arm_fault(oais.FAULT_NAN_DATA)
    with pytest.raises(oais.OAISError) as err:
        r.round(T)
    assert err.value.status == 4, err.value
    assert_same(snapshot(r), before)
    # the data is restored and the round counter did not move: the retried round is the
    # second round of an undisturbed run
    again = r.round(T)
    ref = new()
    ref.round(T)
    want = ref.round(T)
    assert again["round"] == want["round"] == 1
    assert again["logZ"] == want["logZ"] and again["Lambda_hat"] == want["Lambda_hat"]
    r.close()
    ref.close()


@pytest.mark.parametrize("case,N", [("tc_resident", 1 << 16), ("tc_stream", 1 << 17)])
def test_withheld_handoff_times_out_and_the_gpu_stays_usable(case, N):
    # N above one wave of groups (resident: 2 per SM) or CTAs (streamed), so the sweep runs as
    # a persistent grid whose split tiles are handed over between CTAs
    new, T = make(case, N)
    r = new()
    r.round(T)
    before = snapshot(r)
    r.arm_fault(oais.FAULT_WITHHOLD_HANDOFF, 0.05)
    with pytest.raises(oais.OAISError) as err:
        r.round(T)
    assert err.value.status == 5, err.value
    assert_same(snapshot(r), before)
    again = r.round(T)
    ref = new()
    ref.round(T)
    want = ref.round(T)
    assert again["logZ"] == want["logZ"] and again["Lambda_hat"] == want["Lambda_hat"]
    # the device is healthy: an unrelated computation still runs
    x = torch.arange(10, dtype=torch.float64, device="cuda")
    assert float(x.sum().item()) == 45.0
    r.close()
    ref.close()


def test_arm_fault_rejects_what_it_cannot_do():
    new, T = make("fp32_logreg")
    r = new()
    with pytest.raises(oais.OAISError) as err:
        r.arm_fault(oais.FAULT_WITHHOLD_HANDOFF)      # the CUDA-core form hands nothing over
    assert err.value.status == 6
    with pytest.raises(oais.OAISError):
        r.arm_fault(7)
    r.arm_fault(oais.FAULT_NAN_DATA)
    r.arm_fault(oais.FAULT_NONE)                     # disarmed: the round runs
    r.round(T)
    r.close()
