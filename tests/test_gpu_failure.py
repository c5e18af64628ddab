"""Failure paths of the device-side control, through the C ABI.

Every failure is made on the host, in the inputs: NaN / Inf entries written
into the tensor, a factor with a zero column (its Gramian C^(n) is singular,
so the per-mode Cholesky factor of the core build fails), and one bounded
device wait that is made to run out by the library's self-test kernel (an
mbarrier nothing arrives at; no copy or tensor-core operation in flight).
No kernel is made to fault, trap or hang.

Expected behaviour (Sec. 4.6 leaves failure handling open; the library's
contract):
  * non-finite tensor or factors at cp_state_init: error CP_ENONFINITE,
    stop CP_STOP_ERROR, later steps are no-ops;
  * a trial whose factorisation fails: rejected, rho = 0, mu <- mu nu,
    nu <- 2 nu, status.info set, status.error untouched, factors unchanged;
  * a timed-out wait after cp_state_init: the next step stops the run with
    error CP_ETIMEOUT; a state initialised afterwards is not affected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1205_2584_gb300 import synth  # noqa: E402

CP_ENONFINITE, CP_ETIMEOUT, STOP_ERROR = 3, 4, 4


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_2584_gb300 import cpdgn
    return cpdgn


@pytest.mark.parametrize("dtype,mode", [("f64", 0), ("f32", 1), ("bf16x2", 1)])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_tensor_stops_at_init(cp, dtype, mode, bad):
    p = synth.make_problem(300, (16, 9, 10), 3, snr_db=30)
    Y = np.array(p.Y, copy=True)
    Y[3, 4, 5] = bad
    shape = cp.make_shape(p.dims, p.R, dtype)
    Yd = cp.tensor_to_device(Y, dtype)
    a = cp.factors_to_device(p.init)
    a0 = a.clone()
    st = cp.State(shape, a, mu0=1.0, max_iter=20, core_mode=mode)
    st.init(Yd)
    s = st.status()
    assert s["error"] == CP_ENONFINITE and s["stop"] == STOP_ERROR, s
    for _ in range(3):
        st.step(Yd)
    s = st.status()
    assert s["iters"] == 0 and torch.equal(a, a0)
    st.close()


def test_nonfinite_factor_stops_at_init(cp):
    p = synth.make_problem(301, (8, 9, 10), 3, snr_db=30)
    A = [x.copy() for x in p.init]
    A[1][2, 0] = float("nan")
    shape = cp.make_shape(p.dims, p.R, "f64")
    st = cp.State(shape, cp.factors_to_device(A), mu0=1.0, max_iter=5)
    st.init(cp.tensor_to_device(p.Y, "f64"))
    s = st.status()
    assert s["error"] == CP_ENONFINITE and s["stop"] == STOP_ERROR


@pytest.mark.parametrize("mode", [0, 1])
def test_singular_gramian_rejects_trial_and_raises_mu(cp, mode):
    """A zero column in A^(1): C^(1) is singular, the per-mode Cholesky of the
    core build fails, and the trial must be rejected with rho = 0 however the
    residual moved (mu <- 2 mu at nu = 2, then 4 mu), even at a tiny mu."""
    p = synth.make_problem(302, (12, 9, 10), 3, snr_db=30)
    A = [x.copy() for x in p.init]
    A[0][:, 1] = 0.0
    shape = cp.make_shape(p.dims, p.R, "f64")
    a = cp.factors_to_device(A)
    a0 = a.clone()
    mu0 = 1e-9
    st = cp.State(shape, a, mu0=mu0, max_iter=10, core_mode=mode)
    Y = cp.tensor_to_device(p.Y, "f64")
    st.init(Y)
    st.step(Y)
    s = st.status()
    assert s["info"] != 0, s
    assert s["last_accepted"] == 0 and s["accepted"] == 0 and s["iters"] == 1
    assert s["rho"] == 0.0
    assert s["mu"] == pytest.approx(2 * mu0, rel=1e-15) and s["nu"] == 4.0
    assert s["error"] == 0 and s["stop"] == 0
    assert torch.equal(a, a0)
    st.step(Y)
    s = st.status()
    assert s["mu"] == pytest.approx(8 * mu0, rel=1e-15) and s["nu"] == 8.0
    st.close()


def test_batched_nonfinite_problem_is_isolated(cp):
    """One problem of a batch has a NaN entry: it stops with CP_ENONFINITE at
    its start; the others run as they do without it."""
    specs = synth.config4_specs(5, 4)
    probs = [synth.config4_problem(s, dtype="f32") for s in specs]
    Ybad = np.array(probs[2].Y, copy=True)
    Ybad[0, 0, 0] = float("nan")
    items = [(q.Y, q.init, None) for q in probs]
    clean = cp.Batch(items, tol=1e-8, max_iter=40)
    clean.run()
    items[2] = (Ybad, probs[2].init, None)
    b = cp.Batch(items, tol=1e-8, max_iter=40)
    b.run()
    sb, sc = b.statuses(), clean.statuses()
    assert sb[2]["error"] == CP_ENONFINITE and sb[2]["stop"] == STOP_ERROR and sb[2]["iters"] == 0
    for i in (0, 1, 3):
        assert sb[i]["error"] == 0
        assert sb[i]["iters"] == sc[i]["iters"] and sb[i]["rel_err"] == sc[i]["rel_err"]


def test_timed_out_wait_is_reported(cp):
    """The self-test wait (1 ms limit) runs out; a state initialised before it
    reports CP_ETIMEOUT at its next step and stops; one initialised after it
    runs normally."""
    p = synth.make_problem(303, (16, 9, 10), 3, snr_db=30)
    shape = cp.make_shape(p.dims, p.R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    before = cp.State(shape, cp.factors_to_device(p.init), mu0=1.0, max_iter=10)
    before.init(Y)
    before.step(Y)
    assert before.status()["error"] == 0
    cp.selftest_wait_timeout(1_000_000)
    torch.cuda.synchronize()
    after = cp.State(shape, cp.factors_to_device(p.init), mu0=1.0, max_iter=10)
    after.init(Y)
    before.step(Y)
    after.step(Y)
    sb, sa = before.status(), after.status()
    assert sb["error"] == CP_ETIMEOUT and sb["stop"] == STOP_ERROR, sb
    assert sa["error"] == 0 and sa["stop"] == 0 and sa["iters"] == 1, sa
    n = sb["iters"]
    before.step(Y)
    assert before.status()["iters"] == n          # stopped: further steps are no-ops
    before.close()
    after.close()


def test_selftest_rejects_out_of_range_limit(cp):
    with pytest.raises(cp.CPError):
        cp.selftest_wait_timeout(10)
