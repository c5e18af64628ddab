"""Graph capture of the LM step.

A captured K-step graph must give the factors and the device status of K
eager cp_dgn_step calls on the same state, in both core modes, with the
refinement converging before its sweep cap and with the cap reached first
(the sweeps after convergence are launched and return at once; their skip
flag lives on the device, so replaying the graph takes the same path).

Several reductions of the step accumulate float64 partial sums with atomic
adds, whose order varies from run to run, so two runs of the same step (eager
or captured) agree to rounding, not bit for bit: the counts must be equal and
the values within 1e-10 relative.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1205_2584_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_2584_gb300 import cpdgn
    return cpdgn


CASES = [((30, 28, 26), 6, "f64", 0, 8), ((30, 28, 26), 6, "f64", 1, 8), ((30, 28, 26), 6, "f32", 1, 1),
         ((30, 28, 26), 6, "f32", 1, 2), ((48, 40, 24), 8, "bf16x2", 1, 8), ((12, 10, 9, 8), 3, "f64", 1, 8),
         ((20, 20, 20), 5, "f64", 1, 0)]


@pytest.mark.parametrize("dims,R,dtype,mode,refine", CASES)
def test_captured_steps_equal_eager(cp, dims, R, dtype, mode, refine):
    p = synth.make_problem(41, dims, R, dtype=dtype, snr_db=30.0, collinearity=(0.9,))
    shape = cp.make_shape(dims, R, dtype)
    Y = cp.tensor_to_device(p.Y, dtype)
    K = 6
    a1 = cp.factors_to_device(p.init)
    a2 = a1.clone()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st1 = cp.State(shape, a1, mu0=-1.0, max_iter=100, core_mode=mode, refine_iters=refine)
        st1.init(Y)
        for _ in range(K):
            st1.step(Y)
        st2 = cp.State(shape, a2, mu0=-1.0, max_iter=100, core_mode=mode, refine_iters=refine)
        st2.init(Y)
        nk = st2.capture(Y, K)
        st2.launch()
        s1, s2 = st1.status(), st2.status()
    torch.cuda.synchronize()
    assert nk > 0
    assert float(torch.linalg.norm(a1 - a2) / torch.linalg.norm(a1)) < 1e-10
    for k in ("iters", "accepted", "stop", "nu"):
        assert s1[k] == s2[k], k
    for k in ("mu", "resid2", "rel_err"):
        assert s2[k] == pytest.approx(s1[k], rel=1e-10, abs=0.0), k
    assert abs(s1["refine_sweeps"] - s2["refine_sweeps"]) <= 1
    if mode == 1 and refine > 0:
        assert 1 <= s2["refine_sweeps"] <= refine
    if mode == 1 and refine >= 8:
        assert s2["refine_resid"] < 1e-8
