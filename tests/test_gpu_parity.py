"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every input is seeded and synthetic; expected values come from ``oracle/``
only.  Tolerances:
  * float64 tensors: every quantity within 1e-12 relative (norm-wise) except
    the step itself, which must agree with the oracle's fLM_a step to 1e-10
    relative (a bound that holds for the well-conditioned cases used here;
    the two sides solve the same core system with different factorisations).
  * float32 / bfloat16 tensors (float32 arithmetic in the pass over Y): the
    oracle runs on the same rounded tensor values; MTTKRP within 2e-5
    relative norm-wise and the residual within 1e-5 relative.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cp_oracle as O  # noqa: E402
from paper_1205_2584_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_2584_gb300 import cpdgn
    return cpdgn


def rel(a, b):
    a = np.concatenate([np.ravel(np.asarray(x)) for x in a]) if isinstance(a, (list, tuple)) else np.ravel(np.asarray(a))
    b = np.concatenate([np.ravel(np.asarray(x)) for x in b]) if isinstance(b, (list, tuple)) else np.ravel(np.asarray(b))
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def setup(cp, p, dtype=None):
    dtype = dtype or p.dtype
    shape = cp.make_shape(p.dims, p.R, dtype)
    Y = cp.tensor_to_device(p.Y, dtype)
    a = cp.factors_to_device(p.init)
    return shape, Y, a


# ragged and degenerate shapes: N = 2..5, R = 1..32, I_1 = 1, I_n = 1, I_1 above
# 256 / 512 / 768 rows (the tiled pass keeps 1, 2 or 3 rows per thread; above
# that a generic pass takes over), I_2 smaller than a tile of fibres
SHAPES = [((7, 9, 11), 3), ((20, 20, 20), 5), ((13, 6), 4), ((5, 4, 3, 6), 2), ((33, 17, 9), 1),
          ((300, 5, 7), 6), ((4, 3, 2, 3, 2), 3), ((1, 8, 9), 2), ((9, 1, 7), 3), ((11, 12, 13), 32),
          ((600, 4, 5), 3), ((800, 3, 2), 2), ((20, 3, 40), 5), ((64, 2, 3, 50), 7), ((31, 29, 37), 17)]


@pytest.mark.parametrize("dims,R", SHAPES)
def test_gram(cp, dims, R):
    p = synth.make_problem(100, dims, R, snr_db=30)
    shape, Y, a = setup(cp, p, "f64")
    C, Gnm, Gall = cp.gram(shape, a)
    g = O.grams(p.init)
    N = len(dims)
    C = C.cpu().numpy().reshape(N, R, R).transpose(0, 2, 1)
    Gnm = Gnm.cpu().numpy().reshape(N, N, R, R).transpose(0, 1, 3, 2)
    assert rel(C, np.stack(g.C)) < 1e-13
    assert rel(Gnm, g.Gamma_nm) < 1e-13
    assert rel(Gall.cpu().numpy().reshape(R, R).T, g.Gamma_all) < 1e-13


@pytest.mark.parametrize("dims,R", SHAPES)
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_mttkrp_and_residual(cp, dims, R, dtype):
    p = synth.make_problem(101, dims, R, snr_db=20, dtype=dtype)
    shape, Y, a = setup(cp, p)
    m, r2 = cp.mttkrp_all(shape, Y, a)
    M_ref = O.mttkrp_all(p.Y, p.init)
    m_gpu = cp.split_factors(m.cpu(), dims, R)
    r2_ref = O.residual2(p.Y, p.init)
    tol_m, tol_r = (1e-12, 1e-12) if dtype == "f64" else (2e-5, 1e-5)
    for n in range(len(dims)):
        assert rel(m_gpu[n].numpy(), M_ref[n]) < tol_m, n
    assert abs(float(r2.item()) - r2_ref) <= tol_r * r2_ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fit_rel_err(cp, dtype):
    p = synth.make_problem(102, (17, 19, 23), 4, snr_db=25, dtype=dtype)
    shape, Y, a = setup(cp, p)
    yn2 = float(np.sum(p.Y ** 2))
    r2, relerr = cp.fit(shape, Y, a, yn2)
    tol = 1e-12 if dtype == "f64" else 1e-5
    assert abs(relerr.item() - O.rel_error(p.Y, p.init)) <= tol * O.rel_error(p.Y, p.init)


def _core_ref(p, mu):
    return O.spd_core(p.init, mu)


@pytest.mark.parametrize("dims,R,mu", [((7, 9, 11), 3, 0.5), ((20, 20, 20), 5, 1.0),
                                       ((13, 6), 4, 2.0), ((5, 4, 3, 6), 2, 0.3), ((12, 13, 14), 8, 0.7)])
def test_core_build_and_solve(cp, dims, R, mu):
    p = synth.make_problem(103, dims, R, snr_db=30)
    shape, Y, a = setup(cp, p, "f64")
    m, _ = cp.mttkrp_all(shape, Y, a)
    mu_t = torch.tensor([mu], dtype=torch.float64, device="cuda")
    core, Gt, w, info = cp.core_build(shape, a, m, mu_t)
    assert info.item() == 0
    n = len(dims) * R * R
    core_np = core.cpu().numpy().reshape(n, n).T          # column-major -> row index first
    ref = _core_ref(p, mu)
    low = np.tril_indices(n)
    assert rel(core_np[low], ref[low]) < 1e-12
    st = O.flm_step(p.Y, p.init, mu)
    N = len(dims)
    Gt_np = Gt.cpu().numpy().reshape(N, R, R).transpose(0, 2, 1)
    assert rel(Gt_np, np.stack(st.Gt)) < 1e-12
    assert rel(w.cpu().numpy(), st.w) < 1e-11
    f, info2 = cp.core_solve(shape, a, mu_t, core, w)
    assert info2.item() == 0
    assert rel(f.cpu().numpy(), st.f) < 1e-10


def _one_step(cp, p, mu, core_mode, dtype="f64"):
    shape, Y, a = setup(cp, p, dtype)
    st = cp.State(shape, a, mu0=mu, max_iter=10, core_mode=core_mode, normalize=False)
    st.init(Y)
    st.step(Y)
    torch.cuda.synchronize()
    R, dims = p.R, p.dims
    delta = cp.split_factors(st.buffer(cp.State.BUF_DELTA, R * sum(dims)).cpu(), dims, R)
    return st, [d.numpy() for d in delta], a


@pytest.mark.parametrize("core_mode", [0, 1])
@pytest.mark.parametrize("dims,R,mu", [((7, 9, 11), 3, 0.5), ((20, 20, 20), 5, 1.0),
                                       ((6, 5, 4, 3), 2, 0.2), ((15, 16), 3, 1.5),
                                       ((30, 31, 29), 12, 0.8)])
def test_step_matches_oracle(cp, dims, R, mu, core_mode):
    p = synth.make_problem(104, dims, R, snr_db=30)
    st, delta, _ = _one_step(cp, p, mu, core_mode)
    ref = O.flm_step(p.Y, p.init, mu)
    assert rel(delta, ref.delta) < 1e-10
    s = st.status()
    r2_trial = O.residual2(p.Y, ref.A_new)
    assert s["resid2_trial"] == pytest.approx(r2_trial, rel=1e-10)
    den = sum(float(np.sum(d * (g + mu * d))) for d, g in zip(ref.delta, ref.G))
    assert s["denom"] == pytest.approx(den, rel=1e-9)
    assert s["iters"] == 1


def test_step_matches_textbook_small(cp):
    p = synth.make_problem(105, (5, 6, 7), 3, snr_db=30)
    st, delta, _ = _one_step(cp, p, 0.9, 0)
    assert rel(delta, O.textbook_step(p.Y, p.init, 0.9)) < 1e-10


@pytest.mark.parametrize("core_mode", [0, 1])
def test_lm_run_config1(cp, core_mode):
    """Config 1 (20^3, R = 5, float64, SNR 30 dB, mu0 = 1): the first 30
    trials follow the oracle's trajectory, and 200 trials reach the same fit."""
    p = synth.config1(0)
    shape, Y, a = setup(cp, p)
    st = cp.State(shape, a, mu0=1.0, max_iter=200, core_mode=core_mode)
    st.init(Y)
    hist = []
    for _ in range(30):
        st.step(Y)
        hist.append(math.sqrt(st.status()["resid2"] / st.status()["y_norm2"]))
    ref = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=30)
    assert np.allclose(hist, ref.history, rtol=1e-8, atol=0)
    for _ in range(170):
        st.step(Y)
    s = st.status()
    ref200 = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=200)
    # both stop once mu passes 1e30 at the noise floor; the trial count there
    # depends on rounding-level accept/reject decisions
    assert s["stop_reason"] == ref200.stop == "mu_max"
    assert s["iters"] <= 200 and ref200.iters <= 200
    assert s["rel_err"] == pytest.approx(ref200.rel_err, rel=1e-10)


@pytest.mark.parametrize("dims,R", [((8, 9, 10), 3), ((6, 7, 5, 6), 2)])
def test_noiseless_converges_on_gpu(cp, dims, R):
    p = synth.make_problem(21, dims, R, snr_db=None)
    rng = np.random.default_rng(22)
    A0 = [x + 0.3 * rng.standard_normal(x.shape) for x in p.true_factors]
    shape = cp.make_shape(dims, R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    a = cp.factors_to_device(A0)
    st = cp.State(shape, a, mu0=1.0, max_iter=300)
    st.init(Y)
    for _ in range(300):
        st.step(Y)
    assert st.status()["rel_err"] < 1e-10


def test_stop_flag_makes_steps_noops(cp):
    p = synth.make_problem(106, (9, 10, 11), 3, snr_db=30)
    shape, Y, a = setup(cp, p)
    st = cp.State(shape, a, mu0=1.0, max_iter=3)
    st.init(Y)
    for _ in range(3):
        st.step(Y)
    s3 = st.status()
    a3 = a.clone()
    for _ in range(4):
        st.step(Y)
    s7 = st.status()
    assert s3["stop_reason"] == "max_iter" and s7["iters"] == 3
    assert torch.equal(a, a3)


def test_full_size_config2_sampled(cp):
    """200^3, R = 20, collinear, SNR 40 dB, float32 tensor: MTTKRP rows and the
    residual at full size, checked on sampled rows computed one by one."""
    p = synth.config2(0, dtype="f32")
    shape, Y, a = setup(cp, p)
    m, r2 = cp.mttkrp_all(shape, Y, a)
    mg = cp.split_factors(m.cpu(), p.dims, p.R)
    rng = np.random.default_rng(7)
    for n in range(3):
        KR = O.kr_except(p.init, n)
        Yn = O.unfold(p.Y, n)
        for i in rng.integers(0, p.dims[n], size=4):
            ref = Yn[i] @ KR
            assert rel(mg[n][i].numpy(), ref) < 2e-5
    assert float(r2.item()) == pytest.approx(O.residual2(p.Y, p.init), rel=1e-5)


def test_full_size_config3_sampled(cp):
    """60^4, R = 15 (core N R^2 = 900), column norms log-uniform over
    [1e-2, 1e2], SNR 30 dB, bfloat16 tensor (the 4-way SIMT pass): MTTKRP rows
    sampled in every mode and the residual at full size against the oracle on
    the same rounded tensor; then one mixed-precision step, whose trial
    residual must equal the oracle's residual at the GPU's trial point."""
    p = synth.config3(0)
    shape, Y, a = setup(cp, p, "bf16")
    m, r2 = cp.mttkrp_all(shape, Y, a)
    mg = cp.split_factors(m.cpu(), p.dims, p.R)
    rng = np.random.default_rng(11)
    for n in range(4):
        KR = O.kr_except(p.init, n)
        Yn = O.unfold(p.Y, n)
        for i in rng.integers(0, p.dims[n], size=3):
            ref = Yn[i] @ KR
            assert rel(mg[n][i].numpy(), ref) < 2e-5, (n, i)
    assert float(r2.item()) == pytest.approx(O.residual2(p.Y, p.init), rel=1e-5)
    st = cp.State(shape, a.clone(), mu0=-1.0, max_iter=5, core_mode=1, normalize=False)
    st.init(Y)
    st.step(Y)
    torch.cuda.synchronize()
    delta = cp.split_factors(st.buffer(cp.State.BUF_DELTA, p.R * sum(p.dims)).cpu(), p.dims, p.R)
    trial = [a0 + d.numpy() for a0, d in zip(p.init, delta)]
    assert st.status()["resid2_trial"] == pytest.approx(O.residual2(p.Y, trial), rel=1e-5)
    assert st.status()["refine_resid"] < 1e-8
    assert 1 <= st.status()["refine_sweeps"] <= 8
