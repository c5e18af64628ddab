"""The tensor-core pass (3-way float32 tensors, I_1 a multiple of 4) against
the oracle: all-mode MTTKRP, direct residual and LM runs to convergence.

The pass splits operands into bf16 pieces (see the kernel's header); the
MTTKRP is held to 2e-5 relative (norm-wise per mode), the residual to 1e-6
and a converged run's final relative error to 1e-6 of the oracle's on the
same float32-rounded tensor."""
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
    a = np.ravel(np.asarray(a))
    b = np.ravel(np.asarray(b))
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def setup(cp, p):
    shape = cp.make_shape(p.dims, p.R, "f32")
    return shape, cp.tensor_to_device(p.Y, "f32"), cp.factors_to_device(p.init)


# ragged 128-row chunks and blocks, tiny and full-rank R, I_1 < 32
SHAPES = [((132, 136, 5), 7), ((128, 128, 3), 32), ((200, 200, 4), 20), ((4, 5, 6), 1),
          ((36, 300, 2), 16), ((256, 40, 9), 3), ((12, 129, 130), 5)]


@pytest.mark.parametrize("dims,R", SHAPES)
def test_tc_mttkrp_and_residual(cp, dims, R):
    p = synth.make_problem(300 + R, dims, R, dtype="f32", snr_db=30, collinearity=(0.6,))
    shape, Y, a = setup(cp, p)
    m, r2 = cp.mttkrp_all(shape, Y, a)
    got = cp.split_factors(m.cpu(), p.dims, p.R)
    ref = O.mttkrp_all(p.Y, p.init)
    for n in range(3):
        assert rel(got[n].numpy(), ref[n]) < 2e-5, n
    assert float(r2.item()) == pytest.approx(O.residual2(p.Y, p.init), rel=1e-6)


@pytest.mark.parametrize("dims,R", SHAPES[:3])
def test_tc_mttkrp_without_residual_and_fit_alone(cp, dims, R):
    p = synth.make_problem(400 + R, dims, R, dtype="f32", snr_db=30)
    shape, Y, a = setup(cp, p)
    m, _ = cp.mttkrp_all(shape, Y, a, want_resid=False)
    r2, rel_err = cp.fit(shape, Y, a, y_norm2=float(np.sum(p.Y ** 2)))
    torch.cuda.synchronize()
    got = cp.split_factors(m.cpu(), p.dims, p.R)
    ref = O.mttkrp_all(p.Y, p.init)
    for n in range(3):
        assert rel(got[n].numpy(), ref[n]) < 2e-5
    assert float(r2.item()) == pytest.approx(O.residual2(p.Y, p.init), rel=1e-6)
    assert float(rel_err.item()) == pytest.approx(O.rel_error(p.Y, p.init), rel=1e-6)


@pytest.mark.parametrize("core_mode", [0, 1])
def test_tc_lm_run_reaches_oracle_fit(cp, core_mode):
    """Collinear float32 problem run to its stop rule (relative error change
    < 1e-9): final relative error within 1e-6 of the oracle's."""
    p = synth.make_problem(501, (64, 72, 40), 8, dtype="f32", snr_db=40,
                           collinearity=(0.95, 0.81, 0.81))
    shape, Y, a = setup(cp, p)
    st = cp.State(shape, a, mu0=-1.0, tol=1e-9, max_iter=400, core_mode=core_mode)
    st.init(Y)
    for _ in range(400):
        st.step(Y)
        if st.status()["stop"] != 0:
            break
    s = st.status()
    ref = O.lm_fit(p.Y, p.init, mu0=None, max_iter=400, tol=1e-9)
    assert s["stop"] != 0
    assert s["rel_err"] == pytest.approx(ref.rel_err, rel=1e-6), (s, ref.rel_err, ref.iters)


def _one_step_check(cp, dtype, mu, record=None):
    """One fLM step on a reduced-precision tensor against the oracle on the
    same stored values, split into its two error sources:
      (1) the pass: the GPU's MTTKRP M against the oracle's (float32-level),
          and, where the pass gives the gradient blocks G_n = E_(n) KR_n
          directly (float32 tensors), G against the oracle's M - A Gamma;
      (2) the float64 algebra: the GPU step against the oracle's fLM_a step
          computed from the GPU's own M, held to max(1e-10, 1e-15 kappa(core));
      (3) end to end: the GPU step against the oracle's own step, bounded by
          how far (1) moves the step through the damped system,
          ||H_mu^{-1}|| ||M_gpu - M_ref|| (first order; the gradient blocks
          are G_n = M_n - A^(n) Gamma^(n)), with the observed error and kappa
          recorded; and the trial residual (formed from the stored tensor)
          to 1e-6 of the oracle's residual at the GPU's trial point."""
    p = synth.make_problem(502, (16, 24, 20), 4, dtype=dtype, snr_db=30, collinearity=(0.7,))
    shape = cp.make_shape(p.dims, p.R, dtype)
    Y = cp.tensor_to_device(p.Y, dtype)
    a = cp.factors_to_device(p.init)
    st = cp.State(shape, a, mu0=mu, max_iter=10, core_mode=1, normalize=False)
    st.init(Y)
    torch.cuda.synchronize()
    nA = p.R * sum(p.dims)
    B_gpu = [x.numpy().copy() for x in cp.split_factors(st.buffer(cp.State.BUF_M, nA).cpu(), p.dims, p.R)]
    g0 = O.grams(p.init)
    if st.holds_gradient:
        # the pass gave the gradient blocks G_n = E_(n) KR_n; M_n = G_n + A^(n) Gamma^(n)
        G_ref = O.gradient_blocks(p.Y, p.init)
        for n in range(3):
            assert rel(B_gpu[n], G_ref[n]) < 2e-5, n
        M_gpu = [b + a @ g0.Gamma(n) for n, (a, b) in enumerate(zip(p.init, B_gpu))]
    else:
        M_gpu = B_gpu
    st.step(Y)
    torch.cuda.synchronize()
    delta = [x.numpy() for x in cp.split_factors(st.buffer(cp.State.BUF_DELTA, nA).cpu(), p.dims, p.R)]
    M_ref = O.mttkrp_all(p.Y, p.init)
    for n in range(3):
        assert rel(M_gpu[n], M_ref[n]) < 2e-5, n                              # (1)
    ev = np.linalg.eigvalsh(O.spd_core(p.init, mu))
    kappa_core = float(ev[-1] / ev[0])
    own = O.flm_step(p.Y, p.init, mu, M=M_gpu)
    alg_err = rel(np.concatenate([d.ravel() for d in delta]), np.concatenate([d.ravel() for d in own.delta]))
    assert alg_err < max(1e-10, 1e-15 * kappa_core), (alg_err, kappa_core)   # (2)
    ref = O.flm_step(p.Y, p.init, mu)
    Jm = O.jacobian(p.init)
    H = Jm.T @ Jm + mu * np.eye(Jm.shape[1])
    kappa_h = float(np.linalg.cond(H))
    inv_norm = 1.0 / float(np.linalg.eigvalsh(H)[0])
    dM = float(np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(M_gpu, M_ref))))
    d_gpu = np.concatenate([d.ravel() for d in delta])
    d_ref = np.concatenate([d.ravel() for d in ref.delta])
    err = float(np.linalg.norm(d_gpu - d_ref))
    bound = 1.01 * inv_norm * dM + 1e-10 * float(np.linalg.norm(d_ref))
    if record is not None:
        record("step_rel_err", err / float(np.linalg.norm(d_ref)))
        record("kappa_H_mu", kappa_h)
        record("kappa_core", kappa_core)
    assert err <= bound, (err, bound, kappa_h)                                 # (3)
    trial = [a0 + d for a0, d in zip(p.init, delta)]
    assert st.status()["resid2_trial"] == pytest.approx(O.residual2(p.Y, trial), rel=1e-6)


@pytest.mark.parametrize("mu", [0.7, 50.0])
def test_tc_one_step_close_to_oracle(cp, mu, record_property):
    _one_step_check(cp, "f32", mu, record_property)


# --- two-plane bfloat16 tensors (TMA tiles are the tensor-core operands) ---
SHAPES3 = [((136, 136, 5), 7), ((128, 128, 3), 32), ((200, 200, 4), 20), ((8, 5, 6), 1),
           ((40, 300, 2), 16), ((256, 40, 9), 3), ((16, 129, 130), 5)]


def test_tensor_split_is_exact(cp):
    rng = np.random.default_rng(3)
    y = rng.standard_normal(10007) * np.exp(rng.uniform(-20, 20, 10007))
    y32 = torch.from_numpy(y.astype(np.float32)).cuda()
    out = cp.tensor_split(y32)
    torch.cuda.synchronize()
    hi = out[:10007].double().cpu().numpy()
    lo = out[10007:].double().cpu().numpy()
    assert np.array_equal(hi + lo, synth.cast_like(y, "bf16x2"))
    assert np.array_equal(hi, synth.cast_like(y, "bf16"))


@pytest.mark.parametrize("dtype", ["bf16x2", "bf16"])
@pytest.mark.parametrize("dims,R", SHAPES3)
def test_tc3_mttkrp_and_residual(cp, dims, R, dtype):
    """The oracle runs on exactly the values the planes hold, so only the
    factor-side rounding (~2^-22) and float32 accumulation remain."""
    p = synth.make_problem(600 + R, dims, R, dtype=dtype, snr_db=30, collinearity=(0.6,))
    shape = cp.make_shape(p.dims, p.R, dtype)
    Y = cp.tensor_to_device(p.Y, dtype)
    a = cp.factors_to_device(p.init)
    m, r2 = cp.mttkrp_all(shape, Y, a)
    got = cp.split_factors(m.cpu(), p.dims, p.R)
    ref = O.mttkrp_all(p.Y, p.init)
    for n in range(3):
        assert rel(got[n].numpy(), ref[n]) < 1e-5, n
    assert float(r2.item()) == pytest.approx(O.residual2(p.Y, p.init), rel=1e-6)


@pytest.mark.parametrize("core_mode", [0, 1])
def test_tc3_lm_run_reaches_oracle_fit(cp, core_mode):
    p = synth.make_problem(601, (64, 72, 40), 8, dtype="bf16x2", snr_db=40,
                           collinearity=(0.95, 0.81, 0.81))
    shape = cp.make_shape(p.dims, p.R, "bf16x2")
    Y = cp.tensor_to_device(p.Y, "bf16x2")
    a = cp.factors_to_device(p.init)
    st = cp.State(shape, a, mu0=-1.0, tol=1e-9, max_iter=400, core_mode=core_mode)
    st.init(Y)
    for _ in range(400):
        st.step(Y)
        if st.status()["stop"] != 0:
            break
    s = st.status()
    ref = O.lm_fit(p.Y, p.init, mu0=None, max_iter=400, tol=1e-9)
    assert s["stop"] != 0
    assert s["y_norm2"] == pytest.approx(float(np.sum(p.Y ** 2)), rel=1e-12)
    assert s["rel_err"] == pytest.approx(ref.rel_err, rel=1e-6), (s, ref.rel_err, ref.iters)


@pytest.mark.parametrize("mu", [0.7, 50.0])
def test_tc3_one_step_close_to_oracle(cp, mu, record_property):
    _one_step_check(cp, "bf16x2", mu, record_property)
