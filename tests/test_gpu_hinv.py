"""Theorem 4's block form of the inverse damped Hessian (cp_hinv_blocks,
cp_hinv_diag) and the squared angular errors of Sec. 6 (cp_sae), through the
C ABI, against the oracle.

  * Gt and St against the oracle's hinv_blocks (fLM_a's B_mu = K (I + Psi K)^{-1})
    to 1e-10 relative (norm-wise), on N = 2..4 and cores of 12 .. 1200;
  * the inverse assembled from the GPU's blocks (Eq. fastblock) against
    (J^T J + mu I)^{-1} from the explicit Jacobian on tiny inputs, 1e-10;
  * the diagonal against the oracle's, 1e-10;
  * the squared angular errors and the matching against the oracle's
    (linear assignment) on noisy, permuted, sign-flipped estimates: the
    permutation exactly, alpha^2 to 1e-12 absolute; MedSAE of a batch of runs.
"""
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
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


CASES = [((3, 4, 5), 2, 0.7), ((5, 6), 3, 1.3), ((4, 3, 5, 3), 2, 0.2), ((12, 13, 14), 5, 0.9),
         ((30, 31, 29), 12, 2.0), ((40, 41, 39), 20, 5.0)]


@pytest.mark.parametrize("dims,R,mu", CASES)
def test_hinv_blocks_match_oracle(cp, dims, R, mu):
    p = synth.make_problem(140 + R, dims, R, snr_db=30, collinearity=(0.5,))
    shape = cp.make_shape(dims, R, "f64")
    a = cp.factors_to_device(p.init)
    Gt, St, info = cp.hinv_blocks(shape, a, mu)
    torch.cuda.synchronize()
    assert info.item() == 0
    N = len(dims)
    n = N * R * R
    Gt_ref, St_ref = O.hinv_blocks(p.init, mu)
    Gt_np = Gt.cpu().numpy().reshape(N, R, R).transpose(0, 2, 1)
    St_np = St.cpu().numpy().reshape(n, n).T
    assert rel(Gt_np, np.stack(Gt_ref)) < 1e-12
    assert rel(St_np, St_ref) < 1e-10
    diag = cp.hinv_diag(shape, a, Gt, St).cpu().numpy()
    assert rel(diag, O.hinv_diag(p.init, Gt_ref, St_ref)) < 1e-10
    if R * sum(dims) <= 80:
        J = O.jacobian(p.init)
        ref = np.linalg.inv(J.T @ J + mu * np.eye(J.shape[1]))
        assert rel(O.hinv_from_blocks(p.init, list(Gt_np), St_np), ref) < 1e-10


@pytest.mark.parametrize("dims,R", [((6, 7, 8), 4), ((20, 21), 9), ((10, 9, 8, 7), 6), ((15, 16, 17), 32)])
def test_sae_matches_oracle(cp, dims, R):
    rng = np.random.default_rng(150 + R)
    A = [rng.standard_normal((I, R)) for I in dims]
    perm = rng.permutation(R)
    est = [(a + 0.3 * rng.standard_normal(a.shape))[:, perm] * rng.choice([-2.0, 0.5, 1.0], R)[None, :]
           for a in A]
    shape = cp.make_shape(dims, R, "f64")
    a2, pi = cp.sae(shape, cp.factors_to_device(A), cp.factors_to_device(est))
    torch.cuda.synchronize()
    a2_ref, pi_ref = O.sae(A, est)
    assert np.array_equal(pi.cpu().numpy(), pi_ref)
    assert np.max(np.abs(a2.cpu().numpy() - a2_ref)) < 1e-12


def test_medsae_over_runs(cp):
    """MedSAE (dB) of several fits of one collinear problem against the true
    factors: the GPU's per-run squared angular errors give the oracle's
    median."""
    p = synth.make_problem(160, (20, 22, 18), 4, snr_db=30, collinearity=(0.7, 0.7, 0.7))
    shape = cp.make_shape(p.dims, p.R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    runs_gpu, runs_ref = [], []
    for seed in range(4):
        A0 = [np.random.default_rng(seed).standard_normal(t.shape) for t in p.true_factors]
        a = cp.factors_to_device(A0)
        st = cp.State(shape, a, mu0=-1.0, tol=1e-9, max_iter=300)
        st.init(Y)
        for _ in range(300):
            st.step(Y)
            if st.status()["stop"] != 0:
                break
        a2, _ = cp.sae(shape, cp.factors_to_device(p.true_factors), a)
        runs_gpu.append(a2.cpu().numpy())
        runs_ref.append(O.sae(p.true_factors, [x.numpy() for x in cp.split_factors(a.cpu(), p.dims, p.R)])[0])
        st.close()
    assert abs(cp.medsae_db(runs_gpu) - O.medsae(runs_ref)) < 1e-9
