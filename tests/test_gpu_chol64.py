"""The float64 Cholesky factorisation and triangular solves of the core
system (cp_dgn_solve), through the C ABI, against the oracle.

  * f = B_mu w (Theorem 1, Eq. inverse_f1a) against the oracle's fLM_a f to
    1e-10 relative on cores of N R^2 = 12 .. 2700 (one, several and ragged
    32-wide panels; the size of the served large class);
  * the returned lower factor L satisfies L L^T = core to 1e-14 relative
    (norm-wise), checked on the host in float64;
  * a core that is not positive definite reports its first bad pivot
    (1-based) in `info`: -I fails at 1, and a matrix whose leading 37 x 37
    block is SPD but whose 38th pivot is negative fails at 38 (inside the
    second 32-wide panel).
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


CASES = [((5, 6, 7), 2, 0.5), ((12, 13, 11), 5, 1.0), ((30, 31, 29), 10, 0.8), ((8, 9, 7, 6), 3, 0.3),
         ((40, 40, 40), 16, 2.0), ((50, 60, 40), 20, 1.0), ((60, 61, 59), 30, 5.0)]


@pytest.mark.parametrize("dims,R,mu", CASES)
def test_core_solve_matches_oracle(cp, dims, R, mu):
    p = synth.make_problem(120 + R, dims, R, snr_db=30, collinearity=(0.5,))
    shape = cp.make_shape(dims, R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    a = cp.factors_to_device(p.init)
    m, _ = cp.mttkrp_all(shape, Y, a)
    mu_t = torch.tensor([mu], dtype=torch.float64, device="cuda")
    core, Gt, w, info = cp.core_build(shape, a, m, mu_t)
    assert info.item() == 0
    n = len(dims) * R * R
    C = core.cpu().numpy().reshape(n, n).T.copy()
    C = np.tril(C) + np.tril(C, -1).T
    f, info2 = cp.core_solve(shape, a, mu_t, core, w)
    assert info2.item() == 0
    ref = O.flm_step(p.Y, p.init, mu)
    assert rel(f.cpu().numpy(), ref.f) < 1e-10
    L = np.tril(core.cpu().numpy().reshape(n, n).T)
    assert rel(L @ L.T, C) < 1e-14


@pytest.mark.parametrize("N,R,bad", [(2, 5, 1), (3, 6, 38)])
def test_not_positive_definite_reports_pivot(cp, N, R, bad):
    """cp_dgn_solve on a hand-made core of size n = N R^2 whose factorisation
    stops being positive definite at pivot `bad` (1-based): -I at 1; an SPD
    matrix whose pivot 38 has Schur complement -1 (its leading 37 x 37 block
    is SPD) at 38."""
    n = N * R * R
    rng = np.random.default_rng(9)
    X = rng.standard_normal((n, n))
    M = X @ X.T / n + np.eye(n)
    if bad == 1:
        M = -np.eye(n)
    else:
        k = bad - 1
        v = M[k, :k]
        M[k, k] = float(v @ np.linalg.solve(M[:k, :k], v)) - 1.0
    shape = cp.make_shape(tuple([R + 3] * N), R, "f64")
    a = torch.from_numpy(rng.standard_normal(R * (R + 3) * N)).cuda()
    core = torch.from_numpy(np.asfortranarray(M).ravel(order="F").copy()).cuda()
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    mu_t = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    f, info = cp.core_solve(shape, a, mu_t, core, w)
    assert info.item() == bad
