"""cp_spd_invert_f32: the float32 Gauss-Jordan inverse used by the mixed
core solve, against the float64 inverse of the same (float32-rounded) matrix.

Expected values come from numpy's float64 inverse.  Bound: the float32
inverse of an SPD matrix with condition number kappa has relative error
~ n u kappa (u = 6e-8); the test takes 1e-4 * kappa / 10 with kappa computed
in float64 (the matrices are built with kappa ~ 10..100).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_2584_gb300 import cpdgn
    return cpdgn


def spd_with_identity_blocks(n, block, seed, scale=0.45):
    """I + X, X symmetric with zero diagonal blocks of size `block` and
    spectral norm `scale` (< 1, so the matrix is SPD with kappa <= 1.9/0.55)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n))
    X = X + X.T
    if block:
        for b0 in range(0, n, block):
            X[b0:b0 + block, b0:b0 + block] = 0.0
    X *= scale / np.linalg.norm(X, 2)
    return (np.eye(n) + X).astype(np.float32)


def general_spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    return (B @ B.T / n + 0.05 * np.eye(n)).astype(np.float32)


# large cores (the 400^3, R = 30 core is n = 2700) and n % 4 != 0 (scalar operand loads).
# From n = 1024 (n % 4 == 0) a sweep is one launch of 1 + ceil(n / 128)^2 CTAs
# while they fit on the GPU (n <= 1536: 1024, 1100 with a 12-row last pivot
# block, 1200, 1536 with 145 CTAs), else the row-panel launch + update
# (1600: 170 CTAs, 2700).
@pytest.mark.parametrize("n,block,ident", [(1200, 400, 400), (900, 225, 225), (75, 25, 25), (130, 0, 0),
                                           (64, 0, 0), (50, 0, 0), (257, 0, 0), (2700, 900, 900),
                                           (1600, 0, 0), (1537, 0, 0), (1024, 256, 256), (1100, 0, 0),
                                           (1536, 0, 0)])
def test_inverse_matches_float64(cp, n, block, ident):
    M = spd_with_identity_blocks(n, block, 7 + n) if block else general_spd(n, 7 + n)
    ref = np.linalg.inv(M.astype(np.float64))
    kappa = np.linalg.cond(M.astype(np.float64))
    A = torch.from_numpy(np.asfortranarray(M).ravel(order="F").copy()).cuda()
    inv = cp.SpdInverse(n, ident)
    X, info = inv.run(A)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    Xh = X.cpu().numpy().reshape(n, n, order="F").astype(np.float64)
    err = np.linalg.norm(Xh - ref) / np.linalg.norm(ref)
    assert err < 1e-5 * max(kappa, 1.0), (err, kappa)


def test_not_spd_sets_info(cp):
    n = 96
    M = general_spd(n, 3)
    M[70, 70] = -5.0                    # a negative diagonal entry: a pivot must fail
    A = torch.from_numpy(np.asfortranarray(M).ravel(order="F").copy()).cuda()
    _, info = cp.SpdInverse(n, 0).run(A)
    torch.cuda.synchronize()
    assert int(info.item()) > 0


@pytest.mark.parametrize("n,bad", [(1100, 1050), (1200, 700)])
def test_not_spd_sets_info_one_launch_sweeps(cp, n, bad):
    """A failing pivot inside the one-launch sweeps (in block 16 of 18 at
    n = 1100, whose last block has 12 rows; in block 10 of 19 at n = 1200)
    sets info."""
    M = general_spd(n, 5)
    M[bad, bad] = -5.0
    A = torch.from_numpy(np.asfortranarray(M).ravel(order="F").copy()).cuda()
    _, info = cp.SpdInverse(n, 0).run(A)
    torch.cuda.synchronize()
    assert int(info.item()) > 0


def test_invalid_arguments(cp):
    inv = cp.SpdInverse(10, 0)
    A = torch.zeros(100, dtype=torch.float32, device="cuda")
    in_work = cp.ctypes.c_int(0)
    assert cp._lib.cp_spd_invert_f32(10, 11, cp._ptr(A), cp._ptr(inv.work), cp._ptr(inv.pinv), None,
                                     cp.ctypes.byref(in_work), None) == 1
    assert cp._lib.cp_spd_invert_f32(0, 0, cp._ptr(A), cp._ptr(inv.work), cp._ptr(inv.pinv), None,
                                     cp.ctypes.byref(in_work), None) == 1
