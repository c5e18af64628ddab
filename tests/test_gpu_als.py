"""Parity of cp_als_sweep (the ALS rule of Sec. 3, Eq. ALS) with the oracle.

Every input is seeded and synthetic; expected values come from ``oracle/``
only.  Tolerances:
  * float64 tensors: factors within 1e-10 relative (norm-wise) after one
    sweep and 1e-9 after three.  Each mode update solves an R x R system,
    by Cholesky on the GPU and through the pseudo-inverse in the oracle.  The
    seeded factors keep Gamma^(n) well conditioned (I_n >= R, Gaussian
    columns), so the two solves agree to a few hundred ulps.
  * float32 and two-plane bfloat16 tensors (float32 arithmetic in the pass
    over Y): the oracle runs on the same stored values; factors within 1e-4
    relative (MTTKRP error about 1e-6, times the conditioning of Gamma^(n)).
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
    a = np.concatenate([np.ravel(np.asarray(x)) for x in a])
    b = np.concatenate([np.ravel(np.asarray(x)) for x in b])
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_als(cp, p, dtype, sweeps):
    shape = cp.make_shape(p.Y.shape, p.R, dtype)
    Y = cp.tensor_to_device(p.Y, dtype)
    a = cp.factors_to_device(p.init)
    st = cp.State(shape, a, mu0=1.0)
    st.init(Y)
    st.als(Y, sweeps)
    s = st.status()
    got = cp.split_factors(a.cpu(), p.Y.shape, p.R)
    st.close()
    return got, s


def oracle_als(p, sweeps):
    A = [np.array(x) for x in p.init]
    for _ in range(sweeps):
        A = O.als_sweep(p.Y, A)
    return A


# N = 2..4, ragged sizes, R = 1..16, I_1 above one CTA of rows (300)
SHAPES = [((7, 9, 11), 3), ((20, 20, 20), 5), ((13, 6), 4), ((5, 4, 3, 6), 2), ((33, 17, 9), 1),
          ((31, 29, 37), 16), ((300, 8, 7), 6)]


@pytest.mark.parametrize("dims,R", SHAPES)
@pytest.mark.parametrize("sweeps", [1, 3])
def test_als_f64_matches_oracle(cp, dims, R, sweeps):
    p = synth.make_problem(400, dims, R, snr_db=20)
    got, s = run_als(cp, p, "f64", sweeps)
    assert s["error"] == 0
    assert rel(got, oracle_als(p, sweeps)) < (1e-10 if sweeps == 1 else 1e-9)


@pytest.mark.parametrize("dtype,dims,R", [("f32", (40, 30, 20), 4), ("f32", (9, 10, 11, 12), 3),
                                          ("bf16x2", (64, 40, 30), 8)])
def test_als_reduced_precision_tensor_matches_oracle(cp, dtype, dims, R):
    p = synth.make_problem(401, dims, R, dtype=dtype, snr_db=30)
    got, s = run_als(cp, p, dtype, 2)
    assert s["error"] == 0
    assert rel(got, oracle_als(p, 2)) < 1e-4


def test_als_not_positive_definite_keeps_the_mode_and_reports(cp):
    """A zero column in A^(2) and A^(3) makes Gamma^(1) singular: mode 1 keeps
    its factor and the status reports CP_ENOTSPD (pivot 1-based)."""
    p = synth.make_problem(402, (6, 7, 8), 3, snr_db=30)
    p.init[1][:, 2] = 0.0
    p.init[2][:, 2] = 0.0
    shape = cp.make_shape(p.Y.shape, p.R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    a = cp.factors_to_device(p.init)
    st = cp.State(shape, a, mu0=1.0)
    st.init(Y)
    st.als(Y, 1)
    s = st.status()
    got = cp.split_factors(a.cpu(), p.Y.shape, p.R)
    st.close()
    assert s["error"] == 2 and s["info"] == 3
    assert np.array_equal(got[0], p.init[0])


def test_als_invalid_arguments(cp):
    p = synth.make_problem(403, (5, 6, 7), 2, snr_db=30)
    shape = cp.make_shape(p.Y.shape, p.R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    a = cp.factors_to_device(p.init)
    st = cp.State(shape, a, mu0=1.0)
    assert cp._lib.cp_als_sweep(st._h, cp._ptr(Y), 0, None) == 1
    assert cp._lib.cp_als_sweep(None, cp._ptr(Y), 1, None) == 1
    assert cp._lib.cp_als_sweep(st._h, None, 1, None) == 1
    st.close()
