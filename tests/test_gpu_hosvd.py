"""HOSVD initialisation (cp_hosvd) and the HOSVD + ALS start of Sec. 4.6,
through the C ABI, against the oracle.

  * every mode's factor against the oracle's (an SVD of the unfolding with
    the same sign convention), entry by entry, to 1e-9, on the tensor values
    the device holds (float64, float32, bfloat16 and two-plane tensors;
    N = 2..4; R < I_n and R = I_n);
  * R > I_n is rejected with CP_EINVAL;
  * the whole initialisation pipeline, HOSVD then two ALS sweeps then the LM
    iteration to its stop rule, in float64, against the oracle's pipeline:
    final epsilon within 1e-10.
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


CASES = [((20, 21, 22), 5, "f64"), ((40, 30, 50), 10, "f32"), ((12, 13, 14, 15), 4, "bf16"),
         ((64, 40, 24), 8, "bf16x2"), ((7, 9), 7, "f64"), ((128, 64, 33), 20, "f32"),
         ((6, 5, 7, 4), 4, "f64")]


@pytest.mark.parametrize("dims,R,dtype", CASES)
def test_hosvd_matches_oracle(cp, dims, R, dtype):
    p = synth.make_problem(60 + R, dims, R, dtype=dtype, snr_db=25)
    shape = cp.make_shape(dims, R, dtype)
    Y = cp.tensor_to_device(p.Y, dtype)
    a = cp.hosvd(shape, Y, iters=40)
    torch.cuda.synchronize()
    got = cp.split_factors(a.cpu(), dims, R)
    ref = O.hosvd_factors(p.Y, R)
    for n in range(len(dims)):
        assert np.max(np.abs(got[n].numpy() - ref[n])) < 1e-9, n


def test_hosvd_rejects_rank_above_a_dimension(cp):
    shape = cp.make_shape((4, 9, 9), 5, "f64")
    Y = torch.zeros(4 * 81, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CPError):
        cp.hosvd(shape, Y)


def test_hosvd_als_lm_pipeline(cp):
    """Sec. 4.6's start (mode-n singular vectors, then ALS sweeps) followed by
    the LM iteration, on a collinear problem."""
    p = synth.make_problem(61, (24, 26, 22), 6, snr_db=30, collinearity=(0.9, 0.8, 0.8))
    shape = cp.make_shape(p.dims, p.R, "f64")
    Y = cp.tensor_to_device(p.Y, "f64")
    a = cp.hosvd(shape, Y, iters=40)
    st = cp.State(shape, a, mu0=-1.0, tol=1e-10, max_iter=500, mu_max=1e30)
    st.als(Y, 2)
    st.init(Y)
    for _ in range(500):
        st.step(Y)
        if st.status()["stop"] != 0:
            break
    s = st.status()
    A0 = O.hosvd_factors(p.Y, p.R)
    A0 = O.als_sweep(p.Y, O.als_sweep(p.Y, A0))
    ref = O.lm_fit(p.Y, A0, mu0=None, max_iter=500, tol=1e-10)
    assert s["stop_reason"] == ref.stop == "tol"
    assert abs(s["rel_err"] - ref.rel_err) <= 1e-10 * ref.rel_err, (s["rel_err"], ref.rel_err)
