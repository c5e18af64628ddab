"""cp_gram_noalloc: the Gramians without a workspace argument.

For callers that cannot allocate device memory, the library offers one call
whose scratch is a fixed array inside the library.  This test calls it
through the C ABI, twice in a row, and checks each result against cp_gram
(the workspace version) within the float64 tolerance the other Gram tests
use.  It also checks that a shape too large for the fixed scratch is
rejected with CP_ENOMEM.  The file name makes pytest collect it last.
"""
import ctypes

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


def _noalloc(cp, shape, a):
    N, R = shape.N, shape.R
    C = torch.full((N * R * R,), float("nan"), dtype=torch.float64, device="cuda")
    Gnm = torch.full((N * N * R * R,), float("nan"), dtype=torch.float64, device="cuda")
    Gall = torch.full((R * R,), float("nan"), dtype=torch.float64, device="cuda")
    rc = cp._lib.cp_gram_noalloc(ctypes.byref(shape), ctypes.c_void_p(a.data_ptr()),
                                 ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(Gnm.data_ptr()),
                                 ctypes.c_void_p(Gall.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, cp.CODES.get(rc, rc)
    torch.cuda.synchronize()
    return C.cpu().numpy(), Gnm.cpu().numpy(), Gall.cpu().numpy()


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


@pytest.mark.parametrize("dims,R", [((7, 9, 11), 3), ((200, 200, 200), 20), ((5, 4, 3, 6), 2)])
def test_noalloc_gram_matches_cp_gram_twice(cp, dims, R):
    rng = np.random.default_rng(4242)
    shape = cp.make_shape(dims, R, "f64")
    results = []
    for call in range(2):                       # two calls in a row share the scratch
        a = torch.from_numpy(rng.standard_normal(R * sum(dims))).cuda()
        C_ref, Gnm_ref, Gall_ref = (t.cpu().numpy() for t in cp.gram(shape, a))
        C, Gnm, Gall = _noalloc(cp, shape, a)
        assert _rel(C, C_ref) < 1e-13
        assert _rel(Gnm, Gnm_ref) < 1e-13
        assert _rel(Gall, Gall_ref) < 1e-13
        results.append(C)
    assert not np.array_equal(results[0], results[1])   # the second call saw its own input


def test_noalloc_rejects_oversized_shape(cp):
    # ceil(I/8) row blocks * R(R+1)/2 doubles exceeds the 2^18-double scratch
    shape = cp.make_shape((20000, 20000), 32, "f64")
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    C = torch.zeros(2 * 32 * 32, dtype=torch.float64, device="cuda")
    rc = cp._lib.cp_gram_noalloc(ctypes.byref(shape), ctypes.c_void_p(a.data_ptr()),
                                 ctypes.c_void_p(C.data_ptr()), None, None,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert cp.CODES[rc] == "CP_ENOMEM"
