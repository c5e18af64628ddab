"""Thin Python binding of ``libcpdgn.so`` (the C ABI in ``include/cpdgn.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch provides device memory and the current CUDA stream.  If
the library has not been built this module raises at import time; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcpdgn.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_1205_2584_gb300.build` (nvcc, sm_103a)")
_lib = ctypes.CDLL(LIB_PATH)

CP_MAX_N = 8
CP_MAX_R = 32
CP_F64, CP_F32, CP_BF16, CP_BF16X2, CP_C128 = 0, 1, 2, 3, 4
CP_CORE_F64, CP_CORE_MIXED = 0, 1
CODES = {0: "CP_OK", 1: "CP_EINVAL", 2: "CP_ENOTSPD", 3: "CP_ENONFINITE", 4: "CP_ETIMEOUT",
         5: "CP_ENOMEM", 6: "CP_ECUDA"}
STOP = {0: "running", 1: "tol", 2: "mu_max", 3: "max_iter", 4: "error"}
DTYPES = {"f64": CP_F64, "f32": CP_F32, "bf16": CP_BF16, "bf16x2": CP_BF16X2, "c128": CP_C128}
# storage dtype of Y; the CP_BF16X2 form holds 2 J bfloat16 values (hi plane, lo plane)
TORCH_DTYPE = {CP_F64: torch.float64, CP_F32: torch.float32, CP_BF16: torch.bfloat16, CP_BF16X2: torch.bfloat16}


class CPError(RuntimeError):
    pass


class Shape(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("R", ctypes.c_int32), ("I", ctypes.c_int64 * CP_MAX_N),
                ("y_dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("mu0", ctypes.c_double), ("tau", ctypes.c_double), ("tol", ctypes.c_double),
                ("mu_max", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("normalize", ctypes.c_int32), ("core_mode", ctypes.c_int32),
                ("refine_iters", ctypes.c_int32)]


class Status(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("nu", ctypes.c_double), ("resid2", ctypes.c_double),
                ("resid2_trial", ctypes.c_double), ("y_norm2", ctypes.c_double),
                ("rel_err", ctypes.c_double), ("rho", ctypes.c_double), ("denom", ctypes.c_double),
                ("refine_resid", ctypes.c_double), ("reserved_d", ctypes.c_double * 3),
                ("iters", ctypes.c_int32), ("accepted", ctypes.c_int32), ("stop", ctypes.c_int32),
                ("error", ctypes.c_int32), ("last_accepted", ctypes.c_int32), ("info", ctypes.c_int32),
                ("refine_sweeps", ctypes.c_int32), ("core_f64", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


assert ctypes.sizeof(Status) == 128

_vp, _sz = ctypes.c_void_p, ctypes.c_size_t
_sig = {
    "cp_workspace_bytes": [ctypes.POINTER(Shape), ctypes.c_int, ctypes.c_int, ctypes.POINTER(_sz)],
    "cp_gram": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp, _sz, _vp],
    "cp_gram_noalloc": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp],
    "cp_mttkrp_all": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp, _sz, _vp],
    "cp_fit": [ctypes.POINTER(Shape), _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _sz, _vp],
    "cp_dgn_core_build": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp],
    "cp_dgn_solve": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp],
    "cp_state_create": [ctypes.POINTER(Shape), ctypes.POINTER(Opts), _vp, _vp, _sz,
                        ctypes.POINTER(_vp)],
    "cp_state_destroy": [_vp],
    "cp_state_init": [_vp, _vp, _vp],
    "cp_dgn_step": [_vp, _vp, _vp],
    "cp_state_capture": [_vp, _vp, ctypes.c_int, _vp],
    "cp_state_launch": [_vp, _vp],
    "cp_als_sweep": [_vp, _vp, ctypes.c_int, _vp],
    "cp_state_graph_kernels": [_vp],
    "cp_batch_run": [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                     ctypes.c_int, _vp, _vp],
    "cp_tensor_split": [_vp, ctypes.c_int64, _vp, _vp],
    "cp_selftest_wait_timeout": [ctypes.c_int64, _vp],
    "cp_hosvd_workspace_bytes": [ctypes.POINTER(Shape), ctypes.POINTER(_sz)],
    "cp_hosvd": [ctypes.POINTER(Shape), _vp, _vp, ctypes.c_int, _vp, _sz, _vp],
    "cp_hinv_workspace_bytes": [ctypes.POINTER(Shape), ctypes.POINTER(_sz)],
    "cp_hinv_blocks": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp],
    "cp_hinv_diag": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp],
    "cp_sae": [ctypes.POINTER(Shape), _vp, _vp, _vp, _vp, _vp],
    "cp_cstate_workspace_bytes": [ctypes.POINTER(Shape), ctypes.POINTER(_sz)],
    "cp_cstate_create": [ctypes.POINTER(Shape), ctypes.POINTER(Opts), _vp, _vp, _sz, ctypes.POINTER(_vp)],
    "cp_cstate_destroy": [_vp],
    "cp_cstate_init": [_vp, _vp, _vp],
    "cp_cdgn_step": [_vp, _vp, _vp],
    "cp_spd_invert_f32": [ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int),
                          _vp],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.cp_state_status.argtypes = [_vp]
_lib.cp_state_status.restype = _vp
_lib.cp_state_buffer.argtypes = [_vp, ctypes.c_int]
_lib.cp_state_buffer.restype = _vp
_lib.cp_cstate_status.argtypes = [_vp]
_lib.cp_cstate_status.restype = _vp
_lib.cp_cstate_buffer.argtypes = [_vp, ctypes.c_int]
_lib.cp_cstate_buffer.restype = _vp


class BatchProblem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("R", ctypes.c_int32), ("I", ctypes.c_int64 * 4),
                ("y_off", ctypes.c_int64), ("a_off", ctypes.c_int64), ("ws_off", ctypes.c_int64),
                ("mu0", ctypes.c_double)]


_lib.cp_batch_check.argtypes = [ctypes.POINTER(BatchProblem)]
_lib.cp_batch_check.restype = ctypes.c_int
_lib.cp_batch_layout.argtypes = [ctypes.POINTER(BatchProblem), ctypes.c_int, ctypes.POINTER(_sz)]
_lib.cp_batch_layout.restype = ctypes.c_int

EXPORTED = list(_sig) + ["cp_state_status", "cp_state_buffer", "cp_batch_check", "cp_batch_layout",
                         "cp_cstate_status", "cp_cstate_buffer"]


def _check(rc: int, what: str):
    if rc != 0:
        raise CPError(f"{what} failed: {CODES.get(rc, rc)}")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_shape(dims: Sequence[int], R: int, y_dtype) -> Shape:
    s = Shape()
    s.N = len(dims)
    s.R = int(R)
    for n, I in enumerate(dims):
        s.I[n] = int(I)
    s.y_dtype = DTYPES[y_dtype] if isinstance(y_dtype, str) else int(y_dtype)
    return s


def workspace_bytes(shape: Shape, core_mode: int = CP_CORE_F64, state: bool = False) -> int:
    out = _sz(0)
    _check(_lib.cp_workspace_bytes(ctypes.byref(shape), core_mode, 1 if state else 0,
                                   ctypes.byref(out)), "cp_workspace_bytes")
    return out.value


def alloc_workspace(shape: Shape, core_mode: int = CP_CORE_F64, state: bool = False,
                    device="cuda") -> torch.Tensor:
    nb = workspace_bytes(shape, core_mode, state)
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device)


def factors_to_device(factors, device="cuda") -> torch.Tensor:
    """Stack I_n x R float64 factors into the parameter vector a (column-major blocks)."""
    parts = [torch.as_tensor(f, dtype=torch.float64).t().contiguous().reshape(-1) for f in factors]
    return torch.cat(parts).to(device)


def split_factors(a: torch.Tensor, dims: Sequence[int], R: int):
    out, off = [], 0
    for I in dims:
        out.append(a[off:off + I * R].reshape(R, I).t())
        off += I * R
    return out


def tensor_to_device(Y, y_dtype: str, device="cuda") -> torch.Tensor:
    """Column-major (first index fastest) device copy of a numpy tensor; for
    "bf16x2" the float32 values are split on the device (cp_tensor_split)."""
    import numpy as np
    flat = np.asarray(Y, dtype=np.float64).ravel(order="F")
    if y_dtype == "bf16x2":
        return tensor_split(torch.from_numpy(flat).to(torch.float32).to(device))
    return torch.from_numpy(flat).to(TORCH_DTYPE[DTYPES[y_dtype]]).to(device)


def tensor_split(y32: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """float32 device tensor (vec order) -> the two-plane bfloat16 form
    [hi plane | lo plane] consumed by CP_BF16X2 shapes."""
    assert y32.dtype == torch.float32 and y32.is_cuda and y32.is_contiguous()
    J = y32.numel()
    if out is None:
        out = torch.empty(2 * J, dtype=torch.bfloat16, device=y32.device)
    _check(_lib.cp_tensor_split(_ptr(y32), J, _ptr(out), _stream(stream)), "cp_tensor_split")
    return out


class SpdInverse:
    """Buffers of cp_spd_invert_f32 for n x n matrices: `run(A)` inverts the
    float32 column-major SPD matrix A in place of its buffer (A is destroyed)
    and returns the device tensor holding the inverse (A's storage or the
    work buffer) and the device pivot flag."""

    def __init__(self, n: int, ident: int = 0, device="cuda"):
        self.n, self.ident = int(n), int(ident)
        self.work = torch.empty(self.n * self.n, dtype=torch.float32, device=device)
        self.pinv = torch.empty(2 * 64 * 64, dtype=torch.float32, device=device)
        self.info = torch.zeros(1, dtype=torch.int32, device=device)

    def run(self, A: torch.Tensor, stream=None):
        assert A.dtype == torch.float32 and A.is_cuda and A.is_contiguous() and A.numel() == self.n * self.n
        in_work = ctypes.c_int(0)
        _check(_lib.cp_spd_invert_f32(self.n, self.ident, _ptr(A), _ptr(self.work), _ptr(self.pinv),
                                      _ptr(self.info), ctypes.byref(in_work), _stream(stream)),
               "cp_spd_invert_f32")
        return (self.work if in_work.value else A), self.info


# ---------------------------------------------------------------------------
# stand-alone calls
# ---------------------------------------------------------------------------

def gram(shape: Shape, a: torch.Tensor, ws=None, stream=None):
    N, R = shape.N, shape.R
    C = torch.empty(N * R * R, dtype=torch.float64, device=a.device)
    Gnm = torch.empty(N * N * R * R, dtype=torch.float64, device=a.device)
    Gall = torch.empty(R * R, dtype=torch.float64, device=a.device)
    ws = ws if ws is not None else alloc_workspace(shape, device=a.device)
    _check(_lib.cp_gram(ctypes.byref(shape), _ptr(a), _ptr(C), _ptr(Gnm), _ptr(Gall), _ptr(ws), ws.numel(),
                        _stream(stream)), "cp_gram")
    return C, Gnm, Gall


def mttkrp_all(shape: Shape, Y: torch.Tensor, a: torch.Tensor, want_resid=True, ws=None, stream=None):
    m = torch.empty_like(a)
    r2 = torch.empty(1, dtype=torch.float64, device=a.device) if want_resid else None
    ws = ws if ws is not None else alloc_workspace(shape)
    _check(_lib.cp_mttkrp_all(ctypes.byref(shape), _ptr(Y), _ptr(a), _ptr(m), _ptr(r2), _ptr(ws),
                              ws.numel(), _stream(stream)), "cp_mttkrp_all")
    return m, r2


def fit(shape: Shape, Y: torch.Tensor, a: torch.Tensor, y_norm2: float = 0.0, ws=None, stream=None):
    r2 = torch.empty(1, dtype=torch.float64, device=a.device)
    rel = torch.empty(1, dtype=torch.float64, device=a.device)
    ws = ws if ws is not None else alloc_workspace(shape)
    _check(_lib.cp_fit(ctypes.byref(shape), _ptr(Y), _ptr(a), ctypes.c_double(y_norm2), _ptr(r2),
                       _ptr(rel), _ptr(ws), ws.numel(), _stream(stream)), "cp_fit")
    return r2, rel


def core_build(shape: Shape, a: torch.Tensor, m: torch.Tensor, mu: torch.Tensor, ws=None, stream=None):
    N, R = shape.N, shape.R
    n = N * R * R
    core = torch.zeros(n * n, dtype=torch.float64, device=a.device)
    Gt = torch.empty(N * R * R, dtype=torch.float64, device=a.device)
    w = torch.empty(n, dtype=torch.float64, device=a.device)
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    ws = ws if ws is not None else alloc_workspace(shape)
    _check(_lib.cp_dgn_core_build(ctypes.byref(shape), _ptr(a), _ptr(m), _ptr(mu), _ptr(core), _ptr(Gt),
                                  _ptr(w), _ptr(info), _ptr(ws), ws.numel(), _stream(stream)),
           "cp_dgn_core_build")
    return core, Gt, w, info


def core_solve(shape: Shape, a: torch.Tensor, mu: torch.Tensor, core: torch.Tensor, w: torch.Tensor,
               ws=None, stream=None):
    f = torch.empty_like(w)
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    ws = ws if ws is not None else alloc_workspace(shape)
    _check(_lib.cp_dgn_solve(ctypes.byref(shape), _ptr(a), _ptr(mu), _ptr(core), _ptr(w), _ptr(f),
                             _ptr(info), _ptr(ws), ws.numel(), _stream(stream)), "cp_dgn_solve")
    return f, info


# ---------------------------------------------------------------------------
# device-resident LM state
# ---------------------------------------------------------------------------

class State:
    """One decomposition whose factors, damping and counters live on the GPU."""

    BUF_M, BUF_DELTA, BUF_GT, BUF_W, BUF_F, BUF_AT = range(6)

    def __init__(self, shape: Shape, a: torch.Tensor, *, mu0: float = -1.0, tau: float = 1e-3,
                 tol: float = 0.0, mu_max: float = 1e30, max_iter: int = 1000, normalize: bool = True,
                 core_mode: int = CP_CORE_F64, refine_iters: int = 8):
        assert a.dtype == torch.float64 and a.is_cuda and a.is_contiguous()
        self.shape = shape
        self.a = a
        self.opts = Opts(mu0=mu0, tau=tau, tol=tol, mu_max=mu_max, max_iter=max_iter,
                         normalize=1 if normalize else 0, core_mode=core_mode, refine_iters=refine_iters)
        self.ws = alloc_workspace(shape, core_mode, state=True, device=a.device)
        h = ctypes.c_void_p()
        _check(_lib.cp_state_create(ctypes.byref(shape), ctypes.byref(self.opts), _ptr(a), _ptr(self.ws),
                                    self.ws.numel(), ctypes.byref(h)), "cp_state_create")
        self._h = h
        self._status_ptr = _lib.cp_state_status(h)
        # the state's buffer 0 holds the gradient blocks G_n = E_(n) KR_n for
        # every tensor form except the two-plane one (whose pass gives M_n)
        self.holds_gradient = shape.y_dtype != CP_BF16X2
        self._host_status = torch.empty(128, dtype=torch.uint8).pin_memory()

    def init(self, Y: torch.Tensor, stream=None):
        _check(_lib.cp_state_init(self._h, _ptr(Y), _stream(stream)), "cp_state_init")

    def step(self, Y: torch.Tensor, stream=None):
        _check(_lib.cp_dgn_step(self._h, _ptr(Y), _stream(stream)), "cp_dgn_step")

    def capture(self, Y: torch.Tensor, steps: int, stream=None):
        """Capture `steps` steps into the state's CUDA graph (nothing runs)."""
        _check(_lib.cp_state_capture(self._h, _ptr(Y), int(steps), _stream(stream)), "cp_state_capture")
        return _lib.cp_state_graph_kernels(self._h)

    def launch(self, stream=None):
        _check(_lib.cp_state_launch(self._h, _stream(stream)), "cp_state_launch")

    def als(self, Y: torch.Tensor, sweeps: int = 1, stream=None):
        """`sweeps` ALS sweeps on the factors (cp_als_sweep); call init(Y)
        before the next step."""
        _check(_lib.cp_als_sweep(self._h, _ptr(Y), int(sweeps), _stream(stream)), "cp_als_sweep")

    @property
    def graph_kernels(self) -> int:
        return _lib.cp_state_graph_kernels(self._h)

    def status_tensor(self) -> torch.Tensor:
        """Device view (128 bytes) of the state's cp_status."""
        off = self._status_ptr - self.ws.data_ptr()
        return self.ws[off:off + 128]

    def status(self, stream=None) -> dict:
        """Synchronous read of the device status (copies 128 bytes)."""
        st = stream if stream is not None else torch.cuda.current_stream()
        self._host_status.copy_(self.status_tensor(), non_blocking=True)
        st.synchronize()
        s = Status.from_buffer_copy(bytes(self._host_status.numpy()))
        d = s.as_dict()
        d["stop_reason"] = STOP.get(d["stop"], d["stop"])
        return d

    def buffer(self, which: int, count: int) -> torch.Tensor:
        p = _lib.cp_state_buffer(self._h, which)
        off = p - self.ws.data_ptr()
        return self.ws[off:off + 8 * count].view(torch.float64)

    def close(self):
        if self._h:
            _lib.cp_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------

class Batch:
    """Many small decompositions (float32 tensors) run by one persistent launch.

    problems: list of (Y numpy array float32-representable, factors list, mu0).
    Packs tensors, factors and workspace on the device; status stays there.
    """

    def __init__(self, problems, *, tol=0.0, mu_max=1e30, max_iter=1000, normalize=True, tau=1e-3,
                 refine_iters=4, device="cuda"):
        import numpy as np
        count = len(problems)
        arr = (BatchProblem * max(count, 1))()
        ys, afs = [], []
        yoff = aoff = 0
        self.meta = []
        for i, (Y, factors, mu0) in enumerate(problems):
            dims = Y.shape
            R = factors[0].shape[1]
            p = arr[i]
            p.N = len(dims)
            p.R = R
            for k in range(4):
                p.I[k] = int(dims[k]) if k < len(dims) else 1
            p.y_off = yoff
            p.a_off = aoff
            p.mu0 = float(mu0) if mu0 else -1.0
            ys.append(np.asarray(Y, dtype=np.float32).ravel(order="F"))
            afs.append(np.concatenate([np.asarray(f, dtype=np.float64).ravel(order="F") for f in factors]))
            self.meta.append((tuple(int(d) for d in dims), R, aoff))
            yoff += ys[-1].size
            aoff += afs[-1].size
            _check(_lib.cp_batch_check(ctypes.byref(p)), f"cp_batch_check(problem {i})")
        nbytes = _sz(0)
        _check(_lib.cp_batch_layout(arr, count, ctypes.byref(nbytes)), "cp_batch_layout")
        self.count = count
        self.Y = torch.from_numpy(np.concatenate(ys) if ys else np.zeros(1, np.float32)).to(device)
        self.a = torch.from_numpy(np.concatenate(afs) if afs else np.zeros(1)).to(device)
        self.a0 = self.a.clone()
        self.ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=device)
        raw = bytes(memoryview(arr)[: ctypes.sizeof(BatchProblem) * max(count, 1)])
        self.probs = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
        self.status = torch.zeros(max(count, 1) * 128, dtype=torch.uint8, device=device)
        self.opts = Opts(mu0=-1.0, tau=tau, tol=tol, mu_max=mu_max, max_iter=max_iter,
                         normalize=1 if normalize else 0, core_mode=CP_CORE_MIXED, refine_iters=refine_iters)

    def run(self, trials: int = 1 << 30, ctas: int = 0, tile: int = 0, order=None, stream=None):
        """One persistent launch.  tile / order: tuning knobs (see cp_batch_run);
        `order` may be a device int32 tensor, or "cost" for most-expensive-first."""
        if isinstance(order, str) and order == "cost":
            order = self.cost_order()
        _check(_lib.cp_batch_run(_ptr(self.probs), self.count, _ptr(self.Y), _ptr(self.a), _ptr(self.ws),
                                 _ptr(self.status), ctypes.byref(self.opts), int(trials), int(ctas), int(tile),
                                 _ptr(order), _stream(stream)), "cp_batch_run")

    def capture(self, trials: int = 1 << 30, tile: int = 0, order=None, ctas: int = 0):
        """Capture one persistent launch (queue reset + kernel) in a CUDA graph;
        returns the torch.cuda.CUDAGraph (replay() runs it on the current stream)."""
        self.run(trials=1, tile=tile, order=order, ctas=ctas)   # sets the kernel's shared-memory attribute
        torch.cuda.synchronize()
        self.reset()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(trials=trials, tile=tile, order=order, ctas=ctas)
        return g

    def cost_order(self):
        """Queue order with the most expensive problems first (longest-processing-
        time-first list scheduling); cost ~ (N R^2)^3 / 3 + 3 R prod(I)."""
        import numpy as np
        if getattr(self, "_cost_order", None) is None:
            cost = []
            for dims, R, _ in self.meta:
                n = len(dims) * R * R
                cost.append(n ** 3 / 3.0 + 3.0 * R * float(np.prod(dims)))
            idx = np.argsort(-np.asarray(cost), kind="stable").astype(np.int32)
            self._cost_order = torch.from_numpy(idx).to(self.Y.device)
        return self._cost_order

    def reset(self):
        """Back to the starting factors and a zeroed status (queue order kept)."""
        self.a.copy_(self.a0)
        self.status.zero_()

    def run_tuned(self, trials: int = 1 << 30, stream=None, tune_trials: int = 2):
        """Tune (or reuse the cached tuning for these shapes), then run."""
        from . import autotune
        cfg = autotune.tune_batch(self, trials=tune_trials, stream=stream)
        self.run(trials=trials, tile=cfg["tile"], order=None if cfg["order"] == "given" else "cost",
                 ctas=cfg["ctas"], stream=stream)
        return cfg

    def statuses(self):
        raw = self.status.cpu().numpy().tobytes()
        out = []
        for i in range(self.count):
            d = Status.from_buffer_copy(raw[128 * i:128 * (i + 1)]).as_dict()
            d["stop_reason"] = STOP.get(d["stop"], d["stop"])
            out.append(d)
        return out

    def factors(self, i: int):
        dims, R, aoff = self.meta[i]
        return split_factors(self.a[aoff:aoff + R * sum(dims)].cpu(), dims, R)


def selftest_wait_timeout(limit_ns: int = 1_000_000, stream=None):
    """cp_selftest_wait_timeout: one bounded device wait that runs out (see the header)."""
    _check(_lib.cp_selftest_wait_timeout(int(limit_ns), _stream(stream)), "cp_selftest_wait_timeout")


def hosvd(shape: Shape, Y: torch.Tensor, a: Optional[torch.Tensor] = None, iters: int = 30, stream=None):
    """cp_hosvd: HOSVD initial factors into `a` (allocated if None); returns a."""
    R = shape.R
    T = sum(shape.I[n] for n in range(shape.N))
    if a is None:
        a = torch.empty(R * T, dtype=torch.float64, device=Y.device)
    nb = _sz(0)
    _check(_lib.cp_hosvd_workspace_bytes(ctypes.byref(shape), ctypes.byref(nb)), "cp_hosvd_workspace_bytes")
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=Y.device)
    _check(_lib.cp_hosvd(ctypes.byref(shape), _ptr(Y), _ptr(a), int(iters), _ptr(ws), ws.numel(), _stream(stream)),
           "cp_hosvd")
    return a


def hinv_blocks(shape: Shape, a: torch.Tensor, mu: float, stream=None):
    """cp_hinv_blocks: Theorem 4's (Gt, St) of (J^T J + mu I)^{-1} at `a`;
    returns (Gt, St, info) device tensors."""
    N, R = shape.N, shape.R
    n = N * R * R
    Gt = torch.empty(N * R * R, dtype=torch.float64, device=a.device)
    St = torch.empty(n * n, dtype=torch.float64, device=a.device)
    info = torch.zeros(1, dtype=torch.int32, device=a.device)
    mu_t = torch.tensor([float(mu)], dtype=torch.float64, device=a.device)
    nb = _sz(0)
    _check(_lib.cp_hinv_workspace_bytes(ctypes.byref(shape), ctypes.byref(nb)), "cp_hinv_workspace_bytes")
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=a.device)
    _check(_lib.cp_hinv_blocks(ctypes.byref(shape), _ptr(a), _ptr(mu_t), _ptr(Gt), _ptr(St), _ptr(info), _ptr(ws),
                               ws.numel(), _stream(stream)), "cp_hinv_blocks")
    return Gt, St, info


def hinv_diag(shape: Shape, a: torch.Tensor, Gt: torch.Tensor, St: torch.Tensor, stream=None):
    out = torch.empty_like(a)
    _check(_lib.cp_hinv_diag(ctypes.byref(shape), _ptr(a), _ptr(Gt), _ptr(St), _ptr(out), _stream(stream)),
           "cp_hinv_diag")
    return out


def sae(shape: Shape, a_true: torch.Tensor, a_est: torch.Tensor, stream=None):
    """cp_sae: (alpha2 as N x R, perm) device tensors."""
    alpha2 = torch.empty(shape.N * shape.R, dtype=torch.float64, device=a_true.device)
    perm = torch.empty(shape.R, dtype=torch.int32, device=a_true.device)
    _check(_lib.cp_sae(ctypes.byref(shape), _ptr(a_true), _ptr(a_est), _ptr(alpha2), _ptr(perm), _stream(stream)),
           "cp_sae")
    return alpha2.view(shape.N, shape.R), perm


def medsae_db(alpha2_runs) -> float:
    """MedSAE (dB): 10 log10 of the median of the squared angular errors of
    every run given (host-side reduction of cp_sae outputs)."""
    import math
    import numpy as np
    v = np.concatenate([np.ravel(torch.as_tensor(x).double().cpu().numpy()) for x in alpha2_runs])
    return 10.0 * math.log10(float(np.median(v)))


# ---------------------------------------------------------------------------
# complex-valued tensors (cp_cstate_*)
# ---------------------------------------------------------------------------

def ctensor_to_device(Y, device="cuda") -> torch.Tensor:
    """Complex numpy tensor -> complex128 device vector in vec order (first index fastest)."""
    import numpy as np
    flat = np.asarray(Y, dtype=np.complex128).ravel(order="F")
    return torch.from_numpy(flat.copy()).to(device)


def cfactors_to_device(factors, device="cuda") -> torch.Tensor:
    parts = [torch.as_tensor(f, dtype=torch.complex128).t().contiguous().reshape(-1) for f in factors]
    return torch.cat(parts).to(device)


class CState:
    """One complex decomposition whose factors, damping and counters live on the GPU."""

    BUF_G, BUF_DELTA, BUF_AT = 0, 1, 5

    def __init__(self, shape: Shape, a: torch.Tensor, *, mu0: float = -1.0, tau: float = 1e-3, tol: float = 0.0,
                 mu_max: float = 1e30, max_iter: int = 1000, normalize: bool = True):
        assert a.dtype == torch.complex128 and a.is_cuda and a.is_contiguous()
        self.shape, self.a = shape, a
        self.opts = Opts(mu0=mu0, tau=tau, tol=tol, mu_max=mu_max, max_iter=max_iter,
                         normalize=1 if normalize else 0, core_mode=CP_CORE_F64, refine_iters=0)
        nb = _sz(0)
        _check(_lib.cp_cstate_workspace_bytes(ctypes.byref(shape), ctypes.byref(nb)), "cp_cstate_workspace_bytes")
        self.ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=a.device)
        h = ctypes.c_void_p()
        _check(_lib.cp_cstate_create(ctypes.byref(shape), ctypes.byref(self.opts), _ptr(a), _ptr(self.ws),
                                     self.ws.numel(), ctypes.byref(h)), "cp_cstate_create")
        self._h = h
        self._status_ptr = _lib.cp_cstate_status(h)
        self._host_status = torch.empty(128, dtype=torch.uint8).pin_memory()

    def init(self, Y, stream=None):
        _check(_lib.cp_cstate_init(self._h, _ptr(Y), _stream(stream)), "cp_cstate_init")

    def step(self, Y, stream=None):
        _check(_lib.cp_cdgn_step(self._h, _ptr(Y), _stream(stream)), "cp_cdgn_step")

    def status(self, stream=None) -> dict:
        st = stream if stream is not None else torch.cuda.current_stream()
        off = self._status_ptr - self.ws.data_ptr()
        self._host_status.copy_(self.ws[off:off + 128], non_blocking=True)
        st.synchronize()
        d = Status.from_buffer_copy(bytes(self._host_status.numpy())).as_dict()
        d["stop_reason"] = STOP.get(d["stop"], d["stop"])
        return d

    def buffer(self, which: int, count: int) -> torch.Tensor:
        p = _lib.cp_cstate_buffer(self._h, which)
        off = p - self.ws.data_ptr()
        return self.ws[off:off + 16 * count].view(torch.complex128)

    def close(self):
        if self._h:
            _lib.cp_cstate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
