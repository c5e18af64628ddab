"""Serving loop: continuous batching of CP decompositions on one GPU.

Requests arrive over time; each names a tensor (or a seed to synthesise one),
a rank and initial factors.  Every admitted request keeps its tensor,
factors, damping and counters on the device until its stop rule fires:

  * lanes: requests small enough for the batched kernel go to the first lane
    whose size class holds them.  A lane owns a stream, a table of problem
    descriptors and statuses, and draws each request's tensor, factors and
    workspace from one device arena.  A lane advances in rounds: one
    persistent launch (`cp_batch_run`) runs up to `trials` Levenberg-Marquardt
    trials of every active request; between rounds stopped requests are
    retired (factors copied out, arena space freed) and waiting requests
    admitted.  Requests therefore join and leave while others are on the
    device, and the lanes run concurrently on their streams.
  * large requests (outside every lane's class) each run on a device-resident
    `cpdgn.State` (mixed core mode) with a stream of its own; each of their
    rounds is one CUDA graph of `steps` damped Gauss-Newton steps.  States
    are kept per tensor shape and re-armed for the next request of that
    shape, so the graph is captured once per shape.

Admission is by HBM budget: lane requests must fit the arena (first fit) and
a free descriptor slot; a large request needs a free State of its shape, or
room for a new one in what the budget leaves after the arena (idle States of
other shapes are dropped to make room), and at most `large_slots` run at
once.  Waiting requests are admitted in arrival order per class.
Time-to-fit = the moment the host sees the stop flag minus the arrival time.

The batched kernel has a fixed reduction order per problem, runs one
problem per CTA and continues bit-identically across launches, so a lane
request's result does not depend on what else is in flight: alone or in a
mix it is the same to the bit.  Large requests agree to rounding (their
cross-CTA sums use atomics).
"""
from __future__ import annotations

import bisect
import ctypes
import dataclasses
import math
import time
from typing import Dict, List, Optional, Sequence

import numpy as np

_ALIGN = 256
_PARKED = 3     # stop code kept by free descriptor slots (the kernel skips them)
MAX_LARGE = 16  # large requests at once when their number is bounded by the budget alone


# ---------------------------------------------------------------------------
# host-side pieces (no GPU needed)
# ---------------------------------------------------------------------------

class Arena:
    """First-fit allocator over [base, base + size) in `align`-byte units,
    with coalescing of neighbouring free blocks.  Offsets only; the caller
    owns the memory."""

    def __init__(self, size: int, base: int = 0, align: int = _ALIGN):
        self.align = align
        self.base = base
        self.size = size // align * align
        self._free: List[List[int]] = [[base, self.size]] if self.size > 0 else []
        self._used: Dict[int, int] = {}

    @property
    def used(self) -> int:
        return sum(self._used.values())

    def alloc(self, nbytes: int) -> Optional[int]:
        need = max(self.align, (int(nbytes) + self.align - 1) // self.align * self.align)
        for k, (off, sz) in enumerate(self._free):
            if sz >= need:
                if sz == need:
                    del self._free[k]
                else:
                    self._free[k] = [off + need, sz - need]
                self._used[off] = need
                return off
        return None

    def free(self, off: int):
        sz = self._used.pop(off)
        k = bisect.bisect_left(self._free, [off, 0])
        self._free.insert(k, [off, sz])
        if k + 1 < len(self._free) and self._free[k][0] + self._free[k][1] == self._free[k + 1][0]:
            self._free[k][1] += self._free[k + 1][1]
            del self._free[k + 1]
        if k > 0 and self._free[k - 1][0] + self._free[k - 1][1] == self._free[k][0]:
            self._free[k - 1][1] += self._free[k][1]
            del self._free[k]

    def largest_free(self) -> int:
        return max((sz for _, sz in self._free), default=0)


def _rnd(x: int) -> int:
    return (int(x) + _ALIGN - 1) // _ALIGN * _ALIGN


@dataclasses.dataclass
class Request:
    """One decomposition request.  Y (numpy, float32-representable, shape
    `dims`) and init (list of I_n x R arrays) are given, or synthesised on the
    device from `seed` (rank-R model, mode-1 collinearity c, noise at snr_db,
    N(0,1) initial factors)."""
    rid: int
    arrival: float
    dims: tuple
    R: int
    seed: int = 0
    collinearity: float = 0.0
    snr_db: Optional[float] = 30.0
    Y: Optional[np.ndarray] = None
    init: Optional[list] = None

    @property
    def cost(self) -> float:
        return float(self.R) * float(np.prod(self.dims))


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    status: dict
    factors: list
    path: str

    @property
    def time_to_fit(self) -> float:
        return self.done - self.arrival


def poisson_requests(seed: int = 0, rate: float = 200.0, seconds: float = 60.0) -> List[Request]:
    """Poisson arrivals at `rate` per second for `seconds`: 70 % 32^3 R=5,
    25 % 128^3 R=16, 5 % 400^3 R=30; mode-1 collinearity ~ U[0, 0.95]; SNR 30 dB."""
    from .synth import config5_requests
    return [Request(rid=k, arrival=t, dims=tuple(dims), R=R, seed=s, collinearity=c, snr_db=30.0)
            for k, (t, s, dims, R, c) in enumerate(config5_requests(seed, rate, seconds))]


def summarize(results: List[Result], wall: float) -> dict:
    """p50 / p99 / mean time-to-fit (overall and per shape class), throughput.
    Per class the time-to-fit is also split into its queue part (arrival to
    admission: waiting for a slot, arena space or HBM budget) and its run
    part (admission to the stop flag being seen on the host)."""
    ttf = np.array([r.time_to_fit for r in results]) if results else np.zeros(1)
    trials = sum(r.status["iters"] for r in results)
    by: Dict[str, List[Result]] = {}
    for r in results:
        key = "x".join(map(str, r.status["dims"])) + f"-R{r.status['R']}"
        by.setdefault(key, []).append(r)

    def cls(v: List[Result]) -> dict:
        t = np.array([r.time_to_fit for r in v])
        q = np.array([r.admitted - r.arrival for r in v])
        u = np.array([r.done - r.admitted for r in v])
        it = np.array([r.status["iters"] for r in v], dtype=float)
        return {"n": len(v), "p50_s": float(np.percentile(t, 50)), "p99_s": float(np.percentile(t, 99)),
                "queue_p50_s": float(np.percentile(q, 50)), "queue_p99_s": float(np.percentile(q, 99)),
                "run_p50_s": float(np.percentile(u, 50)), "run_p99_s": float(np.percentile(u, 99)),
                "iters_p50": float(np.percentile(it, 50)), "iters_p99": float(np.percentile(it, 99))}

    return {"requests": len(results), "p50_s": float(np.percentile(ttf, 50)),
            "p99_s": float(np.percentile(ttf, 99)), "mean_s": float(ttf.mean()),
            "throughput_req_s": len(results) / wall if wall > 0 else 0.0,
            "trials_per_s": trials / wall if wall > 0 else 0.0,
            "by_class": {k: cls(v) for k, v in sorted(by.items())}}


# ---------------------------------------------------------------------------
# device side
# ---------------------------------------------------------------------------

def _cp():
    from . import cpdgn
    return cpdgn


def _desc(dims: Sequence[int], R: int):
    cp = _cp()
    p = cp.BatchProblem()
    p.N = len(dims)
    p.R = int(R)
    for k in range(4):
        p.I[k] = int(dims[k]) if k < len(dims) else 1
    p.mu0 = -1.0
    return p


def lane_bytes(dims: Sequence[int], R: int) -> Optional[int]:
    """Arena bytes of one lane request (tensor + factors + workspace), or
    None when the batched kernel does not take the shape."""
    cp = _cp()
    if len(dims) > 4:
        return None
    p = (cp.BatchProblem * 1)(_desc(dims, R))
    nb = cp._sz(0)
    if cp._lib.cp_batch_layout(p, 1, ctypes.byref(nb)) != 0:
        return None
    return _rnd(4 * int(np.prod(dims))) + _rnd(8 * R * int(sum(dims))) + _rnd(nb.value - _ALIGN)


def state_bytes(dims: Sequence[int], R: int) -> int:
    """Device bytes of one large request: tensor, factors, State workspace."""
    cp = _cp()
    shape = cp.make_shape(dims, R, "bf16x2" if two_plane_ok(dims, R) else "f32")
    return 4 * int(np.prod(dims)) + 8 * R * int(sum(dims)) + cp.workspace_bytes(shape, cp.CP_CORE_MIXED, True)


def synth_on_device(req: Request, device, dtype=None):
    """Seeded request tensor and initial factors built on the device (torch
    Philox generator), standing in for a client's upload.  Returns (y, a):
    y = vec(Y) (first index fastest) in `dtype` (float32 by default),
    a = float64 packed factors."""
    import torch
    dtype = torch.float32 if dtype is None else dtype
    g = torch.Generator(device=device).manual_seed(int(req.seed))
    facs = []
    for n, I in enumerate(req.dims):
        z = torch.randn(I, req.R, generator=g, device=device, dtype=torch.float64)
        if n == 0 and req.collinearity > 0:
            b = torch.randn(I, 1, generator=g, device=device, dtype=torch.float64)
            z = math.sqrt(req.collinearity) * b + math.sqrt(1.0 - req.collinearity) * z
        facs.append(z)
    letters = "abcdefgh"[:len(req.dims)]
    Y = torch.einsum(",".join(f"{l}z" for l in letters) + "->" + letters, *facs)
    if req.snr_db is not None:
        sigma = 10.0 ** (-req.snr_db / 20.0) * torch.linalg.vector_norm(Y) / math.sqrt(Y.numel())
        Y = Y + sigma * torch.randn(Y.shape, generator=g, device=device, dtype=torch.float64)
    y = Y.permute(*reversed(range(Y.dim()))).contiguous().reshape(-1).to(dtype)
    a = torch.cat([torch.randn(I, req.R, generator=g, device=device, dtype=torch.float64).t().reshape(-1)
                   for I in req.dims])
    return y, a


def two_plane_ok(dims: Sequence[int], R: int) -> bool:
    """Shapes whose State runs on the two-plane bfloat16 tensor (tensor-core pass)."""
    return len(dims) == 3 and int(dims[0]) % 8 == 0 and R <= 32


def _inputs(req: Request, device):
    import torch
    if req.Y is None:
        return synth_on_device(req, device)
    y = torch.from_numpy(np.asarray(req.Y, dtype=np.float32).ravel(order="F").copy()).to(device)
    a = torch.from_numpy(np.concatenate([np.asarray(f, np.float64).ravel(order="F") for f in req.init])).to(device)
    return y, a


class _Lane:
    """One size class of lane requests: descriptor slots, statuses, a stream
    and rounds of `cp_batch_run` over the server's arena."""

    def __init__(self, server, idx: int, max_cost: float, slots: int, trials: int, tile: int):
        import torch
        cp = _cp()
        self.srv = server
        self.max_cost = max_cost
        self.slots = slots
        self.trials = trials
        self.tile = tile
        dev = server.device
        # lanes hold many short requests: their rounds go first when SMs free up
        self.stream = torch.cuda.Stream(device=dev, priority=-1)
        self.ws_base = idx * _ALIGN                 # this lane's queue counter
        self.desc = (cp.BatchProblem * slots)()
        for s in range(slots):
            self.desc[s] = _desc((1, 1), 1)
        self.desc_host = torch.empty(slots * ctypes.sizeof(cp.BatchProblem), dtype=torch.uint8).pin_memory()
        self.desc_dev = torch.empty(self.desc_host.numel(), dtype=torch.uint8, device=dev)
        self.order_host = torch.empty(slots, dtype=torch.int32).pin_memory()
        self.order_dev = torch.empty(slots, dtype=torch.int32, device=dev)
        st = np.zeros((slots, 128), np.uint8)
        so = cp.Status.stop.offset
        st[:, so:so + 4] = np.frombuffer(np.int32(_PARKED).tobytes(), np.uint8)
        self.status = torch.from_numpy(st.reshape(-1)).to(dev)
        self.status_host = torch.empty(slots * 128, dtype=torch.uint8).pin_memory()
        self.free = list(range(slots - 1, -1, -1))
        self.active: Dict[int, dict] = {}
        self.event = None
        self.rounds = 0

    def try_admit(self, req: Request, now: float) -> bool:
        import torch
        if not self.free:
            return False
        nb = lane_bytes(req.dims, req.R)
        off = self.srv.arena.alloc(nb)
        if off is None:
            return False
        s = self.free.pop()
        J = int(np.prod(req.dims))
        d = _desc(req.dims, req.R)
        oy = off
        oa = oy + _rnd(4 * J)
        ow = oa + _rnd(8 * req.R * int(sum(req.dims)))
        d.y_off, d.a_off, d.ws_off = oy // 4, oa // 8, ow - self.ws_base
        self.desc[s] = d
        buf = self.srv.buf
        with torch.cuda.stream(self.stream):
            y, a = _inputs(req, self.srv.device)
            buf[oy:oy + 4 * J].view(torch.float32).copy_(y)
            buf[oa:oa + 8 * a.numel()].view(torch.float64).copy_(a)
            self.status[s * 128:(s + 1) * 128].zero_()
        self.active[s] = {"req": req, "off": off, "a_off": oa, "admitted": now}
        return True

    def launch(self):
        import torch
        cp = _cp()
        raw = bytes(memoryview(self.desc)[:ctypes.sizeof(self.desc)])
        self.desc_host.numpy()[:] = np.frombuffer(raw, np.uint8)
        act = sorted(self.active, key=lambda s: -self.active[s]["req"].cost)   # most expensive first
        rest = sorted(set(range(self.slots)) - set(act))
        self.order_host.numpy()[:] = np.asarray(act + rest, np.int32)
        buf = self.srv.buf
        with torch.cuda.stream(self.stream):
            self.desc_dev.copy_(self.desc_host, non_blocking=True)
            self.order_dev.copy_(self.order_host, non_blocking=True)
            cp._check(cp._lib.cp_batch_run(
                cp._ptr(self.desc_dev), self.slots, cp._ptr(buf), cp._ptr(buf),
                ctypes.c_void_p(buf.data_ptr() + self.ws_base), cp._ptr(self.status),
                ctypes.byref(self.srv.opts), int(self.trials), 0, int(self.tile), cp._ptr(self.order_dev),
                cp._stream(self.stream)), "cp_batch_run")
            self.status_host.copy_(self.status, non_blocking=True)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)
        self.rounds += 1

    def harvest(self, now_fn) -> List[Result]:
        """After a round: retire the stopped requests (factors copied out;
        the slot keeps its stop code, so the kernel skips it until reuse)."""
        import torch
        cp = _cp()
        out = []
        raw = self.status_host.numpy().tobytes()
        for s in sorted(self.active):
            d = cp.Status.from_buffer_copy(raw[128 * s:128 * (s + 1)]).as_dict()
            if d["stop"] == 0:
                continue
            e = self.active.pop(s)
            req = e["req"]
            nA = req.R * int(sum(req.dims))
            a = self.srv.buf[e["a_off"]:e["a_off"] + 8 * nA].view(torch.float64).cpu()
            d["stop_reason"] = cp.STOP.get(d["stop"], d["stop"])
            d["dims"], d["R"] = tuple(req.dims), req.R
            self.srv.arena.free(e["off"])
            self.desc[s] = _desc((1, 1), 1)
            self.free.append(s)
            out.append(Result(req.rid, req.arrival, e["admitted"], now_fn(), d,
                              cp.split_factors(a, req.dims, req.R), "lane"))
        return out


class _StateSlot:
    """A device-resident `State` for one tensor shape (its own stream, tensor
    and factor buffers, and a captured graph of `steps` steps).  A slot is
    re-armed for each request of its shape: the request's tensor and factors
    are copied into the slot's buffers and the state is re-initialised, so
    the captured graph is reused.  Where the shape allows, the tensor is held
    as two bfloat16 planes (split once at admission) for the tensor-core pass."""

    def __init__(self, server, dims, R):
        import torch
        cp = _cp()
        self.dims, self.R = tuple(dims), int(R)
        self.bytes = state_bytes(dims, R)
        self.two_plane = two_plane_ok(dims, R)
        dev = server.device
        self.stream = torch.cuda.Stream(device=dev)
        o = server.opts
        J = int(np.prod(dims))
        with torch.cuda.stream(self.stream):
            if self.two_plane:
                self.y = torch.zeros(2 * J, dtype=torch.bfloat16, device=dev)
            else:
                self.y = torch.zeros(J, dtype=torch.float32, device=dev)
            self.a = torch.zeros(R * int(sum(dims)), dtype=torch.float64, device=dev)
            dtype = "bf16x2" if self.two_plane else "f32"
            self.state = cp.State(cp.make_shape(dims, R, dtype), self.a, mu0=-1.0, tau=o.tau, tol=o.tol,
                                  mu_max=o.mu_max, max_iter=o.max_iter, normalize=bool(o.normalize),
                                  core_mode=cp.CP_CORE_MIXED, refine_iters=server.large_refine)
            self.state.capture(self.y, server.large_steps, stream=self.stream)
        self.host = torch.empty(128, dtype=torch.uint8).pin_memory()
        self.event = None
        self.req = None
        self.admitted = 0.0

    def arm(self, server, req: Request, now: float):
        import torch
        with torch.cuda.stream(self.stream):
            y, a = _inputs(req, server.device)
            if self.two_plane:
                _cp().tensor_split(y.contiguous(), out=self.y, stream=self.stream)
            else:
                self.y.copy_(y)
            self.a.copy_(a)
            self.state.init(self.y, stream=self.stream)
        self.req = req
        self.admitted = now
        self.launch()

    def launch(self):
        import torch
        with torch.cuda.stream(self.stream):
            self.state.launch(stream=self.stream)
            self.host.copy_(self.state.status_tensor(), non_blocking=True)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)

    def finished(self) -> Optional[dict]:
        cp = _cp()
        d = cp.Status.from_buffer_copy(bytes(self.host.numpy())).as_dict()
        if d["stop"] == 0:
            return None
        d["stop_reason"] = cp.STOP.get(d["stop"], d["stop"])
        d["dims"], d["R"] = self.dims, self.R
        return d

    def close(self):
        self.state.close()


class Server:
    """Continuous-batching server for one GPU.

    hbm_budget: bytes that admitted requests may hold in total; arena_bytes
    of it back the lanes (default half), the rest the large requests.
    lanes: (max_cost, slots, trials per round) per lane, cost = R prod(I_n);
    a request joins the first lane whose class holds it and whose shape the
    batched kernel takes, else it is a large request; at most large_slots
    large requests run at once (they share the GPU), or, with large_slots = 0,
    as many as the large-request budget holds (at most MAX_LARGE).  All
    requests share the
    stop rule (tol, mu_max, max_iter) and the kernel tile size, so a lane
    request's arithmetic is the same whatever else is in flight.
    """

    def __init__(self, hbm_budget: float, arena_bytes: Optional[int] = None,
                 lanes=((64 ** 3 * 12, 1024, 8),), tile: int = 16,
                 tol: float = 1e-8, max_iter: int = 1000, mu_max: float = 1e30, normalize: bool = True,
                 refine_iters: int = 4, large_steps: int = 4, large_refine: int = 8,
                 large_slots: int = 4, device="cuda"):
        import torch
        cp = _cp()
        self.device = torch.device(device)
        self.budget = int(hbm_budget)
        arena_bytes = int(arena_bytes if arena_bytes is not None else self.budget // 2)
        if arena_bytes > self.budget:
            raise ValueError("arena larger than the HBM budget")
        head = _ALIGN * len(lanes)                 # one queue counter per lane
        self.buf = torch.empty(head + arena_bytes, dtype=torch.uint8, device=self.device)
        self.arena = Arena(arena_bytes, base=head)
        self.large_budget = self.budget - arena_bytes
        self.large_used = 0
        self.peak_bytes = 0
        self.opts = cp.Opts(mu0=-1.0, tau=1e-3, tol=tol, mu_max=mu_max, max_iter=max_iter,
                            normalize=1 if normalize else 0, core_mode=cp.CP_CORE_MIXED,
                            refine_iters=refine_iters)
        self.lanes = [_Lane(self, k, mc, sl, tr, tile) for k, (mc, sl, tr) in enumerate(lanes)]
        self.busy: List[_StateSlot] = []
        self.idle: List[_StateSlot] = []
        self.large_steps = large_steps
        self.large_refine = large_refine
        self.large_slots = large_slots
        self.peak_busy = 0
        self.large_rounds = 0

    def route(self, req: Request):
        """The lane that takes `req`, or None for the large-request path."""
        if lane_bytes(req.dims, req.R) is not None:
            for ln in self.lanes:
                if req.cost <= ln.max_cost:
                    return ln
        return None

    def serve(self, requests: List[Request], time_limit: Optional[float] = None,
              realtime: bool = True) -> List[Result]:
        """Run until every request has stopped (or time_limit seconds).
        realtime: requests arrive at their `arrival` times; otherwise all are
        queued at the start."""
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            ln = self.route(r)
            if ln is None and state_bytes(r.dims, r.R) > self.large_budget:
                raise ValueError(f"request {r.rid} never fits the large-request budget")
            if ln is not None and lane_bytes(r.dims, r.R) > self.arena.size:
                raise ValueError(f"request {r.rid} never fits the arena")
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        waiting: Dict[int, List[Request]] = {}
        results: List[Result] = []
        qi = 0
        while qi < len(pending) or any(waiting.values()) or any(l.active for l in self.lanes) or self.busy:
            t = now()
            if time_limit is not None and t > time_limit:
                break
            while qi < len(pending) and (not realtime or pending[qi].arrival <= t):
                r = pending[qi]
                ln = self.route(r)
                waiting.setdefault(-1 if ln is None else self.lanes.index(ln), []).append(r)
                qi += 1
            progressed = False
            # large requests: re-arm an idle slot of the same shape, or make a
            # slot within the budget (dropping idle slots of other shapes)
            q = waiting.get(-1, [])
            cap = self.large_slots if self.large_slots > 0 else MAX_LARGE
            while q and len(self.busy) < cap:
                slot = self._state_slot(q[0])
                if slot is None:
                    break
                slot.arm(self, q.pop(0), now())
                self.busy.append(slot)
                self.large_rounds += 1
                progressed = True
            for L in list(self.busy):
                if not L.event.query():
                    continue
                d = L.finished()
                if d is None:
                    L.launch()
                    self.large_rounds += 1
                else:
                    a = L.a.cpu()
                    results.append(Result(L.req.rid, L.req.arrival, L.admitted, now(), d,
                                          cp_split(a, L.dims, L.R), "state"))
                    self.busy.remove(L)
                    self.idle.append(L)
                progressed = True
            # lanes: between rounds retire, admit, launch
            for k, ln in enumerate(self.lanes):
                if ln.event is not None:
                    if not ln.event.query():
                        continue
                    results.extend(ln.harvest(now))
                    ln.event = None
                q = waiting.get(k, [])
                while q and ln.try_admit(q[0], now()):
                    q.pop(0)
                if ln.active:
                    ln.launch()
                    progressed = True
            self.peak_bytes = max(self.peak_bytes, self.arena.used + self.large_used)
            self.peak_busy = max(self.peak_busy, len(self.busy))
            if not progressed:
                time.sleep(5e-5)
        torch.cuda.synchronize(self.device)
        return results

    def _state_slot(self, req: Request) -> Optional[_StateSlot]:
        key = (tuple(req.dims), int(req.R))
        for k, sl in enumerate(self.idle):
            if (sl.dims, sl.R) == key:
                return self.idle.pop(k)
        need = state_bytes(req.dims, req.R)
        while self.large_used + need > self.large_budget and self.idle:
            old = self.idle.pop(0)
            old.close()
            self.large_used -= old.bytes
        if self.large_used + need > self.large_budget:
            return None
        self.large_used += need
        return _StateSlot(self, req.dims, req.R)

    def close(self):
        for L in self.busy + self.idle:
            L.close()
        self.busy.clear()
        self.idle.clear()
        self.large_used = 0


def cp_split(a, dims, R):
    return _cp().split_factors(a, dims, R)
