"""Serving loop on the GPU: requests in a mix give the same result as alone,
fits agree with the oracle, admission keeps to the HBM budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cp_oracle as O  # noqa: E402
from paper_1205_2584_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def sv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1205_2584_gb300 import serve
    return serve


def _req(serve, rid, seed, dims, R, arrival=0.0, dtype="f32"):
    p = synth.make_problem(seed, dims, R, dtype=dtype, snr_db=30.0, collinearity=(0.8,))
    return serve.Request(rid=rid, arrival=arrival, dims=tuple(dims), R=R, Y=p.Y, init=p.init), p


SMALL = [((20, 22, 18), 4), ((32, 32, 32), 5), ((16, 30, 12), 3), ((40, 12, 25), 6)]
MEDIUM = [((64, 64, 64), 12), ((96, 50, 40), 16)]
LARGE = [((300, 24, 20), 4)]          # I_1 > 256: outside the batched kernel
# I_1 > 256 and a multiple of 8: a State on the two-plane bfloat16 tensor; its
# values are drawn two-plane representable, so the oracle sees the same tensor
LARGE2 = [((264, 24, 20), 4)]


def _mix(serve):
    reqs, probs = [], []
    for k, (dims, R) in enumerate(SMALL + MEDIUM + LARGE + LARGE2):
        r, p = _req(serve, k, 900 + k, dims, R, dtype="bf16x2" if (dims, R) in LARGE2 else "f32")
        reqs.append(r)
        probs.append(p)
    return reqs, probs


def _server(serve, **kw):
    kw.setdefault("hbm_budget", 1 << 30)
    kw.setdefault("lanes", ((32768 * 8, 64, 8), (float("inf"), 32, 3)))
    kw.setdefault("tol", 1e-8)
    kw.setdefault("max_iter", 300)
    return serve.Server(**kw)


def test_lane_request_same_alone_and_in_mix(sv):
    reqs, _ = _mix(sv)
    srv = _server(sv)
    mixed = {r.rid: r for r in srv.serve(reqs, realtime=False)}
    srv.close()
    assert sorted(mixed) == list(range(len(reqs)))
    for pick in (1, 4):                       # one per lane
        alone_srv = _server(sv)
        alone = alone_srv.serve([reqs[pick]], realtime=False)[0]
        alone_srv.close()
        m = mixed[pick]
        assert m.path == alone.path == "lane"
        assert m.status["iters"] == alone.status["iters"]
        assert m.status["rel_err"] == alone.status["rel_err"]           # bit-identical
        for fa, fm in zip(alone.factors, m.factors):
            assert torch.equal(fa, fm)


def test_large_request_alone_and_in_mix_agree(sv):
    reqs, _ = _mix(sv)
    srv = _server(sv)
    mixed = {r.rid: r for r in srv.serve(reqs, realtime=False)}
    srv.close()
    for k in (len(SMALL + MEDIUM), len(reqs) - 1):     # float32 and two-plane State requests
        srv = _server(sv)
        alone = srv.serve([reqs[k]], realtime=False)[0]
        srv.close()
        assert mixed[k].path == alone.path == "state"
        assert mixed[k].status["rel_err"] == pytest.approx(alone.status["rel_err"], rel=1e-6)


def test_served_fits_match_oracle(sv):
    reqs, probs = _mix(sv)
    srv = _server(sv)
    got = {r.rid: r for r in srv.serve(reqs, realtime=False)}
    srv.close()
    for k in (0, 2, 4, len(reqs) - 2, len(reqs) - 1):
        ref = O.lm_fit(probs[k].Y, probs[k].init, mu0=None, max_iter=300, tol=1e-8)
        assert got[k].status["stop"] != 0
        assert got[k].status["rel_err"] == pytest.approx(ref.rel_err, rel=1e-6), (k, got[k].status, ref.rel_err)


def test_admission_respects_hbm_budget_and_refills(sv):
    """An arena that holds two small requests at a time and a large budget
    for one large request: requests wait, are admitted as others retire, and
    every one still finishes with the same result as alone."""
    serve = sv
    small = [_req(serve, k, 1000 + k, (32, 32, 32), 5)[0] for k in range(6)]
    big = [_req(serve, 10 + k, 1100 + k, (300, 24, 20), 4)[0] for k in range(2)]
    per = serve.lane_bytes((32, 32, 32), 5)
    per_big = serve.state_bytes((300, 24, 20), 4)
    srv = _server(serve, arena_bytes=2 * per + 255, hbm_budget=2 * per + 255 + per_big + 1024)
    res = {r.rid: r for r in srv.serve(small + big, realtime=False)}
    assert srv.peak_bytes <= srv.budget
    assert sorted(res) == [0, 1, 2, 3, 4, 5, 10, 11]
    # at most two small requests in flight at any time
    spans = sorted((res[k].admitted, res[k].done) for k in range(6))
    for t, _ in spans:
        assert sum(1 for a, d in spans if a <= t < d) <= 2
    # the second large request waits for the first
    assert res[11].admitted >= res[10].done or res[10].admitted >= res[11].done
    srv.close()
    srv = _server(serve)
    alone = srv.serve([small[5]], realtime=False)[0]
    srv.close()
    assert alone.status["rel_err"] == res[5].status["rel_err"]


def test_realtime_arrivals_overlap(sv):
    """Requests arriving while others run are admitted into running lanes."""
    serve = sv
    reqs = [_req(serve, k, 1200 + k, (32, 32, 32), 5, arrival=0.004 * k)[0] for k in range(12)]
    srv = _server(serve)
    res = srv.serve(reqs, realtime=True)
    srv.close()
    assert len(res) == 12
    s = serve.summarize(res, max(r.done for r in res))
    assert s["p99_s"] >= s["p50_s"] > 0
    ad = sorted(r.admitted for r in res)
    assert ad[-1] - ad[0] > 0.02        # admitted over time, not all at once


def test_budget_bound_large_slots(sv):
    """large_slots = 0: as many large requests run at once as the large-request
    budget holds (here three States of one shape); the others wait and every
    request still finishes with the result it has alone."""
    serve = sv
    big = [_req(serve, k, 1200 + k, (300, 24, 20), 4)[0] for k in range(6)]
    per_big = serve.state_bytes((300, 24, 20), 4)
    arena = 1 << 20
    srv = _server(serve, arena_bytes=arena, hbm_budget=arena + 3 * per_big + 1024, large_slots=0)
    res = {r.rid: r for r in srv.serve(big, realtime=False)}
    assert sorted(res) == list(range(6))
    assert srv.peak_busy == 3
    assert srv.peak_bytes <= srv.budget
    srv.close()
    srv = _server(serve)
    alone = srv.serve([big[4]], realtime=False)[0]
    srv.close()
    assert alone.status["rel_err"] == pytest.approx(res[4].status["rel_err"], rel=1e-6)
