"""Batched form (many small decompositions in one persistent launch) against
the CPU oracle.

The batched kernel reads float32 tensors and uses float32 products for the
O(T R^2) and O(J R) work (float64 for the R x R factorisations, the core
refinement and the control), so it is held to the reduced-precision bar:
  * one trial: the step agrees with the oracle's fLM_a step on the same
    rounded tensor to 1e-4 relative (well-conditioned starting points);
  * runs to convergence: the final relative error agrees with the oracle's
    to 1e-6 relative;
  * a problem gives bit-identical results alone and inside a batch, and
    across launches (every reduction of the batched kernel has a fixed order).
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


MIX = [((10, 12, 14), 3), ((33, 20, 17), 5), ((64, 64, 64), 12), ((16, 40, 25), 8), ((12, 10, 11, 9), 3),
       ((50, 37), 6), ((25, 25, 25), 10), ((61, 13, 47), 7)]


def _problems(seed0, shapes, snr=30.0, mu0=1.0):
    out = []
    for k, (dims, R) in enumerate(shapes):
        p = synth.make_problem(seed0 + k, dims, R, dtype="f32", snr_db=snr, collinearity=(0.8,))
        out.append(p)
    return out


@pytest.mark.parametrize("mu", [1.0, 0.3])
def test_batch_one_trial_matches_oracle_step(cp, mu):
    probs = _problems(300, MIX)
    b = cp.Batch([(p.Y, p.init, mu) for p in probs], max_iter=1, normalize=False)
    b.run(trials=1)
    torch.cuda.synchronize()
    st = b.statuses()
    for k, p in enumerate(probs):
        ref = O.flm_step(p.Y, p.init, mu)
        assert st[k]["iters"] == 1
        r2_ref = O.residual2(p.Y, ref.A_new)
        assert st[k]["resid2_trial"] == pytest.approx(r2_ref, rel=1e-4), k
        if st[k]["last_accepted"]:
            got = b.factors(k)
            assert rel([g.numpy() for g in got], ref.A_new) < 1e-4, k


def test_batch_runs_to_oracle_fit(cp):
    shapes = [((10, 12, 14), 3), ((20, 18, 16), 4), ((14, 15, 16, 7), 2), ((30, 9), 3)]
    probs = _problems(400, shapes)
    b = cp.Batch([(p.Y, p.init, 1.0) for p in probs], tol=1e-10, max_iter=400)
    b.run()
    torch.cuda.synchronize()
    st = b.statuses()
    for k, p in enumerate(probs):
        ref = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=400, tol=1e-10)
        assert st[k]["stop"] != 0, st[k]
        assert st[k]["rel_err"] == pytest.approx(ref.rel_err, rel=1e-6), (k, st[k]["rel_err"], ref.rel_err)


def test_batch_alone_equals_in_mix(cp):
    probs = _problems(500, MIX)
    pick = 3
    alone = cp.Batch([(probs[pick].Y, probs[pick].init, 1.0)], max_iter=25)
    alone.run()
    mixed = cp.Batch([(p.Y, p.init, 1.0) for p in probs], max_iter=25)
    mixed.run(ctas=3)
    torch.cuda.synchronize()
    sa, sm = alone.statuses()[0], mixed.statuses()[pick]
    assert sa["iters"] == sm["iters"] == 25
    assert sa["rel_err"] == pytest.approx(sm["rel_err"], rel=0)
    fa = [f.numpy() for f in alone.factors(0)]
    fm = [f.numpy() for f in mixed.factors(pick)]
    assert rel(fa, fm) == 0.0


def test_batch_continues_across_launches(cp):
    probs = _problems(600, MIX[:4])
    one = cp.Batch([(p.Y, p.init, 1.0) for p in probs], max_iter=12)
    one.run()
    two = cp.Batch([(p.Y, p.init, 1.0) for p in probs], max_iter=12)
    for _ in range(4):
        two.run(trials=3)
    torch.cuda.synchronize()
    for s1, s2 in zip(one.statuses(), two.statuses()):
        assert s1["iters"] == s2["iters"] == 12
        assert s1["rel_err"] == pytest.approx(s2["rel_err"], rel=0)


def test_config4_full_batch_sampled(cp):
    """512 problems, I_n ~ U{10..64}, R ~ U{3..12}, mode-1 collinearity 0.8,
    SNR 30 dB, float32 tensors: one persistent launch, 30 trials each; a
    sample of problems is checked against the oracle run for 30 trials."""
    specs = synth.config4_specs(0, 512)
    probs = [synth.config4_problem(s, dtype="f32") for s in specs]
    b = cp.Batch([(p.Y, p.init, None) for p in probs], max_iter=30)
    b.run()
    torch.cuda.synchronize()
    st = b.statuses()
    assert all(s["iters"] == 30 or s["stop"] in (1, 2) for s in st)
    rng = np.random.default_rng(0)
    for k in rng.choice(512, size=4, replace=False):
        p = probs[k]
        ref = O.lm_fit(p.Y, p.init, mu0=None, max_iter=30)
        assert st[k]["rel_err"] == pytest.approx(ref.rel_err, rel=1e-3), (k, specs[k])


def test_autotuner_choice_runs_and_matches(cp):
    """The tuned launch (tile size, queue order) reaches the same fit as the
    default launch; the tuner leaves the batch at its starting point."""
    from paper_1205_2584_gb300 import autotune
    probs = _problems(700, MIX)
    b = cp.Batch([(p.Y, p.init, 1.0) for p in probs], max_iter=40)
    cfg = autotune.tune_batch(b, trials=2, cache=False)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert cfg["tile"] in (8, 16, 32) and cfg["order"] in ("given", "cost") and cfg["ctas"] in (sms, 2 * sms)
    assert len(cfg["timings"]) == 12
    st0 = b.statuses()
    assert all(s["iters"] == 0 for s in st0)
    b.run(tile=cfg["tile"], order=None if cfg["order"] == "given" else "cost", ctas=cfg["ctas"])
    ref = cp.Batch([(p.Y, p.init, 1.0) for p in probs], max_iter=40)
    ref.run()
    torch.cuda.synchronize()
    # the tile size regroups float32 partial sums, so trajectories agree to
    # rounding; a problem that reaches its noise floor may stop a few trials
    # apart (mu passes mu_max), at the same fit
    for s1, s2 in zip(b.statuses(), ref.statuses()):
        assert s1["rel_err"] == pytest.approx(s2["rel_err"], rel=1e-6)
