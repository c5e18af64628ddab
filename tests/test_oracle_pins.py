"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: brute-force
loops over tensor entries, central finite differences (exact for the
multilinear / per-coordinate-quadratic functions involved), the textbook
full-Hessian step, the closed-form K^{-1} of Appendix E, structural counts
printed in Sec. 4.4, the generator angles and magnitudes printed in Sec. 6,
Appendix F's closed forms, Nielsen's rule at special values and limits.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import cp_oracle as O
from paper_1205_2584_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a = np.concatenate([np.ravel(x) for x in a]) if isinstance(a, (list, tuple)) else np.ravel(a)
    b = np.concatenate([np.ravel(x) for x in b]) if isinstance(b, (list, tuple)) else np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _small(seed=0, dims=(3, 4, 5), R=2, snr=30.0):
    return synth.make_problem(seed, dims, R, snr_db=snr)


# --------------------------------------------------------------------- algebra


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 2, 3)])
def test_unfold_matches_kolda_index_formula(dims):
    rng = np.random.default_rng(1)
    Y = rng.standard_normal(dims)
    N = len(dims)
    for n in range(N):
        Yn = O.unfold(Y, n)
        for idx in itertools.product(*[range(d) for d in dims]):
            col, stride = 0, 1
            for k in range(N):
                if k == n:
                    continue
                col += idx[k] * stride
                stride *= dims[k]
            assert Yn[idx[n], col] == Y[idx]


def test_khatri_rao_columnwise_kronecker():
    rng = np.random.default_rng(2)
    A, B, C = rng.standard_normal((3, 2)), rng.standard_normal((4, 2)), rng.standard_normal((2, 2))
    kr = O.khatri_rao([A, B, C])
    for r in range(2):
        np.testing.assert_array_equal(kr[:, r], np.kron(np.kron(A[:, r], B[:, r]), C[:, r]))


def test_cp_full_bruteforce():
    rng = np.random.default_rng(3)
    A = [rng.standard_normal((I, 3)) for I in (3, 4, 2, 3)]
    Y = O.cp_full(A)
    for idx in itertools.product(*[range(a.shape[0]) for a in A]):
        v = sum(math.prod(A[n][idx[n], r] for n in range(4)) for r in range(3))
        assert abs(Y[idx] - v) < 1e-13


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 3), (4, 5)])
def test_mttkrp_bruteforce(dims):
    rng = np.random.default_rng(4)
    R = 3
    Y = rng.standard_normal(dims)
    A = [rng.standard_normal((I, R)) for I in dims]
    N = len(dims)
    for n in range(N):
        M = O.mttkrp(Y, A, n)
        ref = np.zeros((dims[n], R))
        for idx in itertools.product(*[range(d) for d in dims]):
            for r in range(R):
                ref[idx[n], r] += Y[idx] * math.prod(A[k][idx[k], r] for k in range(N) if k != n)
        np.testing.assert_allclose(M, ref, rtol=1e-12, atol=1e-12)


def test_residual_bruteforce():
    p = _small()
    Yh = O.cp_full(p.init)
    ref = sum((p.Y[idx] - Yh[idx]) ** 2 for idx in itertools.product(*[range(d) for d in p.dims]))
    assert abs(O.residual2(p.Y, p.init) - ref) < 1e-10 * ref


def test_grams_definition():
    rng = np.random.default_rng(5)
    A = [rng.standard_normal((I, 3)) for I in (4, 5, 6, 3)]
    g = O.grams(A)
    for n in range(4):
        for m in range(4):
            ref = np.ones((3, 3))
            for k in range(4):
                if k not in (n, m):
                    for r in range(3):
                        for s in range(3):
                            ref[r, s] *= sum(A[k][i, r] * A[k][i, s] for i in range(A[k].shape[0]))
            np.testing.assert_allclose(g.Gamma_nm[n, m], ref, rtol=1e-13)


# ------------------------------------------------------- Jacobian and gradient


def test_jacobian_central_differences():
    """Y_hat is linear in every single parameter, so a central difference is
    exact up to rounding: pins Lemma 2's J (commutation Q_n, KR order)."""
    rng = np.random.default_rng(6)
    A = [rng.standard_normal((I, 2)) for I in (3, 2, 4)]
    J = O.jacobian(A)
    x0 = O.join_params(A)
    dims = [a.shape[0] for a in A]
    h = 0.5
    for p in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        xp[p] += h
        xm[p] -= h
        col = (O.vec(O.cp_full(O.split_params(xp, dims, 2))) -
               O.vec(O.cp_full(O.split_params(xm, dims, 2)))) / (2 * h)
        np.testing.assert_allclose(J[:, p], col, atol=1e-12)


@pytest.mark.parametrize("dims", [(3, 4, 5), (3, 2, 3, 2)])
def test_gradient_central_differences(dims):
    """g = -(d/da) 0.5 ||Y - Y_hat||^2, a quadratic in each single coordinate,
    so the central difference is exact up to rounding (Eq. mappingJ)."""
    p = synth.make_problem(7, dims, 3, snr_db=20)
    A = p.init
    x0 = O.join_params(A)
    g = O.join_params(O.gradient_blocks(p.Y, A))
    h = 1e-3
    fd = np.empty_like(x0)
    for q in range(x0.size):
        xp, xm = x0.copy(), x0.copy()
        xp[q] += h
        xm[q] -= h
        fp = 0.5 * O.residual2(p.Y, O.split_params(xp, dims, 3))
        fm = 0.5 * O.residual2(p.Y, O.split_params(xm, dims, 3))
        fd[q] = -(fp - fm) / (2 * h)
    assert _rel(g, fd) < 1e-8


def test_gradient_equals_JT_e():
    p = _small(dims=(3, 4, 5, 2), R=3)
    A = p.init
    J = O.jacobian(A)
    e = O.vec(p.Y - O.cp_full(A))
    assert _rel(O.join_params(O.gradient_blocks(p.Y, A)), J.T @ e) < 1e-13


# ------------------------------------------------------------ Hessian structure


@pytest.mark.parametrize("dims,R", [((3, 4, 5), 2), ((2, 3, 2, 3), 3), ((4, 3), 2)])
def test_hessian_low_rank_adjustment(dims, R):
    """Theorem 2: J^T J = G + Z K Z^T."""
    rng = np.random.default_rng(8)
    A = [rng.standard_normal((I, R)) for I in dims]
    J = O.jacobian(A)
    g = O.grams(A)
    H = O.block_G(g, dims) + O.block_Z(A) @ O.kernel_K(g) @ O.block_Z(A).T
    assert _rel(H, J.T @ J) < 1e-14


def test_hessian_block_structure_counts():
    """Sec. 4.1 (Fig. 1): H consists of N(N-1)R^2 rank-one blocks off the
    block diagonal and N R^2 diagonal blocks on it."""
    dims, R = (3, 4, 5, 6, 7), 3
    rng = np.random.default_rng(9)
    A = [rng.standard_normal((I, R)) for I in dims]
    J = O.jacobian(A)
    H = J.T @ J
    offs = np.concatenate([[0], np.cumsum([I * R for I in dims])])
    rank_one = diag = 0
    for n, m in itertools.product(range(5), range(5)):
        for r, s in itertools.product(range(R), range(R)):
            r0 = offs[n] + r * dims[n]
            c0 = offs[m] + s * dims[m]
            blk = H[r0:r0 + dims[n], c0:c0 + dims[m]]
            if n == m:
                if np.allclose(blk, np.diag(np.diag(blk)), atol=1e-12):
                    diag += 1
            elif np.linalg.matrix_rank(blk, tol=1e-9 * np.abs(blk).max()) == 1:
                rank_one += 1
    assert rank_one == 5 * 4 * R * R
    assert diag == 5 * R * R


def test_kernel_inverse_closed_form():
    """Appendix E: K K~ = I with K~^(n,m) = (1/(N-1) - delta) diag(vec(C^n * C^m / Gamma)) P_R."""
    for dims in [(3, 4, 5), (3, 4, 5, 6), (4, 5)]:
        rng = np.random.default_rng(10)
        A = [rng.standard_normal((I, 3)) for I in dims]
        g = O.grams(A)
        K = O.kernel_K(g)
        assert np.abs(K @ O.kernel_K_inverse_closed_form(g) - np.eye(K.shape[0])).max() < 1e-12


def test_core_densities_paper_example():
    """Sec. 4.4 densities of Phi_1 and Phi_2 on the paper's 3x4x5x6x7, R = 3 example."""
    line = [l for l in open(os.path.join(GOLD, "core_density.txt")) if not l.startswith("#")][0].split()
    dims = tuple(int(v) for v in line[0].split("x"))
    R = int(line[1])
    d1 = int(line[2]) / int(line[3])
    d2 = int(line[4]) / int(line[5])
    rng = np.random.default_rng(11)
    A = [rng.standard_normal((I, R)) for I in dims]
    g = O.grams(A)
    K = O.kernel_K(g)
    Psi = O.psi_mu(g, O.damped_inverses(g, 0.5))
    Phi1 = np.eye(K.shape[0]) + Psi @ K
    Phi2 = O.kernel_K_inverse_closed_form(g) + Psi
    n2 = K.shape[0] ** 2
    assert np.count_nonzero(Phi1) / n2 == pytest.approx(d1, abs=1e-12)
    assert np.count_nonzero(Phi2) / n2 == pytest.approx(d2, abs=1e-12)


# ---------------------------------------------- fast step == textbook step


@pytest.mark.parametrize("dims,R,mu", [((4, 5, 6), 3, 1.0), ((4, 5, 6), 3, 0.1),
                                        ((3, 4, 3, 4), 2, 1.0), ((5, 6), 3, 0.3),
                                        ((6, 5, 4), 4, 10.0)])
def test_fast_step_equals_textbook(dims, R, mu):
    """Theorems 1/3 are identities: the fLM_a step equals (J^T J + mu I)^{-1} g
    to 1e-10 relative on well-conditioned inputs."""
    p = synth.make_problem(12, dims, R, snr_db=30)
    t = O.textbook_step(p.Y, p.init, mu)
    f = O.flm_step(p.Y, p.init, mu)
    assert _rel(f.delta, t) < 1e-10


def test_fast_step_variant_b_and_spd_core():
    p = synth.make_problem(13, (4, 5, 6), 3, snr_db=30)
    mu = 0.7
    t = O.textbook_step(p.Y, p.init, mu)
    fb = O.flm_step(p.Y, p.init, mu, variant="b")
    assert _rel(fb.delta, t) < 1e-10
    fa = O.flm_step(p.Y, p.init, mu)
    assert _rel(O.f_from_spd_core(p.init, mu, fa.w), fa.f) < 1e-11
    Mc = O.spd_core(p.init, mu)
    assert np.allclose(Mc, Mc.T, atol=1e-12)
    assert np.linalg.eigvalsh(Mc).min() > 0


def test_w_is_L_transpose_g_and_printed_form_differs():
    """w = L_mu^T g with L_mu = blkdiag(Gt^(n) kron A^(n)) (Theorem 3, Eq. iGZ_LM);
    the corrected w_mu matches it and the printed Gamma Gt form does not."""
    p = synth.make_problem(14, (4, 5, 6), 3, snr_db=30)
    A, mu = p.init, 0.5
    g = O.grams(A)
    Gt = O.damped_inverses(g, mu)
    L = __import__("scipy.linalg", fromlist=["block_diag"]).block_diag(
        *[np.kron(Gt[n], A[n]) for n in range(3)])
    J = O.jacobian(A)
    gvec = J.T @ O.vec(p.Y - O.cp_full(A))
    w_ref = L.T @ gvec
    M = O.mttkrp_all(p.Y, A)
    assert _rel(O.w_mu(A, M, g, Gt), w_ref) < 1e-12
    printed = np.concatenate([O.vec(A[n].T @ M[n] @ Gt[n] - g.Gamma_all @ Gt[n]) for n in range(3)])
    assert _rel(printed, w_ref) > 1e-2


def test_orthogonal_factors_singular_K():
    """Sec. 4.4: mutually orthogonal columns make K singular; fLM_a and the SPD
    core still give the textbook step."""
    rng = np.random.default_rng(15)
    dims, R = (5, 6, 7), 3
    A = [np.linalg.qr(rng.standard_normal((I, R)))[0] * 1.5 for I in dims]
    Y = synth.add_noise(rng, synth.tensor_from_factors(
        [rng.standard_normal((I, R)) for I in dims]), 30.0)
    g = O.grams(A)
    K = O.kernel_K(g)
    assert np.linalg.matrix_rank(K) < K.shape[0]
    mu = 0.4
    t = O.textbook_step(Y, A, mu)
    f = O.flm_step(Y, A, mu)
    assert _rel(f.delta, t) < 1e-10
    assert _rel(O.f_from_spd_core(A, mu, f.w), f.f) < 1e-10


def test_large_mu_limit_is_scaled_gradient():
    """Sec. 3: as mu grows the step tends to g / mu (gradient descent)."""
    p = _small(dims=(4, 5, 6), R=3)
    mu = 1e9
    f = O.flm_step(p.Y, p.init, mu)
    G = O.gradient_blocks(p.Y, p.init)
    assert _rel([d * mu for d in f.delta], G) < 1e-5


# ---------------------------------------------------------------- LM control


def test_nielsen_rule_special_values():
    mu = 8.0
    assert O.nielsen_update(mu, 2.0, 1.0) == (pytest.approx(mu / 3), 2.0)    # 1 - 1 = 0 -> floor 1/3
    assert O.nielsen_update(mu, 2.0, 0.5) == (pytest.approx(mu), 2.0)        # 1 - 0 = 1
    assert O.nielsen_update(mu, 2.0, 0.75)[0] == pytest.approx(mu * (1 - 0.125))
    assert O.nielsen_update(mu, 2.0, 1e-9)[0] == pytest.approx(mu * 2.0, rel=1e-6)  # -> 1 + 1
    assert O.nielsen_update(mu, 4.0, -0.3) == (mu * 4.0, 8.0)


def test_gain_ratio_denominator_positive():
    """Delta^T (g + mu Delta) = Delta^T H Delta + 2 mu ||Delta||^2 > 0."""
    for seed in range(5):
        p = synth.make_problem(16 + seed, (4, 5, 6), 3, snr_db=10)
        for mu in (1e-3, 1.0, 100.0):
            st = O.flm_step(p.Y, p.init, mu)
            den = sum(float(np.sum(d * (gn + mu * d))) for d, gn in zip(st.delta, st.G))
            J = O.jacobian(p.init)
            dvec = O.join_params(st.delta)
            ref = float(np.sum((J @ dvec) ** 2)) + 2 * mu * float(np.sum(dvec ** 2))
            assert den > 0
            assert den == pytest.approx(ref, rel=1e-9)


def test_normalize_keeps_model_and_equalises_norms():
    rng = np.random.default_rng(20)
    A = [rng.standard_normal((I, 4)) * s for I, s in zip((5, 6, 7), (0.1, 3.0, 10.0))]
    B = O.normalize_equal_energy(A)
    assert _rel(O.cp_full(B), O.cp_full(A)) < 1e-14
    norms = np.stack([np.linalg.norm(b, axis=0) for b in B])
    assert np.allclose(norms, norms[0][None, :], rtol=1e-13)
    for n in range(3):
        assert np.all(np.sign(B[n]) == np.sign(A[n]))


@pytest.mark.parametrize("dims,R", [((8, 9, 10), 3), ((6, 7, 5, 6), 2)])
def test_noiseless_exact_rank_converges(dims, R):
    """An exact-rank noiseless tensor is fitted to epsilon < 1e-10."""
    p = synth.make_problem(21, dims, R, snr_db=None)
    rng = np.random.default_rng(22)
    A0 = [a + 0.3 * rng.standard_normal(a.shape) for a in p.true_factors]
    res = O.lm_fit(p.Y, A0, mu0=1.0, max_iter=300, tol=0.0)
    assert res.rel_err < 1e-10


def test_lm_fast_and_textbook_trajectories_agree():
    """The first LM iterations with the fast and the textbook step coincide."""
    p = synth.make_problem(23, (6, 7, 8), 3, snr_db=30)
    a = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=8)
    b = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=8, step="textbook")
    assert np.allclose(a.history, b.history, rtol=1e-9, atol=0)


def test_accepted_errors_monotone():
    p = synth.make_problem(24, (10, 11, 12), 4, snr_db=30, collinearity=(0.9, 0.9, 0.9))
    res = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=60)
    h = np.array(res.history)
    assert np.all(np.diff(h) <= 1e-15)



def test_initial_mu_is_tau_times_max_diag_of_JtJ():
    """Eq. mu0: mu_0 = tau max diag(H), H = J^T J formed from the explicit
    Jacobian (Lemma 2).  The column norms differ per mode and component so
    that max diag Gamma^(n), max diag C^(n) and max diag of the all-mode
    Hadamard product Gamma are three different numbers; only the first is
    right."""
    rng = np.random.default_rng(40)
    dims, R = (3, 4, 5), 3
    scales = [np.array([1.0, 3.0, 0.5]), np.array([2.0, 0.2, 1.5]), np.array([0.7, 4.0, 1.1])]
    A = [rng.standard_normal((I, R)) * s[None, :] for I, s in zip(dims, scales)]
    J = O.jacobian(A)
    hmax = float(np.max(np.diag(J.T @ J)))
    for tau in (1e-3, 0.5):
        assert O.initial_mu(A, tau) == pytest.approx(tau * hmax, rel=1e-13)
    g = O.grams(A)
    wrong = {float(np.max([np.max(np.diag(c)) for c in g.C])), float(np.max(np.diag(g.Gamma_all)))}
    for w in wrong:
        assert abs(w - hmax) > 1e-3 * hmax


def test_initial_mu_hand_computed_example():
    """Two 2 x 2 factors with orthogonal columns: diag Gamma^(1) = diag C^(2),
    diag Gamma^(2) = diag C^(1); with column norms^2 (1, 4) and (9, 0.25) the
    largest diagonal entry of H is 9 (printed rule: tau times it)."""
    A = [np.array([[1.0, 0.0], [0.0, 2.0]]), np.array([[3.0, 0.0], [0.0, 0.5]])]
    assert O.initial_mu(A, 1.0) == pytest.approx(9.0, rel=1e-15)
    assert O.initial_mu(A, 1e-3) == pytest.approx(9e-3, rel=1e-15)


def test_initial_mu_unit_columns_special_case():
    """Eq. mu0's last form: with unit-length columns in modes n < N,
    max diag H = max{1, diag C^(N)}."""
    rng = np.random.default_rng(41)
    dims, R = (4, 5, 6), 3
    A = [rng.standard_normal((I, R)) for I in dims]
    for n in range(2):
        A[n] /= np.linalg.norm(A[n], axis=0)
    for s in (0.3, 2.5):                      # last-mode norms below / above 1
        B = [A[0], A[1], A[2] / np.linalg.norm(A[2], axis=0) * s]
        expect = max(1.0, float(np.max(np.diag(B[2].T @ B[2]))))
        assert O.initial_mu(B, 1.0) == pytest.approx(expect, rel=1e-13)


def test_lm_fit_relative_change_stop_on_constructed_history():
    """Sec. 4.6 stop rule as read here: stop on the first ACCEPTED trial whose
    relative change of epsilon is below tol.  A reference run (tol = 0) gives
    the history; tol is then placed between that trial's change and every
    earlier accepted change, and the run must stop exactly there, with the
    factors of the reference run at that trial."""
    p = synth.make_problem(42, (7, 8, 9), 3, snr_db=30, collinearity=(0.8, 0.8, 0.8))
    eps0 = O.rel_error(p.Y, p.init)
    ref = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=30, tol=0.0)
    h = [eps0] + list(ref.history)
    acc = [h[t + 1] != h[t] for t in range(len(ref.history))]
    chg = [abs(h[t] - h[t + 1]) / h[t] for t in range(len(ref.history))]
    assert any(not a for a in acc[:25]), "the constructed history should hold a rejected trial"
    run_min, target = math.inf, None
    for t in range(len(chg)):
        if not acc[t]:
            continue
        if t >= 4 and chg[t] < run_min:
            target = t
            break
        run_min = min(run_min, chg[t])
    assert target is not None
    tol = 0.5 * (chg[target] + run_min)
    res = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=30, tol=tol)
    assert res.stop == "tol"
    assert res.iters == target + 1
    assert res.history == ref.history[:target + 1]
    ref_t = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=target + 1, tol=0.0)
    assert _rel(res.A, ref_t.A) == 0.0
    # a rejected trial never stops the run, whatever tol is: with tol above
    # every change, the run stops at the first accepted trial
    first_acc = acc.index(True)
    res2 = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=30, tol=10.0)
    assert res2.stop == "tol" and res2.iters == first_acc + 1


def test_lm_fit_mu_max_and_max_iter_stops():
    p = synth.make_problem(43, (5, 6, 7), 2, snr_db=20)
    res = O.lm_fit(p.Y, p.init, mu0=1.0, max_iter=7, tol=0.0)
    assert res.stop == "max_iter" and res.iters == 7
    # mu_max below mu_0 after any damping growth: the first rejected trial, or
    # an accepted one whose mu stays above mu_max, ends the run
    res = O.lm_fit(p.Y, p.init, mu0=1e6, max_iter=50, tol=0.0, mu_max=1e6)
    assert res.stop == "mu_max" and res.mu > 1e6

# ------------------------------------------------------------------ generator


def _angles(A):
    An = A / np.linalg.norm(A, axis=0)
    return np.degrees(np.arccos(np.clip(An.T @ An, -1, 1)))


def test_generator_angles_printed():
    rows = [l.split() for l in open(os.path.join(GOLD, "collinear_angles.txt")) if l.strip() and not l.startswith("#")]
    rng = np.random.default_rng(25)
    for nu, t1, tq in [(float(a), float(b), float(c)) for a, b, c in rows]:
        A = synth.paper_collinear(rng, 50, 5, nu)
        th = _angles(A)
        assert abs(th[0, 1] - t1) <= 0.6 and abs(th[0, 4] - t1) <= 0.6
        assert abs(th[1, 2] - tq) <= 0.6 and abs(th[3, 4] - tq) <= 0.6
        assert math.degrees(math.atan(nu)) == pytest.approx(th[0, 1], abs=1e-9)
        assert math.degrees(math.atan(nu * math.sqrt(nu * nu + 2))) == pytest.approx(th[2, 3], abs=1e-9)


def test_generator_magnitudes_printed():
    rows = [l.split() for l in open(os.path.join(GOLD, "magnitudes.txt")) if l.strip() and not l.startswith("#")]
    for N, nu, lam in rows:
        v = synth.paper_magnitudes(4, int(N), float(nu))
        assert v[0] == 1.0
        assert round(float(v[1]), 1) == float(lam)


def test_generator_appendix_f_closed_forms():
    """Appendix F: for the noiseless Eq. (modify_1) tensor with I_n = I,
    Y_(n) Y_(n)^T = U Sigma U^T, Sigma has an (R-2)-fold eigenvalue (x-1)(y-1),
    lambda_1 + lambda_R = x y + (R-2)(R+x+y) + 3, lambda_1 lambda_R = (x-1)(y-1);
    ||Y||^2 = trace(Sigma) = R^2 + (R-1)(x y - 1) (the printed
    R^2 + (R-1) x y - 1 is off by R-2)."""
    N, R, I, nu = 3, 5, 12, 0.6
    rng = np.random.default_rng(26)
    Us, As = [], []
    for _ in range(N):
        U, _ = np.linalg.qr(rng.standard_normal((I, R)))
        A = U.copy()
        A[:, 1:] = U[:, :1] + nu * U[:, 1:]
        Us.append(U)
        As.append(A)
    Y = synth.tensor_from_factors(As)
    x, y = 1 + nu * nu, (1 + nu * nu) ** (N - 1)
    S = Us[0].T @ O.unfold(Y, 0) @ O.unfold(Y, 0).T @ Us[0]
    ev = np.sort(np.linalg.eigvalsh(S))[::-1]
    assert np.allclose(ev[1:-1], (x - 1) * (y - 1), rtol=1e-10)
    assert ev[0] + ev[-1] == pytest.approx(x * y + (R - 2) * (R + x + y) + 3, rel=1e-10)
    assert ev[0] * ev[-1] == pytest.approx((x - 1) * (y - 1), rel=1e-8)
    assert float(np.sum(Y * Y)) == pytest.approx(R * R + (R - 1) * (x * y - 1), rel=1e-10)


def test_generator_snr_realised():
    rng = np.random.default_rng(27)
    Y0 = synth.tensor_from_factors([rng.standard_normal((30, 4)) for _ in range(3)])
    Y = synth.add_noise(rng, Y0, 30.0)
    snr = 10 * math.log10(float(np.sum(Y0 ** 2)) / float(np.sum((Y - Y0) ** 2)))
    assert abs(snr - 30.0) < 0.2


def test_generator_collinearity_recipe():
    rng = np.random.default_rng(28)
    A = synth.collinear_columns(rng, 20000, 4, 0.81)
    An = A / np.linalg.norm(A, axis=0)
    C = An.T @ An
    assert np.allclose(C[np.triu_indices(4, 1)], 0.81, atol=0.03)


# ------------------------------------------------------------------------- ALS


@pytest.mark.parametrize("dims,R", [((5, 6, 7), 3), ((4, 3, 5, 4), 2), ((9, 8), 3)])
def test_als_mode_update_is_the_least_squares_solution(dims, R):
    """Each mode update of the ALS rule (Sec. 3, Eq. ALS) is the minimiser of
    ||Y_(n) - A KR_n^T||_F over A: compared with numpy's least-squares solver
    (an SVD-based solve of KR_n A^T = Y_(n)^T, not the normal equations)."""
    p = synth.make_problem(31, dims, R, snr_db=20)
    A = [np.array(a) for a in p.init]
    for n in range(len(dims)):
        got = O.als_sweep(p.Y, A, modes=[n])[n]
        want = np.linalg.lstsq(O.kr_except(A, n), O.unfold(p.Y, n).T, rcond=None)[0].T
        assert _rel(got, want) < 1e-10
        A[n] = got


def test_als_update_zeroes_the_mode_gradient_and_never_raises_the_error():
    """After mode n's update its gradient block M_n - A^(n) Gamma^(n) vanishes
    (gradient pinned by finite differences above), and no update raises
    ||Y - Y_hat||."""
    p = synth.make_problem(32, (7, 8, 6), 3, snr_db=25, collinearity=(0.8, 0.8, 0.8))
    A = [np.array(a) for a in p.init]
    r2 = O.residual2(p.Y, A)
    for sweep in range(3):
        for n in range(3):
            A = O.als_sweep(p.Y, A, modes=[n])
            G = O.gradient_blocks(p.Y, A)[n]
            assert np.linalg.norm(G) < 1e-10 * max(1.0, np.linalg.norm(O.mttkrp(p.Y, A, n)))
            r2n = O.residual2(p.Y, A)
            assert r2n <= r2 * (1 + 1e-12)
            r2 = r2n


def test_als_exact_factors_are_a_fixed_point():
    """On a noiseless exact-rank tensor the generating factors are returned
    unchanged by a full sweep."""
    p = synth.make_problem(33, (6, 5, 7), 3, snr_db=None)
    A = O.als_sweep(p.Y, p.true_factors)
    assert _rel(A, p.true_factors) < 1e-11


# ------------------------------------------------------------------ HOSVD


def test_hosvd_matches_eigenvectors_of_the_unfolding_gram():
    """The oracle's HOSVD (an SVD of Y_(n)) against an independent route: the
    leading eigenvectors of Y_(n) Y_(n)^T by a symmetric eigensolver, compared
    as subspace projectors and, with the sign convention applied, column by
    column (the singular values are distinct here)."""
    p = synth.make_problem(50, (9, 10, 11), 3, snr_db=20)
    U = O.hosvd_factors(p.Y, 3)
    for n in range(3):
        Yn = O.unfold(p.Y, n)
        w, V = np.linalg.eigh(Yn @ Yn.T)
        V = O.sign_fix(V[:, ::-1][:, :3])
        assert np.allclose(U[n] @ U[n].T, V @ V.T, atol=1e-10)
        assert np.allclose(U[n], V, atol=1e-9)
        assert np.allclose(U[n].T @ U[n], np.eye(3), atol=1e-12)


def test_hosvd_recovers_orthogonal_factor_subspaces():
    """A noiseless CP tensor with orthonormal factor columns and distinct
    weights: the mode-n singular vectors are the factor columns (up to
    order and sign), so the HOSVD subspace is the factor's column space."""
    rng = np.random.default_rng(51)
    dims, R = (7, 8, 9), 3
    Q = [np.linalg.qr(rng.standard_normal((I, R)))[0] for I in dims]
    lam = np.array([5.0, 3.0, 1.5])
    Y = O.cp_full([Q[0] * lam[None, :], Q[1], Q[2]])
    U = O.hosvd_factors(Y, R)
    for n in range(3):
        assert np.allclose(U[n] @ U[n].T, Q[n] @ Q[n].T, atol=1e-12)
        # singular values of Y_(n) are the weights: columns in weight order, up to sign
        assert np.allclose(np.abs(U[n].T @ Q[n]), np.eye(R), atol=1e-12)


def test_sign_fix_convention():
    U = np.array([[0.1, -0.9], [-0.8, 0.2], [0.3, 0.1]])
    V = O.sign_fix(U)
    assert np.array_equal(V[:, 0], -U[:, 0]) and np.array_equal(V[:, 1], -U[:, 1])
    with pytest.raises(ValueError):
        O.hosvd_factors(np.zeros((2, 3, 4)), 3)


# ------------------------------------------------- Theorem 4 and MedSAE


@pytest.mark.parametrize("dims,R,mu", [((3, 4, 5), 2, 0.7), ((4, 3, 5, 3), 2, 0.2), ((5, 6), 3, 1.3)])
def test_theorem4_blocks_give_the_inverse_damped_hessian(dims, R, mu):
    """Eq. fastblock assembled from Theorem 4's blocks equals (J^T J + mu I)^{-1}
    formed from the explicit Jacobian (Lemma 2); the diagonal helper equals
    its diagonal."""
    p = synth.make_problem(70 + R, dims, R, snr_db=30)
    Gt, St = O.hinv_blocks(p.init, mu)
    H = O.hinv_from_blocks(p.init, Gt, St)
    J = O.jacobian(p.init)
    ref = np.linalg.inv(J.T @ J + mu * np.eye(J.shape[1]))
    assert _rel(H, ref) < 1e-10
    assert _rel(O.hinv_diag(p.init, Gt, St), np.diag(ref)) < 1e-10
    # St is symmetric (H is) and its size is N^2 R^4 entries, Gt N R^2
    assert _rel(St, St.T) < 1e-12


def test_sae_zero_for_permuted_scaled_sign_flipped_copy():
    rng = np.random.default_rng(80)
    A = [rng.standard_normal((I, 4)) for I in (6, 7, 8)]
    perm = np.array([2, 0, 3, 1])
    sc = [np.array([2.0, -1.0, 0.5, -3.0]), np.array([1.0, -1.0, 4.0, 1.0]), np.array([0.5, 1.0, -0.5, 2.0])]
    B = [A[n][:, perm] * sc[n][None, :] for n in range(3)]
    a2, pi = O.sae(A, B)
    assert np.allclose(a2, 0.0, atol=1e-14)
    assert np.array_equal(perm[pi], np.arange(4))


def test_sae_known_angle_and_assignment_bruteforce():
    """One column rotated by a known angle theta: alpha^2 = theta^2 there;
    the matching equals the best permutation found by enumeration."""
    rng = np.random.default_rng(81)
    A = [np.linalg.qr(rng.standard_normal((I, 5)))[0] for I in (9, 8, 7)]
    theta = 0.3
    B = [a.copy() for a in A]
    B[1][:, 2] = math.cos(theta) * A[1][:, 2] + math.sin(theta) * np.linalg.qr(
        np.column_stack([A[1], rng.standard_normal(8)]))[0][:, 5]
    a2, pi = O.sae(A, B)
    assert a2[1, 2] == pytest.approx(theta ** 2, rel=1e-12)
    assert np.allclose(np.delete(a2.ravel(), 1 * 5 + 2), 0.0, atol=1e-14)
    # assignment optimality against enumeration on noisy estimates
    for seed in range(5):
        r = np.random.default_rng(90 + seed)
        Ah = [a + 0.6 * r.standard_normal(a.shape) for a in A]
        a2, pi = O.sae(A, Ah)
        cos = np.stack([np.abs((A[n] / np.linalg.norm(A[n], axis=0)).T @ (Ah[n] / np.linalg.norm(Ah[n], axis=0)))
                        for n in range(3)]).sum(axis=0)
        best = max(itertools.permutations(range(5)), key=lambda q: sum(cos[i, q[i]] for i in range(5)))
        assert sum(cos[i, pi[i]] for i in range(5)) == pytest.approx(sum(cos[i, best[i]] for i in range(5)),
                                                                      rel=1e-12)


def test_medsae_definition():
    a2 = [np.array([[1e-4, 4e-4], [9e-4, 1e-2]]), np.array([[2.5e-3]])]
    assert O.medsae(a2) == pytest.approx(10 * math.log10(9e-4), rel=1e-12)


# --------------------------------------------------------- complex (Sec. 5)


@pytest.mark.parametrize("dims,R,mu", [((4, 5, 6), 3, 0.3), ((5, 6), 2, 2.0), ((3, 4, 3, 4), 2, 0.8)])
def test_complex_fast_step_equals_textbook(dims, R, mu):
    """Theorem 8 (with the reading of the damped inverse as Gt^T in matrix
    form) against (J^H J + mu I)^{-1} J^H e from the explicit holomorphic
    Jacobian."""
    p = synth.make_complex_problem(200 + R, dims, R, snr_db=20)
    ref = O.ctextbook_step(p.Y, p.init, mu)
    d, G, Gt, w, f = O.cflm_step(p.Y, p.init, mu)
    assert _rel(d, ref) < 1e-10


def test_complex_hessian_and_gradient_structure():
    """Theorems 5-7: J^H J = G + Z K Z^H with G = blkdiag(Gamma^(n) kron I),
    Z = blkdiag(I_R kron A^(n)), K^(n,m) = P_R diag(vec Gamma^(n,m)); the
    gradient blocks Y_(n) conj(KR_n) - A^(n) Gamma^(n)T equal J^H vec(E)."""
    p = synth.make_complex_problem(210, (3, 4, 5), 2, snr_db=20)
    A = p.init
    J = O.jacobian(A)
    H = J.conj().T @ J
    g = O.cgrams(A)
    R = 2
    Gm = sla.block_diag(*[np.kron(g.Gamma(n), np.eye(a.shape[0])) for n, a in enumerate(A)])
    Z = sla.block_diag(*[np.kron(np.eye(R), a) for a in A])
    _, _, K = O.cspd_core(A, 1.0)
    assert _rel(H, Gm + Z @ K @ Z.conj().T) < 1e-13
    e = O.vec(p.Y - O.cp_full(A))
    assert _rel(O.join_params(O.cgradient_blocks(p.Y, A)), J.conj().T @ e) < 1e-13


def test_complex_gradient_finite_differences():
    """f(a) = ||Y - Y_hat(a)||^2: a real step h e_k changes f by -2 h Re g_k,
    an imaginary step i h e_k by -2 h Im g_k (g = J^H vec(E))."""
    p = synth.make_complex_problem(211, (3, 4, 3), 2, snr_db=10)
    dims, R = p.dims, p.R
    a = O.join_params(p.init)
    g = O.join_params(O.cgradient_blocks(p.Y, p.init))
    f = lambda x: float(np.sum(np.abs(p.Y - O.cp_full(O.split_params(x, dims, R))) ** 2))
    h = 1e-6
    for k in (0, 5, 11, len(a) - 1):
        e = np.zeros_like(a)
        e[k] = h
        dre = (f(a + e) - f(a - e)) / (2 * h)
        dim = (f(a + 1j * e) - f(a - 1j * e)) / (2 * h)
        assert dre == pytest.approx(-2 * g[k].real, rel=1e-6, abs=1e-8)
        assert dim == pytest.approx(-2 * g[k].imag, rel=1e-6, abs=1e-8)


def test_complex_spd_core_gives_the_fast_f():
    p = synth.make_complex_problem(212, (5, 6, 4), 3, snr_db=20)
    mu = 0.4
    core, S, K = O.cspd_core(p.init, mu)
    assert _rel(core, core.conj().T) < 1e-14
    assert np.min(np.linalg.eigvalsh(core)) > 0
    _, _, _, w, f = O.cflm_step(p.Y, p.init, mu)
    Kw = K @ w
    fs = Kw - K @ (S @ np.linalg.solve(core, S.conj().T @ Kw))
    assert _rel(fs, f) < 1e-12


def test_complex_noiseless_converges():
    p = synth.make_complex_problem(213, (7, 8, 6), 3, snr_db=None)
    rng = np.random.default_rng(214)
    A0 = [a + 0.3 * (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)) for a in p.true_factors]
    res = O.clm_fit(p.Y, A0, mu0=1.0, max_iter=300)
    assert res.rel_err < 1e-10
