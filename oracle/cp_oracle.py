"""CPU oracle for the low-complexity damped Gauss-Newton (fLM) step for CP.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run this module; the
product path (the CUDA library and its Python binding) never does, and this
module imports nothing from it.  Everything is float64 numpy; library
primitives (matmul, solve, Cholesky) serve as steps, with no blocking,
fusion or reordering beyond what the cited definitions state.

Paper: A.-H. Phan, P. Tichavsky, A. Cichocki, "Low Complexity Damped
Gauss-Newton Algorithms for CANDECOMP/PARAFAC" (arXiv 1205.2584).

Conventions (Sec. 2; Appendix A):
  * ``vec`` is column-major (first index fastest); the mode-n unfolding
    Y_(n) has rows i_n and columns ordered with the remaining indices, the
    earliest fastest (Kolda's convention), so that
    Y_(n) = A^(n) (KR_n)^T with KR_n = A^(N) (.) ... A^(n+1) (.) A^(n-1) (.) ... A^(1).
  * The parameter vector is a = [vec A^(1); ...; vec A^(N)] (Eq. vecV).
  * Modes are 0-based in code (n = 0 .. N-1).

Two independent routes to the same step (Theorem 3 is an identity):
  * ``textbook_step``: forms J (Lemma 2), H = J^T J and g = J^T vec(E),
    solves (H + mu I) d = g by Cholesky (Eq. GaussNewton_v2).  Tiny inputs.
  * ``flm_step``: Algorithm 1 with variant fLM_a (Sec. 4.4 (a)): K, Psi,
    Phi_1 = I + Psi K, f = K Phi_1^{-1} w by LU with partial pivoting,
    then the factor update of Theorem 1 (Eq. fast_low_LM1a).

Readings where the paper is garbled or silent (each applies to both routes
and to the GPU path):
  * w (Theorem 1, Eq. proj_ZGJE_LMa) prints "Gamma Gt_mu" with Gamma the
    Hadamard product of all Gramians; the proof in Appendix D (first line of
    Eq. proj_ZGJE_LM) gives w_n = vec(A^(n)T (A_mu^(n) - A^(n) Gamma^(n) Gt^(n))),
    i.e. the matrix product C^(n) Gamma^(n), which is what J^T-based w equals.
  * Nielsen's damping rule (Sec. 4.6) prints "2 max{...}" without mu; the
    cited rule is mu <- mu max{1/3, 1 - (2 rho - 1)^3}, nu <- 2 if rho > 0,
    else mu <- mu nu, nu <- 2 nu.
  * A trial step is accepted iff ||e_t|| < ||e_{t-1}|| (Sec. 4.6).
  * Normalisation (Algorithm 1 step 10): after an accepted step every
    component's energy is spread equally over the modes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg as sla

# ---------------------------------------------------------------------------
# Tensor algebra (Sec. 2, Notation 1; Appendix A)
# ---------------------------------------------------------------------------


def unfold(Y: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding Y_(n) (I_n x prod_{k != n} I_k), Kolda's column order."""
    return np.reshape(np.moveaxis(Y, n, 0), (Y.shape[n], -1), order="F")


def khatri_rao(mats: Sequence[np.ndarray]) -> np.ndarray:
    """Column-wise Kronecker product mats[0] (.) mats[1] (.) ...; the row index
    of the last matrix runs fastest (Sec. 2)."""
    out = mats[0]
    R = out.shape[1]
    for M in mats[1:]:
        out = (out[:, None, :] * M[None, :, :]).reshape(-1, R)
    return out


def kr_except(A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """KR_n = A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1) (Notation 1)."""
    return khatri_rao([A[k] for k in reversed(range(len(A))) if k != n])


def cp_full(A: Sequence[np.ndarray]) -> np.ndarray:
    """Y_hat = sum_r a_r^(1) o ... o a_r^(N) (Eq. CP_nolambda), built through
    its mode-1 unfolding Y_hat_(1) = A^(1) KR_1^T."""
    dims = tuple(a.shape[0] for a in A)
    Y1 = A[0] @ kr_except(A, 0).T
    return np.reshape(Y1, dims, order="F")


def vec(X: np.ndarray) -> np.ndarray:
    return np.reshape(X, -1, order="F")


def unvec(v: np.ndarray, shape) -> np.ndarray:
    return np.reshape(v, shape, order="F")


def perm_PR(R: int) -> np.ndarray:
    """Commutation matrix P_R with P_R vec(X^T) = vec(X) for X (R x R) (Theorem 1)."""
    P = np.zeros((R * R, R * R))
    for i in range(R):
        for j in range(R):
            # vec(X)[i + R j] = X[i, j] = vec(X^T)[j + R i]
            P[i + R * j, j + R * i] = 1.0
    return P


def commutation_Qn(dims: Sequence[int], n: int) -> np.ndarray:
    """Q_n with vec(Y) = Q_n vec(Y_(n)) (Lemma 1 of Appendix A), built from the
    definition of the unfolding as a permutation of entries."""
    J = int(np.prod(dims))
    idx = np.arange(J).reshape(dims, order="F")
    src = vec(unfold(idx, n))          # position p of vec(Y_(n)) holds vec(Y)[src[p]]
    Q = np.zeros((J, J))
    Q[src, np.arange(J)] = 1.0
    return Q


# ---------------------------------------------------------------------------
# Gramians (Sec. 3 Eq. ALS; Theorem 1 Eq. Gamma_a)
# ---------------------------------------------------------------------------


@dataclass
class Grams:
    C: List[np.ndarray]            # C^(n) = A^(n)T A^(n)
    Gamma_nm: np.ndarray           # [n, m] -> Gamma^(n,m) = Hadamard_{k != n, m} C^(k)
    Gamma_all: np.ndarray          # Gamma = Hadamard_k C^(k)

    def Gamma(self, n: int) -> np.ndarray:
        return self.Gamma_nm[n, n]


def grams(A: Sequence[np.ndarray]) -> Grams:
    N = len(A)
    R = A[0].shape[1]
    C = [a.T @ a for a in A]
    G = np.empty((N, N, R, R))
    for n in range(N):
        for m in range(N):
            P = np.ones((R, R))
            for k in range(N):
                if k != n and k != m:
                    P = P * C[k]
            G[n, m] = P
    full = np.ones((R, R))
    for k in range(N):
        full = full * C[k]
    return Grams(C=C, Gamma_nm=G, Gamma_all=full)


# ---------------------------------------------------------------------------
# Gradient quantities (Sec. 4.6 Eq. mappingJ; Sec. 3)
# ---------------------------------------------------------------------------


def mttkrp(Y: np.ndarray, A: Sequence[np.ndarray], n: int) -> np.ndarray:
    """M_n = Y_(n) KR_n (the damped-ALS numerator, Algorithm 1 step 6)."""
    return unfold(Y, n) @ kr_except(A, n)


def mttkrp_all(Y, A) -> List[np.ndarray]:
    return [mttkrp(Y, A, n) for n in range(len(A))]


def residual2(Y: np.ndarray, A: Sequence[np.ndarray]) -> float:
    """||E||_F^2 with E = Y - Y_hat, summed directly (no expansion)."""
    E = Y - cp_full(A)
    return float(np.sum(E * E))


def rel_error(Y, A) -> float:
    """epsilon = ||Y - Y_hat||_F / ||Y||_F (Sec. 6.1)."""
    return math.sqrt(residual2(Y, A)) / float(np.linalg.norm(Y))


def gradient_blocks(Y, A, M: Optional[List[np.ndarray]] = None,
                    g: Optional[Grams] = None) -> List[np.ndarray]:
    """g = J^T vec(E) in blocks G_n = M_n - A^(n) Gamma^(n) (Eq. mappingJ)."""
    if M is None:
        M = mttkrp_all(Y, A)
    if g is None:
        g = grams(A)
    return [M[n] - A[n] @ g.Gamma(n) for n in range(len(A))]


# ---------------------------------------------------------------------------
# Textbook dGN (Sec. 3 Eq. GaussNewton_v2; Lemma 2 Eq. Jacobian)
# ---------------------------------------------------------------------------


def jacobian(A: Sequence[np.ndarray]) -> np.ndarray:
    """J = [Q_n (KR_n kron I_{I_n})]_n, the Jacobian of vec(Y_hat) w.r.t. a."""
    dims = [a.shape[0] for a in A]
    blocks = []
    for n in range(len(A)):
        blocks.append(commutation_Qn(dims, n) @ np.kron(kr_except(A, n), np.eye(dims[n])))
    return np.hstack(blocks)


def split_params(x: np.ndarray, dims: Sequence[int], R: int) -> List[np.ndarray]:
    out, off = [], 0
    for I in dims:
        out.append(unvec(x[off:off + I * R], (I, R)))
        off += I * R
    return out


def join_params(A: Sequence[np.ndarray]) -> np.ndarray:
    return np.concatenate([vec(a) for a in A])


def textbook_step(Y: np.ndarray, A: Sequence[np.ndarray], mu: float) -> List[np.ndarray]:
    """d = (J^T J + mu I)^{-1} J^T vec(Y - Y_hat), solved by Cholesky."""
    J = jacobian(A)
    e = vec(Y - cp_full(A))
    H = J.T @ J
    gvec = J.T @ e
    d = sla.cho_solve(sla.cho_factor(H + mu * np.eye(H.shape[0]), lower=True), gvec)
    return split_params(d, [a.shape[0] for a in A], A[0].shape[1])


# ---------------------------------------------------------------------------
# Structured Hessian pieces (Theorem 2; Theorem 1 Eq. Knm_a; Appendix E)
# ---------------------------------------------------------------------------


def kernel_K(g: Grams) -> np.ndarray:
    """K = [K^(n,m)], K^(n,m) = (1 - delta_nm) P_R diag(vec Gamma^(n,m)) (Eq. Knm_a)."""
    N, R = g.Gamma_nm.shape[0], g.Gamma_nm.shape[2]
    P = perm_PR(R)
    R2 = R * R
    K = np.zeros((N * R2, N * R2))
    for n in range(N):
        for m in range(N):
            if n != m:
                K[n * R2:(n + 1) * R2, m * R2:(m + 1) * R2] = P @ np.diag(vec(g.Gamma_nm[n, m]))
    return K


def kernel_K_inverse_closed_form(g: Grams) -> np.ndarray:
    """Appendix E, Eq. inv_K: K~^(n,m) = (1/(N-1) - delta_nm) diag(vec(C^(n) * C^(m) / Gamma)) P_R."""
    N, R = g.Gamma_nm.shape[0], g.Gamma_nm.shape[2]
    P = perm_PR(R)
    R2 = R * R
    Kt = np.zeros((N * R2, N * R2))
    for n in range(N):
        for m in range(N):
            coef = 1.0 / (N - 1) - (1.0 if n == m else 0.0)
            D = np.diag(vec(g.C[n] * g.C[m] / g.Gamma_all))
            Kt[n * R2:(n + 1) * R2, m * R2:(m + 1) * R2] = coef * D @ P
    return Kt


def block_G(g: Grams, dims: Sequence[int]) -> np.ndarray:
    """G = blkdiag(Gamma^(n) kron I_{I_n}) (Theorem 2, Eq. G)."""
    return sla.block_diag(*[np.kron(g.Gamma(n), np.eye(I)) for n, I in enumerate(dims)])


def block_Z(A: Sequence[np.ndarray]) -> np.ndarray:
    """Z = blkdiag(I_R kron A^(n)) (Theorem 2, Eq. Z)."""
    R = A[0].shape[1]
    return sla.block_diag(*[np.kron(np.eye(R), a) for a in A])


def damped_inverses(g: Grams, mu: float) -> List[np.ndarray]:
    """Gt_mu^(n) = (Gamma^(n) + mu I)^{-1} (Algorithm 1 step 5)."""
    R = g.Gamma_nm.shape[2]
    return [np.linalg.inv(g.Gamma(n) + mu * np.eye(R)) for n in range(g.Gamma_nm.shape[0])]


def psi_mu(g: Grams, Gt: Sequence[np.ndarray]) -> np.ndarray:
    """Psi_mu = blkdiag(Gt_mu^(n) kron C^(n)) (Eq. ZiGZ_LM_a)."""
    return sla.block_diag(*[np.kron(Gt[n], g.C[n]) for n in range(len(Gt))])


# ---------------------------------------------------------------------------
# Fast dGN step, Algorithm 1 / Theorem 1, variant fLM_a
# ---------------------------------------------------------------------------


@dataclass
class FastStep:
    delta: List[np.ndarray]        # Delta A^(n) = A_new^(n) - A^(n)
    A_new: List[np.ndarray]
    G: List[np.ndarray]            # gradient blocks at the old point
    Gt: List[np.ndarray]           # Gt_mu^(n)
    w: np.ndarray                  # w_mu (N R^2)
    f: np.ndarray                  # f = B_mu w_mu (N R^2)
    M: List[np.ndarray]            # M_n = Y_(n) KR_n


def w_mu(A, M, g: Grams, Gt) -> np.ndarray:
    """w_n = vec(A^(n)T (A_mu^(n) - A^(n) Gamma^(n) Gt^(n))), Appendix D (the
    step before Eq. proj_ZGJE_LM), with A_mu^(n) = M_n Gt^(n)."""
    parts = []
    for n in range(len(A)):
        A_mu = M[n] @ Gt[n]
        parts.append(vec(A[n].T @ (A_mu - A[n] @ g.Gamma(n) @ Gt[n])))
    return np.concatenate(parts)


def flm_step(Y, A, mu: float, variant: str = "a", M=None) -> FastStep:
    """One fast dGN step (Algorithm 1 steps 2-9, Theorem 1).

    variant "a": f = K (I + Psi K)^{-1} w, LU with partial pivoting (fLM_a).
    variant "b": f = (K^{-1} + Psi)^{-1} w with K^{-1} from Appendix E (fLM_b);
    requires every entry of every Gamma^(n,m) to be non-zero.
    """
    N = len(A)
    R = A[0].shape[1]
    R2 = R * R
    g = grams(A)                                   # step 3 (C, Gamma^(n,m))
    if M is None:
        M = mttkrp_all(Y, A)                       # step 6 numerator
    K = kernel_K(g)                                # step 3
    Gt = damped_inverses(g, mu)                    # step 5
    w = w_mu(A, M, g, Gt)                          # step 7
    Psi = psi_mu(g, Gt)                            # step 8
    if variant == "a":
        Phi1 = np.eye(N * R2) + Psi @ K
        f = K @ np.linalg.solve(Phi1, w)           # step 9, Eq. inverse_f1a
    elif variant == "b":
        Phi2 = kernel_K_inverse_closed_form(g) + Psi
        f = np.linalg.solve(Phi2, w)               # step 9, Eq. inverse_f2a
    else:
        raise ValueError(variant)
    A_new, delta = [], []
    for n in range(N):                             # step 10-11, Eq. fast_low_LM1a
        Fn = unvec(f[n * R2:(n + 1) * R2], (R, R))
        A_mu = M[n] @ Gt[n]
        An = A_mu + A[n] @ (np.eye(R) - (Fn + g.Gamma(n)) @ Gt[n])
        A_new.append(An)
        delta.append(An - A[n])
    G = gradient_blocks(Y, A, M, g)
    return FastStep(delta=delta, A_new=A_new, G=G, Gt=Gt, w=w, f=f, M=M)


# ---------------------------------------------------------------------------
# Symmetric positive definite form of the core system (reading of Sec. 4.4)
# ---------------------------------------------------------------------------


def spd_core_factors(g: Grams, mu: float) -> List[np.ndarray]:
    """S_n with S_n S_n^T = Psi_mu^(n) = Gt^(n) kron C^(n): S_n = U_n kron L_n, where
    Gamma^(n) + mu I = L_G L_G^T, U_n = L_G^{-T} (so U_n U_n^T = Gt^(n)) and
    C^(n) = L_n L_n^T (lower Cholesky factors)."""
    N, R = g.Gamma_nm.shape[0], g.Gamma_nm.shape[2]
    S = []
    for n in range(N):
        LG = np.linalg.cholesky(g.Gamma(n) + mu * np.eye(R))
        U = np.linalg.inv(LG).T
        LC = np.linalg.cholesky(g.C[n])
        S.append(np.kron(U, LC))
    return S


def spd_core(A, mu: float) -> np.ndarray:
    """Core matrix Mc = I + S^T K S (N R^2 square, SPD when every A^(n) has full
    column rank).  Because K (I + Psi K)^{-1} = K - K S Mc^{-1} S^T K (push-through
    identity with Psi = S S^T), f = B_mu w can be obtained from Mc."""
    g = grams(A)
    S = sla.block_diag(*spd_core_factors(g, mu))
    K = kernel_K(g)
    return np.eye(S.shape[0]) + S.T @ K @ S


def f_from_spd_core(A, mu: float, w: np.ndarray) -> np.ndarray:
    """f = K w - K S Mc^{-1} S^T K w (equal to B_mu w)."""
    g = grams(A)
    S = sla.block_diag(*spd_core_factors(g, mu))
    K = kernel_K(g)
    Mc = np.eye(S.shape[0]) + S.T @ K @ S
    Kw = K @ w
    y = sla.cho_solve(sla.cho_factor(Mc, lower=True), S.T @ Kw)
    return Kw - K @ (S @ y)


# ---------------------------------------------------------------------------
# Levenberg-Marquardt control (Sec. 4.6), normalisation (Algorithm 1 step 10)
# ---------------------------------------------------------------------------


def nielsen_update(mu: float, nu: float, rho: float):
    """Damping update of Sec. 4.6 in Nielsen's form (reading: the printed rule
    drops the factor mu).  Returns (mu, nu)."""
    if rho > 0:
        return mu * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), 2.0
    return mu * nu, 2.0 * nu


def gain_ratio(r2_old: float, r2_new: float, delta, G, mu: float) -> float:
    """rho = (||e_{t-1}||^2 - ||e_t||^2) / (Delta a^T (g + mu Delta a)) (Sec. 4.6).

    The denominator equals Delta^T H Delta + 2 mu ||Delta||^2 >= 0; when it is
    not positive (a step that underflowed to zero) rho is read as 0, i.e. the
    trial counts as rejected."""
    den = sum(float(np.sum(d * (gn + mu * d))) for d, gn in zip(delta, G))
    if not den > 0.0:
        return 0.0
    return (r2_old - r2_new) / den


def normalize_equal_energy(A: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Scale component r in every mode to norm lambda_r^(1/N), lambda_r =
    prod_n ||a_r^(n)|| (signs and Y_hat unchanged); components with a zero
    column are left as they are."""
    N = len(A)
    norms = np.stack([np.linalg.norm(a, axis=0) for a in A])     # N x R
    out = [a.copy() for a in A]
    for r in range(A[0].shape[1]):
        if np.any(norms[:, r] == 0):
            continue
        lam = float(np.prod(norms[:, r]))
        target = lam ** (1.0 / N)
        for n in range(N):
            out[n][:, r] = A[n][:, r] * (target / norms[n, r])
    return out


def initial_mu(A, tau: float = 1e-3) -> float:
    """mu_0 = tau max diag(H) = tau max_n max diag Gamma^(n) (Eq. mu0)."""
    g = grams(A)
    return tau * max(float(np.max(np.diag(g.Gamma(n)))) for n in range(len(A)))


@dataclass
class LMResult:
    A: List[np.ndarray]
    resid2: float
    rel_err: float
    iters: int                     # every trial step
    accepted: int
    mu: float
    stop: str
    history: List[float] = field(default_factory=list)   # epsilon after each trial


def lm_fit(Y, A0, mu0: Optional[float] = None, max_iter: int = 200, tol: float = 0.0,
           normalize: bool = True, tau: float = 1e-3, mu_max: float = 1e30,
           step: str = "fast") -> LMResult:
    """Algorithm 1's outer loop with the Sec. 4.6 damping control.

    Every trial counts as an iteration.  Stop on an accepted step whose
    relative change |eps_{t-1} - eps_t| / eps_{t-1} < tol, when mu > mu_max, or
    after max_iter trials.  ``step="textbook"`` replaces the fast step by the
    full (J^T J + mu I) solve (tiny inputs only)."""
    A = [np.array(a, dtype=np.float64, copy=True) for a in A0]
    ynorm = float(np.linalg.norm(Y))
    mu = initial_mu(A, tau) if mu0 is None else float(mu0)
    nu = 2.0
    r2 = residual2(Y, A)
    M = mttkrp_all(Y, A)
    hist = []
    accepted = 0
    stop = "max_iter"
    it = 0
    while it < max_iter:
        it += 1
        if step == "textbook":
            d = textbook_step(Y, A, mu)
            st = FastStep(delta=d, A_new=[a + x for a, x in zip(A, d)],
                          G=gradient_blocks(Y, A, M), Gt=[], w=np.empty(0),
                          f=np.empty(0), M=M)
        else:
            st = flm_step(Y, A, mu, M=M)
        r2_new = residual2(Y, st.A_new)
        rho = gain_ratio(r2, r2_new, st.delta, st.G, mu)
        if r2_new < r2:
            eps_old, eps_new = math.sqrt(r2) / ynorm, math.sqrt(r2_new) / ynorm
            A = normalize_equal_energy(st.A_new) if normalize else st.A_new
            r2 = r2_new
            M = mttkrp_all(Y, A)
            accepted += 1
            mu, nu = nielsen_update(mu, nu, rho)
            hist.append(eps_new)
            if eps_old > 0 and abs(eps_old - eps_new) / eps_old < tol:
                stop = "tol"
                break
        else:
            mu, nu = nielsen_update(mu, nu, rho)
            hist.append(math.sqrt(r2) / ynorm)
        if mu > mu_max:
            stop = "mu_max"
            break
    return LMResult(A=A, resid2=r2, rel_err=math.sqrt(r2) / ynorm, iters=it,
                    accepted=accepted, mu=mu, stop=stop, history=hist)


# ---------------------------------------------------------------------------
# ALS (Sec. 3, Eq. ALS): the initialisation sweeps run before fLM (Sec. 4.6)
# ---------------------------------------------------------------------------


def als_sweep(Y: np.ndarray, A: Sequence[np.ndarray],
              modes: Optional[Sequence[int]] = None) -> List[np.ndarray]:
    """One sweep of the ALS rule: for n in ``modes`` (every mode, in order, by
    default) A^(n) <- Y_(n) KR_n (Gamma^(n))^+, with Gamma^(n) = Hadamard_{k != n}
    C^(k) formed from the current factors (modes earlier in the sweep already
    replaced).  The pseudo-inverse is the one the rule prints; it is the
    inverse whenever the other factors have full column rank."""
    A = [np.array(a, dtype=np.float64, copy=True) for a in A]
    for n in (range(len(A)) if modes is None else modes):
        A[n] = mttkrp(Y, A, n) @ np.linalg.pinv(grams(A).Gamma(n))
    return A


# ---------------------------------------------------------------------------
# HOSVD initialisation (Algorithm 1 step 1; Sec. 4.6: the factors are often
# initialised with the mode-n singular vectors of the data tensor, then a few
# ALS sweeps are run)
# ---------------------------------------------------------------------------


def sign_fix(U: np.ndarray) -> np.ndarray:
    """Sign convention for singular vectors (they are defined up to sign):
    each column is flipped so that its entry of largest magnitude is positive
    (the first such entry on ties)."""
    U = np.array(U, dtype=np.float64, copy=True)
    for r in range(U.shape[1]):
        k = int(np.argmax(np.abs(U[:, r])))
        if U[k, r] < 0:
            U[:, r] = -U[:, r]
    return U


def hosvd_factors(Y: np.ndarray, R: int) -> List[np.ndarray]:
    """A^(n) = the R leading left singular vectors of the unfolding Y_(n)
    (descending singular values, sign_fix applied); needs R <= I_n."""
    out = []
    for n in range(Y.ndim):
        if R > Y.shape[n]:
            raise ValueError("HOSVD initialisation needs R <= I_n in every mode")
        U, s, _ = np.linalg.svd(unfold(Y, n), full_matrices=False)
        out.append(sign_fix(U[:, :R]))
    return out


# ---------------------------------------------------------------------------
# Theorem 4: the damped Hessian's inverse in block form (memory saving), and
# the MedSAE measure of Sec. 6 (Eq. MedSAE)
# ---------------------------------------------------------------------------


def hinv_blocks(A, mu: float):
    """Theorem 4's compact representation of H_mu^{-1}: Gt^(n) (N matrices
    R x R) and St = D B_mu D (N R^2 x N R^2), D = blkdiag(Gt^(n) kron I_R),
    B_mu = K (I + Psi_mu K)^{-1} (Eq. inverse_f1a); block (n, m) of St is
    St^(n,m).  Reading: the proof's B^(n,m) is the (n, m) block of B_mu (the
    block the product L_mu B_mu L_mu^T places at (n, m))."""
    g = grams(A)
    N, R = len(A), A[0].shape[1]
    Gt = damped_inverses(g, mu)
    K = kernel_K(g)
    Psi = psi_mu(g, Gt)
    n = N * R * R
    B = K @ np.linalg.inv(np.eye(n) + Psi @ K)
    D = sla.block_diag(*[np.kron(Gt[k], np.eye(R)) for k in range(N)])
    return Gt, D @ B @ D


def hinv_from_blocks(A, Gt, St) -> np.ndarray:
    """Eq. fastblock: H_mu^{-1} block (n, m) =
    delta_nm (Gt^(n) kron I_{I_n}) - (I_R kron A^(n)) St^(n,m) (I_R kron A^(m)T)."""
    N, R = len(A), A[0].shape[1]
    dims = [a.shape[0] for a in A]
    offs = np.concatenate([[0], np.cumsum([R * I for I in dims])])
    R2 = R * R
    H = np.zeros((offs[-1], offs[-1]))
    for n in range(N):
        for m in range(N):
            blk = -np.kron(np.eye(R), A[n]) @ St[n * R2:(n + 1) * R2, m * R2:(m + 1) * R2] @ \
                np.kron(np.eye(R), A[m].T)
            if n == m:
                blk = blk + np.kron(Gt[n], np.eye(dims[n]))
            H[offs[n]:offs[n + 1], offs[m]:offs[m + 1]] = blk
    return H


def hinv_diag(A, Gt, St) -> np.ndarray:
    """Diagonal of H_mu^{-1} from Theorem 4's blocks, entry by entry in the
    parameter order of Eq. vecV (A^(n)[i, r] at i + I_n r of block n):
    Gt^(n)[r, r] - sum_{s, s'} A^(n)[i, s] St^(n,n)[s + R r, s' + R r] A^(n)[i, s']."""
    N, R = len(A), A[0].shape[1]
    R2 = R * R
    out = []
    for n in range(N):
        I = A[n].shape[0]
        Snn = St[n * R2:(n + 1) * R2, n * R2:(n + 1) * R2]
        d = np.empty(I * R)
        for r in range(R):
            blk = Snn[r * R:(r + 1) * R, r * R:(r + 1) * R]
            for i in range(I):
                d[i + I * r] = Gt[n][r, r] - A[n][i] @ blk @ A[n][i]
        out.append(d)
    return np.concatenate(out)


def sae(A_true, A_est):
    """Squared angular errors alpha^2 of Eq. MedSAE per mode and component
    after matching the components' order: the permutation pi maximises
    sum_r sum_n |cos(a_r^(n), ahat_pi(r)^(n))| (a linear assignment), and
    alpha_r^(n) = arccos |cos(a_r^(n), ahat_pi(r)^(n))| (reading: the absolute
    value, since CP determines a component's sign only up to flips that
    cancel across modes).  Returns (alpha2 N x R, pi)."""
    from scipy.optimize import linear_sum_assignment
    N, R = len(A_true), A_true[0].shape[1]
    cos = np.empty((N, R, R))
    for n in range(N):
        a = A_true[n] / np.linalg.norm(A_true[n], axis=0)
        b = A_est[n] / np.linalg.norm(A_est[n], axis=0)
        cos[n] = np.abs(a.T @ b)
    score = cos.sum(axis=0)
    rows, pi = linear_sum_assignment(-score)
    alpha2 = np.empty((N, R))
    for n in range(N):
        for r in range(R):
            alpha2[n, r] = math.acos(min(1.0, cos[n, r, pi[r]])) ** 2
    return alpha2, pi


def medsae(alpha2_runs) -> float:
    """MedSAE (Eq. MedSAE) in dB: 10 log10 of the median of the squared
    angular errors over every run, mode and component given."""
    v = np.concatenate([np.ravel(a) for a in alpha2_runs])
    return 10.0 * math.log10(float(np.median(v)))


# ---------------------------------------------------------------------------
# Complex-valued tensors (Sec. 5: Theorems 5-8).  The model Y_hat is
# holomorphic in the factors; the damped Gauss-Newton update is
# a <- a + (J^H J + mu I)^{-1} J^H vec(Y - Y_hat) (Eq. GaussNewton_v_complex).
# C^(n) = A^(n)H A^(n) (Hermitian), Gamma^(n,m) = Hadamard_{k != n,m} C^(k).
# ---------------------------------------------------------------------------


def cgrams(A):
    """Complex Gramians: C^(n) = A^(n)H A^(n), Gamma^(n,m), Gamma (Theorem 5)."""
    N = len(A)
    R = A[0].shape[1]
    C = [a.conj().T @ a for a in A]
    G = np.empty((N, N, R, R), dtype=complex)
    for n in range(N):
        for m in range(N):
            P = np.ones((R, R), dtype=complex)
            for k in range(N):
                if k != n and k != m:
                    P = P * C[k]
            G[n, m] = P
    full = np.ones((R, R), dtype=complex)
    for k in range(N):
        full = full * C[k]
    return Grams(C=C, Gamma_nm=G, Gamma_all=full)


def cgradient_blocks(Y, A):
    """g = J^H vec(E) in blocks Y_(n) (Hadamard... ) : G_n = Y_(n) conj(KR_n) - A^(n) Gamma^(n)T
    (Theorem 7, Eq. grad_complex_g)."""
    g = cgrams(A)
    return [unfold(Y, n) @ kr_except(A, n).conj() - A[n] @ g.Gamma(n).T for n in range(len(A))]


def ctextbook_step(Y, A, mu: float):
    """(J^H J + mu I)^{-1} J^H vec(Y - Y_hat) with the holomorphic Jacobian of
    Lemma 2 (complex factors), solved by Cholesky (Hermitian)."""
    J = jacobian(A)
    e = vec(Y - cp_full(A))
    H = J.conj().T @ J
    gvec = J.conj().T @ e
    d = sla.cho_solve(sla.cho_factor(H + mu * np.eye(H.shape[0]), lower=True), gvec)
    return split_params(d, [a.shape[0] for a in A], A[0].shape[1])


def cflm_step(Y, A, mu: float, G=None):
    """Theorem 8's fast complex step.  Kronecker-form Psi_mu = blkdiag(Gt^(n)
    kron C^(n)) with Gt^(n) = (Gamma^(n) + mu I)^{-1} (Eq. ZiGZ_LM_cplx),
    K = [P_R diag(vec Gamma^(n,m))] (Theorem 6), B_mu = K (I + Psi_mu K)^{-1};
    in matrix form the damped inverse acts as X -> X Gt^(n)T (reading: the
    printed Gt of the matrix-form update is the transpose (Gamma^(n)T + mu I)^{-1},
    the form the paper's own earlier statement of the update uses), so
      A_mu = Y_(n) conj(KR_n) Gt^T,   w_n = vec(A^(n)H (A_mu - A^(n) Gamma^(n)T Gt^T)),
      Delta_n = A_mu + A^(n) (I - (F_n + Gamma^(n)T) Gt^T) - A^(n)   (Eq. fast_low_LM1-complex).
    G (optional): the gradient blocks to use (M_n = G_n + A^(n) Gamma^(n)T).
    Returns (delta, G, Gt, w, f)."""
    N = len(A)
    R = A[0].shape[1]
    R2 = R * R
    g = cgrams(A)
    P = perm_PR(R)
    K = np.zeros((N * R2, N * R2), dtype=complex)
    for n in range(N):
        for m in range(N):
            if n != m:
                K[n * R2:(n + 1) * R2, m * R2:(m + 1) * R2] = P @ np.diag(vec(g.Gamma_nm[n, m]))
    Gt = [np.linalg.inv(g.Gamma(n) + mu * np.eye(R)) for n in range(N)]
    Psi = sla.block_diag(*[np.kron(Gt[n], g.C[n]) for n in range(N)])
    if G is None:
        M = [unfold(Y, n) @ kr_except(A, n).conj() for n in range(N)]
    else:
        M = [G[n] + A[n] @ g.Gamma(n).T for n in range(N)]
    parts = []
    for n in range(N):
        A_mu = M[n] @ Gt[n].T
        parts.append(vec(A[n].conj().T @ (A_mu - A[n] @ g.Gamma(n).T @ Gt[n].T)))
    w = np.concatenate(parts)
    f = K @ np.linalg.solve(np.eye(N * R2) + Psi @ K, w)
    delta, G = [], []
    for n in range(N):
        Fn = unvec(f[n * R2:(n + 1) * R2], (R, R))
        A_mu = M[n] @ Gt[n].T
        An = A_mu + A[n] @ (np.eye(R) - (Fn + g.Gamma(n).T) @ Gt[n].T)
        delta.append(An - A[n])
        G.append(M[n] - A[n] @ g.Gamma(n).T)
    return delta, G, Gt, w, f


def clm_fit(Y, A0, mu0: Optional[float] = None, max_iter: int = 200, tol: float = 0.0,
            normalize: bool = True, tau: float = 1e-3, mu_max: float = 1e30) -> LMResult:
    """The LM loop of lm_fit for complex tensors with the fast complex step:
    the same acceptance, Nielsen rule and stop tests; the gain ratio's
    denominator is Re(Delta^H (g + mu Delta)) (the decrease of ||E||^2 the
    linear model predicts); normalisation spreads each component's norm
    equally over the modes with real positive scales (phases kept); mu_0 =
    tau max diag(H) = tau max_n max Gamma^(n)[r, r]."""
    A = [np.array(a, dtype=complex, copy=True) for a in A0]
    ynorm = float(np.linalg.norm(Y))
    if mu0 is None:
        g0 = cgrams(A)
        mu = tau * max(float(np.max(np.real(np.diag(g0.Gamma(n))))) for n in range(len(A)))
    else:
        mu = float(mu0)
    nu = 2.0

    def r2(A):
        E = Y - cp_full(A)
        return float(np.sum(np.abs(E) ** 2))
    rr = r2(A)
    hist, accepted, stop, it = [], 0, "max_iter", 0
    while it < max_iter:
        it += 1
        delta, G, _, _, _ = cflm_step(Y, A, mu)
        An = [a + d for a, d in zip(A, delta)]
        rn = r2(An)
        den = sum(float(np.real(np.vdot(d, gn + mu * d))) for d, gn in zip(delta, G))
        rho = (rr - rn) / den if den > 0 else 0.0
        if rn < rr:
            eo, en = math.sqrt(rr) / ynorm, math.sqrt(rn) / ynorm
            if normalize:
                norms = np.stack([np.linalg.norm(a, axis=0) for a in An])
                for r in range(An[0].shape[1]):
                    if np.all(norms[:, r] > 0):
                        t = float(np.prod(norms[:, r])) ** (1.0 / len(An))
                        for n in range(len(An)):
                            An[n][:, r] = An[n][:, r] * (t / norms[n, r])
            A, rr = An, rn
            accepted += 1
            mu, nu = nielsen_update(mu, nu, rho)
            hist.append(en)
            if eo > 0 and abs(eo - en) / eo < tol:
                stop = "tol"
                break
        else:
            mu, nu = nielsen_update(mu, nu, rho)
            hist.append(math.sqrt(rr) / ynorm)
        if mu > mu_max:
            stop = "mu_max"
            break
    return LMResult(A=A, resid2=rr, rel_err=math.sqrt(rr) / ynorm, iters=it, accepted=accepted, mu=mu,
                    stop=stop, history=hist)


def cspd_core(A, mu: float):
    """The Hermitian positive definite core of the complex step (the complex
    counterpart of spd_core): S_n = U_n kron L_n with Gamma^(n) + mu I =
    L_G L_G^H, U_n = L_G^{-H}, C^(n) = L_n L_n^H, so S S^H = Psi_mu; core =
    I + S^H K S and f = K w - K S core^{-1} S^H K w.  Returns (core, S, K)."""
    g = cgrams(A)
    N, R = len(A), A[0].shape[1]
    R2 = R * R
    S = []
    for n in range(N):
        LG = np.linalg.cholesky(g.Gamma(n) + mu * np.eye(R))
        U = np.linalg.inv(LG).conj().T
        LC = np.linalg.cholesky(g.C[n])
        S.append(np.kron(U, LC))
    S = sla.block_diag(*S)
    P = perm_PR(R)
    K = np.zeros((N * R2, N * R2), dtype=complex)
    for n in range(N):
        for m in range(N):
            if n != m:
                K[n * R2:(n + 1) * R2, m * R2:(m + 1) * R2] = P @ np.diag(vec(g.Gamma_nm[n, m]))
    return np.eye(N * R2) + S.conj().T @ K @ S, S, K
