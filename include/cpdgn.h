/*
 * cpdgn.h -- C ABI of the GB300 library for the low-complexity damped
 * Gauss-Newton (Levenberg-Marquardt) step for rank-R CP decomposition of a
 * dense N-way tensor (Phan, Tichavsky, Cichocki, "Low Complexity Damped
 * Gauss-Newton Algorithms for CANDECOMP/PARAFAC", arXiv 1205.2584).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Tensor Y (I_1 x ... x I_N) is dense with the first index fastest
 *    (column-major vec, Sec. 2 and Appendix A).  Its element type is
 *    cp_shape.y_dtype: float64, float32, bfloat16, or a pair of bfloat16
 *    planes (CP_BF16X2, see below).
 *  - Factors are passed as ONE float64 device buffer `a` holding the paper's
 *    parameter vector a = [vec A^(1); ...; vec A^(N)] (Eq. vecV): A^(n) is
 *    I_n x R column-major at offset R * (I_1 + ... + I_{n-1}).  Buffers named
 *    `m`, `g`, `delta` use the same layout.
 *  - R x R matrices are column-major; families of them are stored back to
 *    back (C: N of them; Gamma_nm: N*N of them, (n, m) at index n*N + m).
 *  - The core system is N R^2 x N R^2, column-major; vectors w and f have
 *    length N R^2, mode-major, each R x R block column-major (Theorem 1:
 *    F_n is f[n R^2 : (n+1) R^2] reshaped R x R).
 *  - Every pointer is a device pointer unless its comment says "host".
 *    The caller owns every buffer; the library allocates no device memory
 *    on any call below; cp_state_create allocates a small host-side handle
 *    (plus, in the mixed core mode, a CUDA stream and two events).  All
 *    device work is enqueued on `stream` and is asynchronous; device
 *    outputs are valid after the stream is synchronised.
 *  - Return value: CP_OK or a CP_E* code for errors detected on the host
 *    (bad arguments, workspace too small, launch failure).  Errors found on
 *    the device (non-positive pivot, non-finite values) are written to a
 *    device status word (the `info` argument or cp_status.error); no kernel
 *    traps.
 *  - Limits: 2 <= N <= CP_MAX_N, 1 <= R <= CP_MAX_R, every I_n >= 1,
 *    prod I_n < 2^62.
 */
#ifndef CPDGN_H
#define CPDGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CP_MAX_N 8
#define CP_MAX_R 32

/* element type of the tensor.
 * CP_BF16X2: the tensor is stored as two bfloat16 planes of J elements each,
 * back to back in one buffer (hi plane first, then lo plane, both in the
 * column-major vec order); entry j has the value hi[j] + lo[j], 16 significant
 * bits.  cp_tensor_split() writes this form from a float32 tensor (hi = the
 * float32 value rounded to bfloat16, lo = the remainder rounded to bfloat16).
 * The planes are the direct operands of the tensor-core pass, so this form is
 * accepted only where that pass applies: N = 3, I_1 a multiple of 8 (the
 * buffer must be 16-byte aligned); other shapes return CP_EINVAL. */
enum cp_dtype { CP_F64 = 0, CP_F32 = 1, CP_BF16 = 2, CP_BF16X2 = 3,
                CP_C128 = 4 /* complex128 (re, im interleaved): cp_cstate_* calls only */ };

/* status codes */
enum cp_code {
  CP_OK = 0,
  CP_EINVAL = 1,      /* bad argument: null pointer, N, R or I out of range */
  CP_ENOTSPD = 2,     /* core system or Gamma^(n) + mu I not positive definite */
  CP_ENONFINITE = 3,  /* NaN or Inf met on the device: in the tensor or the
                         initial factors (cp_state_init stops the run), or in
                         a trial's step or residual (the trial is rejected) */
  CP_ETIMEOUT = 4,    /* a bounded device wait ran out (tensor-core pass);
                         the run stops with CP_STOP_ERROR */
  CP_ENOMEM = 5,      /* workspace smaller than cp_workspace_bytes() */
  CP_ECUDA = 6        /* a CUDA runtime call failed */
};

/* core-system solver of cp_dgn_solve / cp_dgn_step */
enum cp_core_mode {
  CP_CORE_F64 = 0,    /* float64 Cholesky of the core system */
  CP_CORE_MIXED = 1   /* float32 Gauss-Jordan inverse + float64 iterative refinement
                         (stops at 1e-15 ||b|| for a float64 tensor, 1e-12 ||b||
                         for a float32 / bfloat16 one, or on stagnation);
                         a trial whose refinement does not reach 1e-14 ||b|| for a
                         float64 tensor, 1e-8 ||b|| for a float32 / bfloat16 one
                         (an ill-conditioned core) is solved by the float64
                         Cholesky instead (cp_status.core_f64 = 1) */
};

/* stop reasons in cp_status.stop */
enum cp_stop { CP_RUNNING = 0, CP_STOP_TOL = 1, CP_STOP_MU = 2, CP_STOP_MAXIT = 3,
               CP_STOP_ERROR = 4 };

typedef struct cp_shape {
  int32_t N;               /* tensor order, 2..CP_MAX_N */
  int32_t R;               /* rank, 1..CP_MAX_R */
  int64_t I[CP_MAX_N];     /* I_1..I_N; entries beyond N ignored */
  int32_t y_dtype;         /* enum cp_dtype of Y; float32 and bfloat16 tensors
                              are contracted with float32 arithmetic (on the
                              tensor cores, with operands split into bfloat16
                              pieces, where the shape allows), float64 tensors
                              with float64 arithmetic */
  int32_t reserved;
} cp_shape;

typedef struct cp_opts {
  double mu0;              /* > 0: initial damping; <= 0: tau * max_n max diag Gamma^(n)
                              (Eq. mu0) */
  double tau;              /* used when mu0 <= 0 */
  double tol;              /* stop when an accepted step changes the relative error
                              epsilon by less than tol (relative) */
  double mu_max;           /* stop when mu exceeds this (Sec. 4.6: e.g. 1e30) */
  int32_t max_iter;        /* stop after this many trial steps (accepted or not) */
  int32_t normalize;       /* 1: spread each component's energy equally over the
                              modes after every accepted step (Algorithm 1 step 10) */
  int32_t core_mode;       /* enum cp_core_mode */
  int32_t refine_iters;    /* max refinement sweeps in CP_CORE_MIXED (e.g. 6) */
} cp_opts;

/* Device-resident state of one decomposition, 128 bytes. */
typedef struct cp_status {
  double mu;               /* current damping */
  double nu;               /* Nielsen's growth factor */
  double resid2;           /* ||Y - Y_hat||_F^2 at the current (accepted) factors */
  double resid2_trial;     /* the same at the last trial factors */
  double y_norm2;          /* ||Y||_F^2 */
  double rel_err;          /* epsilon = sqrt(resid2 / y_norm2) */
  double rho;              /* last gain ratio (Sec. 4.6) */
  double denom;            /* last Delta a^T (g + mu Delta a) */
  double refine_resid;     /* last relative residual of the core solve */
  double reserved_d[3];
  int32_t iters;           /* trial steps taken */
  int32_t accepted;        /* accepted steps */
  int32_t stop;            /* enum cp_stop */
  int32_t error;           /* enum cp_code of the first device-side error:
                              CP_ENONFINITE (see cp_code), CP_ETIMEOUT, CP_EINVAL
                              (all-zero tensor: epsilon undefined), CP_ENOTSPD
                              (cp_als_sweep only; a failed core factorisation
                              in a trial only sets `info` and rejects it) */
  int32_t last_accepted;   /* 1 if the last trial was accepted */
  int32_t info;            /* first non-positive pivot (1-based) of the last factorisation */
  int32_t refine_sweeps;   /* refinement residuals formed by the last CP_CORE_MIXED solve */
  int32_t core_f64;        /* 1 if the last CP_CORE_MIXED trial solved its core system
                              by the float64 Cholesky fallback (the refinement did
                              not reach its target, see CP_CORE_MIXED, or the
                              float32 inverse met a bad pivot); 0 otherwise */
} cp_status;

typedef struct cp_state cp_state;   /* opaque host handle */

/* Bytes of device workspace needed by cp_mttkrp_all / cp_fit / cp_dgn_core_build /
 * cp_dgn_solve (`what` = 0) or by a cp_state (`what` = 1) for this shape and
 * core mode.  Host-only; no device work.  Returns CP_EINVAL on a bad shape. */
int cp_workspace_bytes(const cp_shape* shape, int core_mode, int what, size_t* bytes);

/* Gramians (Theorem 1, Eq. Gamma_a; Sec. 3 Eq. ALS):
 *   C[n]        = A^(n)T A^(n)                       (N R x R matrices)
 *   Gamma_nm[n*N+m] = Hadamard_{k != n, m} C^(k)     (N*N R x R; all ones when
 *                                                     no factor remains; the
 *                                                     diagonal n = m is Gamma^(n))
 *   Gamma_all   = Hadamard_k C^(k)                   (R x R)
 * Gamma_nm and Gamma_all may be NULL to skip them.  Row blocks of every A^(n)
 * are reduced on separate CTAs and summed in a fixed order in `ws`
 * (cp_workspace_bytes(shape, 0, 0) bytes suffice), so the result is
 * deterministic and C^(n) exactly symmetric. */
int cp_gram(const cp_shape* shape, const double* a, double* C, double* Gamma_nm,
            double* Gamma_all, void* ws, size_t ws_bytes, void* stream);

/* cp_gram without a workspace argument, for callers that cannot allocate
 * device memory (for example code inside a host framework that owns the
 * whole device memory pool, or a plugin given only its inputs and outputs).
 * It computes exactly what cp_gram computes; the paper has no counterpart of
 * this call.  Its scratch (the per-row-block partial sums) is a fixed
 * 2 MiB float64 array inside the library, present on every GPU that loads the
 * library until the process exits; shapes whose partial sums exceed it
 * (more than 2^18 doubles: ceil(I_n/8) summed over n, times R(R+1)/2)
 * return CP_ENOMEM.  The call allocates nothing.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it per device ordinal, so make that first call before
 * any stream capture; after cudaDeviceReset the cached address is no longer
 * valid, so do not call this again on a device the process has reset.
 * All calls share the array: calls that overlap on the GPU race; order them
 * (one stream, or events). */
int cp_gram_noalloc(const cp_shape* shape, const double* a, double* C, double* Gamma_nm,
                    double* Gamma_all, void* stream);

/* All-mode MTTKRP in one pass over Y (Algorithm 1 step 6, Sec. 4.6 Eq. mappingJ):
 *   m = [vec M_1; ...; vec M_N],  M_n = Y_(n) (A^(N) (.) ... A^(n+1) (.) A^(n-1) (.) ... A^(1)),
 * and, if resid2 != NULL, *resid2 = ||Y - Y_hat||_F^2 summed directly from the
 * entries (Sec. 4.6, e_t), in the same pass.  Y is read once.  `ws` must hold
 * cp_workspace_bytes(shape, 0, 0) bytes.  m and resid2 are overwritten. */
int cp_mttkrp_all(const cp_shape* shape, const void* Y, const double* a, double* m,
                  double* resid2, void* ws, size_t ws_bytes, void* stream);

/* Direct residual ||Y - Y_hat||_F^2 -> *resid2 and, if y_norm2 > 0 (host value),
 * the relative error sqrt(resid2 / y_norm2) -> *rel_err (device scalars;
 * rel_err may be NULL).  Sec. 6.1 (epsilon). */
int cp_fit(const cp_shape* shape, const void* Y, const double* a, double y_norm2,
           double* resid2, double* rel_err, void* ws, size_t ws_bytes, void* stream);

/* Float32 tensor -> the CP_BF16X2 form (see enum cp_dtype): out[j] = hi, the
 * float32 value rounded to bfloat16 (nearest even), out[J + j] = lo, the
 * remainder y - hi rounded to bfloat16.  Y: J float32 values on the device;
 * out: 2 J bfloat16 (4 J bytes) on the device, 16-byte aligned, not
 * overlapping Y.  Enqueued on `stream`; the layout is the tensor's own, so
 * any shape works.  Not a step of the paper's method: it prepares the tensor
 * once for the tensor-core pass, which reads the two planes directly.
 * CP_EINVAL for null pointers, J < 1 or an unaligned out. */
int cp_tensor_split(const float* Y, int64_t J, void* out, void* stream);

/* Core system of one damped step at factors `a` with MTTKRP `m` and damping
 * *mu (device scalar), Theorems 1 and 3 in symmetric positive definite form:
 *   Gt[n]  = (Gamma^(n) + mu I)^{-1}                         (Algorithm 1 step 5)
 *   w      = [vec(A^(n)T (M_n Gt^(n) - A^(n) Gamma^(n) Gt^(n)))]_n   (Appendix D)
 *   core   = I + S^T K S,  S = blkdiag(U_n kron L_n),        (lower triangle written)
 * where K is Theorem 1's kernel (Eq. Knm_a), Gamma^(n) + mu I = L_G L_G^T,
 * U_n = L_G^{-T} and C^(n) = L_n L_n^T, so that S S^T = Psi_mu (Eq. ZiGZ_LM_a)
 * and K (I + Psi_mu K)^{-1} = K - K S core^{-1} S^T K.
 * core: N R^2 x N R^2 float64 column-major (only the lower triangle is
 * written); Gt: N R x R; w: N R^2.  info (device int, may be NULL) receives
 * n+1 if Gamma^(n) + mu I or C^(n) is not positive definite. */
int cp_dgn_core_build(const cp_shape* shape, const double* a, const double* m,
                      const double* mu, double* core, double* Gt, double* w, int* info,
                      void* ws, size_t ws_bytes, void* stream);

/* Solve the core system built by cp_dgn_core_build for f = B_mu w
 * (Theorem 1, Eq. inverse_f1a):  f = K w - K S core^{-1} S^T K w, by float64
 * Cholesky.  core (in/out): on return holds its lower Cholesky factor (the
 * upper triangle is left unspecified).  info (device int) receives 0, or the
 * 1-based index of the first non-positive pivot (N R^2 + 1 if a bounded
 * wait of the factorisation ran out; the device's timeout count then also
 * grows).  a and mu must be those given to cp_dgn_core_build.  The
 * factorisation is one persistent launch whose CTAs (at most one per SM)
 * meet at grid barriers, so it should not share the GPU with other work
 * that fills every SM. */
int cp_dgn_solve(const cp_shape* shape, const double* a, const double* mu, double* core,
                 const double* w, double* f, int* info, void* ws, size_t ws_bytes,
                 void* stream);

/* Float32 inverse of an n x n symmetric positive definite matrix by blocked
 * Gauss-Jordan elimination: the core-system inverse of the mixed solve
 * (CP_CORE_MIXED; the float64 refinement of cp_dgn_step then recovers the
 * float64 solution of Theorem 1, Eq. inverse_f1a, with it).  No pivoting
 * (each pivot block is a Schur complement of an SPD matrix).
 *   A      (in, destroyed): n x n float32, column-major, full storage;
 *          16-byte aligned; when ident > 0 its leading ident x ident block
 *          must be the identity (it is eliminated in one step; the core's
 *          diagonal R^2 x R^2 blocks are the identity).
 *   work   n x n float32, 16-byte aligned, not overlapping A.
 *   pinv   2 x 64 x 64 float32 of scratch.
 *   info   device int (may be NULL): receives 0, or the 1-based index of
 *          the first non-positive or non-finite pivot (the result is then
 *          not an inverse), or n + 1 if a bounded wait of the tensor-core
 *          kernels (n % 4 == 0, n >= 1024) ran out.
 *   in_work  host int: receives 1 if the inverse is left in work, 0 if in A
 *          (fixed by n and ident, known before the device work runs).
 * Enqueued on `stream`.  From n = 1024 (n % 4 == 0) up to n = 1536 a sweep
 * is one launch whose first CTA forms and inverts the next pivot block, and
 * the first pivot after the identity block is formed on a second stream of
 * the library; otherwise every next pivot is.  The second stream is forked
 * from and joined back to `stream` (graph-capturable).
 * CP_EINVAL for null pointers, n < 1, ident < 0 or ident > n. */
int cp_spd_invert_f32(int64_t n, int64_t ident, float* A, float* work, float* pinv, int* info,
                      int* in_work, void* stream);

/* ---- one Levenberg-Marquardt trial on the device (Algorithm 1, Sec. 4.6) ---- */

/* Create a host handle for one decomposition.  a: the caller's float64
 * factor buffer (R * sum I_n), updated in place by every accepted step;
 * ws: device workspace of cp_workspace_bytes(shape, opts->core_mode, 1) bytes,
 * which holds cp_status and every intermediate.  Both must stay valid until
 * cp_state_destroy.  *out receives the handle (host memory owned by the
 * library, freed by cp_state_destroy).  In CP_CORE_MIXED the handle also owns
 * one non-blocking CUDA stream and two events (created here, destroyed by
 * cp_state_destroy): the core inversion forks its pivot chain onto that
 * stream and joins it back, so steps stay ordered on the caller's stream. */
int cp_state_create(const cp_shape* shape, const cp_opts* opts, double* a, void* ws,
                    size_t ws_bytes, cp_state** out);
int cp_state_destroy(cp_state* st);

/* Start a decomposition of Y from the current contents of `a`: one pass over
 * Y for the MTTKRP, ||Y - Y_hat||^2 and ||Y||^2; sets mu_0 (Eq. mu0 or
 * opts->mu0), nu = 2 and the counters.  If ||Y||^2, the residual or mu_0 is
 * not finite (NaN / Inf in Y or in `a`) the status gets error = CP_ENONFINITE
 * and stop = CP_STOP_ERROR (an all-zero Y: CP_EINVAL); later steps are then
 * no-ops.  It also records the device's count of timed-out tensor-core waits,
 * so that cp_dgn_step can report one that happens later. */
int cp_state_init(cp_state* st, const void* Y, void* stream);

/* One damped Gauss-Newton trial: Gramians, damped inverses, w, core build and
 * solve, update Delta A^(n) = (G_n - A^(n) F_n) Gt^(n) (equivalent to Eq.
 * fast_low_LM1a), one pass over Y at the trial factors (MTTKRP and direct
 * residual), gain ratio, accept/reject, Nielsen's mu update, equal-energy
 * normalisation and the stop test -- all on the device, with no host
 * synchronisation, so a sequence of calls can be captured in a CUDA graph.
 * Once the device status says stop != CP_RUNNING every later call is a no-op
 * on the device.  Failure handling (Sec. 4.6 leaves it open): a trial whose
 * core system or Gamma^(n) + mu I is not positive definite (status.info =
 * the first bad pivot, 1-based), or whose step or residual is not finite
 * (status.error = CP_ENONFINITE unless an error is recorded already), is
 * rejected with rho = 0, so mu grows by nu; a bounded device wait of the
 * tensor-core pass that ran out since cp_state_init (counted per device, over
 * every call of the process) stops the run with error = CP_ETIMEOUT. */
int cp_dgn_step(cp_state* st, const void* Y, void* stream);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * CTA initialises an mbarrier that nothing ever arrives at and waits on it
 * with the same bounded wait the tensor-core pass uses, limited to limit_ns
 * nanoseconds (1e3 .. 1e10); no copy or tensor-core operation is in flight.
 * The wait runs out, the kernel returns normally and adds one to the
 * device's count of timed-out waits, which a state initialised before this
 * call reports at its next cp_dgn_step as CP_ETIMEOUT.  CP_EINVAL for a
 * limit out of range. */
int cp_selftest_wait_timeout(int64_t limit_ns, void* stream);

/* Capture `steps` consecutive cp_dgn_step calls on `stream` into a CUDA graph
 * owned by the state (replacing any earlier one).  Nothing runs during the
 * capture.  The graph reads and writes the same buffers as cp_dgn_step, so
 * replaying it is exactly `steps` calls of cp_dgn_step on Y.  Host-side
 * CUDA-graph objects are allocated here and freed by cp_state_destroy. */
int cp_state_capture(cp_state* st, const void* Y, int steps, void* stream);

/* Launch the captured graph once on `stream` (CP_EINVAL if none). */
int cp_state_launch(cp_state* st, void* stream);

/* Number of kernel nodes in the captured graph (-1 for a NULL state). */
int cp_state_graph_kernels(cp_state* st);

/* Device address of the state's cp_status (inside ws). */
cp_status* cp_state_status(cp_state* st);

/* `sweeps` (>= 1) sweeps of the ALS rule (Sec. 3, Eq. ALS), the
 * initialisation the paper runs before fLM (Sec. 4.6): for n = 1..N in turn,
 *   A^(n) <- Y_(n) (A^(N) (.) ... A^(n+1) (.) A^(n-1) (.) ... A^(1)) (Gamma^(n))^{-1},
 *   Gamma^(n) = Hadamard_{k != n} C^(k),
 * with the MTTKRP from a pass over Y at the current factors (earlier modes of
 * the sweep already replaced) and Gamma^(n) factored by Cholesky (the rule's
 * pseudo-inverse is this inverse when the other factors have full column
 * rank).  The state's factor buffer `a` is updated in place.  The damping,
 * the counters and the cached MTTKRP of the LM iteration are not maintained:
 * call cp_state_init before the next cp_dgn_step.  If Gamma^(n) is not
 * positive definite, mode n keeps its factor and the status records
 * error = CP_ENOTSPD and info = the failing pivot (1-based), unless it holds
 * an error already.  Asynchronous on `stream`, no host synchronisation
 * (graph-capturable); CP_EINVAL for a NULL state or tensor or sweeps < 1. */
int cp_als_sweep(cp_state* st, const void* Y, int sweeps, void* stream);

/* Device address of an intermediate of the last trial, for inspection:
 * 0 = the pass output at the current factors (R*T): the gradient blocks
 *     G_n = E_(n) (A^(N) (.) ... (.) A^(1) without A^(n)), E = Y - Y_hat, which
 *     equal M_n - A^(n) Gamma^(n) (Sec. 4.6: g = J^T vec(E)) but are formed from
 *     the residual tensor so that their rounding is relative to E, not to Y;
 *     for a CP_BF16X2 tensor the MTTKRP M_n itself,
 * 1 = delta (last step, R*T),
 * 2 = Gt (N R x R), 3 = w (N R^2), 4 = f (N R^2), 5 = a_trial (R*T).
 * Returns NULL for an unknown id. */
double* cp_state_buffer(cp_state* st, int id);

/* ---- HOSVD initialisation (Algorithm 1 step 1; Sec. 4.6) ---- */

/* Bytes of device workspace cp_hosvd needs for this shape (host-only). */
int cp_hosvd_workspace_bytes(const cp_shape* shape, size_t* bytes);

/* Initial factors from the mode-n singular vectors of the data tensor (the
 * initialisation Sec. 4.6 describes, followed there by a few ALS sweeps, see
 * cp_als_sweep):  A^(n) <- the R leading left singular vectors of the
 * unfolding Y_(n), i.e. the R leading eigenvectors of Y_(n) Y_(n)^T, in
 * descending order, each column's sign fixed so that its entry of largest
 * magnitude is positive.  Y: the tensor in shape->y_dtype; a: the float64
 * factor vector (Eq. vecV), overwritten; ws: cp_hosvd_workspace_bytes(shape)
 * bytes.  Y_(n) Y_(n)^T is accumulated in float64 on the device; its leading
 * eigenvectors come from `iters` steps of subspace iteration with
 * m = R + min(R, 32) (at most I_n) columns orthonormalised by Cholesky QR,
 * then a Rayleigh-Ritz step with a Jacobi eigensolver; the result converges
 * like (lambda_{m+1} / lambda_R)^iters.  Needs R <= I_n in every mode
 * (else CP_EINVAL), 1 <= iters <= 1000; asynchronous on `stream`. */
int cp_hosvd(const cp_shape* shape, const void* Y, double* a, int iters, void* ws, size_t ws_bytes,
             void* stream);

/* ---- the damped Hessian's inverse in block form (Theorem 4) and MedSAE ---- */

/* Bytes of device workspace cp_hinv_blocks needs (host-only). */
int cp_hinv_workspace_bytes(const cp_shape* shape, size_t* bytes);

/* Theorem 4's memory-saving form of (H + mu I)^{-1}, H = J^T J at the factors
 * `a` (Eq. vecV) and damping *mu (device scalar):
 *   block (n, m) = delta_nm (Gt^(n) kron I_{I_n})
 *                  - (I_R kron A^(n)) St^(n,m) (I_R kron A^(m)T)            (Eq. fastblock)
 *   Gt^(n) = (Gamma^(n) + mu I)^{-1}  -> Gt: N R x R (column-major, back to back);
 *   St = D B_mu D, D = blkdiag(Gt^(n) kron I_R), B_mu = K (I + Psi_mu K)^{-1}
 *   (Eq. inverse_f1a)                 -> St: N R^2 x N R^2 column-major, block
 *   (n, m) = St^(n,m) (rows n R^2 .., columns m R^2 ..), symmetric.
 * B_mu is formed as K - K S M^{-1} S^T K with the symmetric positive definite
 * core M = I + S^T K S factored by the float64 Cholesky (cp_dgn_solve).
 * The two outputs hold N R^2 + N^2 R^4 numbers against the (R T)^2 of the
 * inverse itself.  info (device int): 0, or a failed pivot as in
 * cp_dgn_core_build / cp_dgn_solve (the outputs are then not valid).  ws:
 * cp_hinv_workspace_bytes(shape) bytes.  Float64 throughout; O((N R^2)^3)
 * operations; N R^2 <= 6400.  Asynchronous on `stream`. */
int cp_hinv_blocks(const cp_shape* shape, const double* a, const double* mu, double* Gt, double* St,
                   int* info, void* ws, size_t ws_bytes, void* stream);

/* The diagonal of (H + mu I)^{-1} (R T values in the order of Eq. vecV) from
 * Theorem 4's blocks: entry (A^(n)[i, r]) =
 *   Gt^(n)[r, r] - sum_{s, s'} A^(n)[i, s] St^(n,n)[s + R r, s' + R r] A^(n)[i, s'].
 * Gt, St as written by cp_hinv_blocks for the same `a`. */
int cp_hinv_diag(const cp_shape* shape, const double* a, const double* Gt, const double* St, double* diag,
                 void* stream);

/* Squared angular errors between true and estimated components (Sec. 6,
 * Eq. MedSAE), after matching the components' order: the permutation pi
 * maximises sum_r sum_n |cos(a_r^(n), ahat_pi(r)^(n))| (solved exactly by the
 * Hungarian method), and alpha2[n R + r] = arccos(|cos(a_r^(n), ahat_pi(r)^(n))|)^2
 * (the absolute value: a component's sign is fixed only up to flips that
 * cancel across modes); perm[r] = pi(r).  a_true, a_est: factor vectors of
 * the same shape (Eq. vecV); alpha2: N R doubles; perm: R ints (device).
 * MedSAE in dB is 10 log10 of the median of alpha2 over the runs compared. */
int cp_sae(const cp_shape* shape, const double* a_true, const double* a_est, double* alpha2, int* perm,
           void* stream);

/* ---- complex-valued tensors (Sec. 5, Theorems 5-8) ---- */

/* The damped Gauss-Newton iteration for a complex tensor (shape->y_dtype =
 * CP_C128: complex128, real and imaginary parts interleaved, first index
 * fastest) with complex factors (the factor vector a of Eq. vecV in complex128
 * entries, 2 R T doubles).  Each trial: C^(n) = A^(n)H A^(n),
 * Gamma^(n,m) = Hadamard_{k != n,m} C^(k) (Theorem 5); the gradient blocks
 * G_n = E_(n) conj(KR_n) = Y_(n) conj(KR_n) - A^(n) Gamma^(n)T (Theorem 7) from
 * one pass over the tensor; the fast step of Theorem 8 in Hermitian positive
 * definite core form (core = I + S^H K S, S_n = U_n kron L_n,
 * Gamma^(n) + mu I = L_G L_G^H, U_n = L_G^{-H}, C^(n) = L_n L_n^H), the core
 * solved in float64 through its real symmetric representation
 * [[Re, -Im], [Im, Re]] by the float64 Cholesky; the update
 * Delta_n = (G_n - A^(n) F_n) Gt^(n)T, Gt^(n) = (Gamma^(n) + mu I)^{-1} (the
 * matrix form of Theorem 8's damped inverse acts through its transpose);
 * the Sec. 4.6 control with gain-ratio denominator Re(Delta^H (g + mu Delta))
 * and normalisation by real positive scales.  Limits: R <= 16, I_1 <= 256,
 * N R^2 <= 3200 (CP_EINVAL otherwise).  Same conventions as the real state:
 * caller-owned factor buffer and workspace, all work on `stream`, no host
 * synchronisation, later steps no-ops once stopped (cp_status.core_f64 = 1). */
typedef struct cp_cstate cp_cstate;
int cp_cstate_workspace_bytes(const cp_shape* shape, size_t* bytes);
int cp_cstate_create(const cp_shape* shape, const cp_opts* opts, double* a, void* ws, size_t ws_bytes,
                     cp_cstate** out);
int cp_cstate_destroy(cp_cstate* st);
int cp_cstate_init(cp_cstate* st, const void* Y, void* stream);
int cp_cdgn_step(cp_cstate* st, const void* Y, void* stream);
cp_status* cp_cstate_status(cp_cstate* st);
/* 0 = gradient blocks at the current factors, 1 = last step, 5 = trial factors
 * (complex128, R T entries each); NULL for another id. */
double* cp_cstate_buffer(cp_cstate* st, int id);

/* ---- batched form: many small decompositions in one persistent launch ---- */

/* One problem of a batch.  Limits: 2 <= N <= 4, 1 <= R <= 16, I_1 <= 256,
 * sum_{n>=2} I_n R <= 12288, N R^2 <= 1024. */
typedef struct cp_batch_problem {
  int32_t N;
  int32_t R;
  int64_t I[4];
  int64_t y_off;     /* element offset of its float32 tensor (first index fastest)
                        in the packed tensor buffer */
  int64_t a_off;     /* float64 offset of its parameter vector a in the packed
                        factor buffer (same layout as the single-problem calls) */
  int64_t ws_off;    /* byte offset of its workspace; set by cp_batch_layout */
  double mu0;        /* > 0: initial damping; otherwise opts->tau * max diag Gamma^(n) */
} cp_batch_problem;

/* CP_OK if the problem fits the batched kernel's limits (host-only). */
int cp_batch_check(const cp_batch_problem* p);

/* Host-only: assign every problem's ws_off and return the total workspace
 * bytes (*ws_bytes) for cp_batch_run.  CP_EINVAL if a problem is out of range. */
int cp_batch_layout(cp_batch_problem* probs, int count, size_t* ws_bytes);

/* Run the batch: one persistent launch of `ctas` CTAs (<= 0: one per SM) that
 * take problems from a device work queue; each CTA runs a taken problem's
 * Levenberg-Marquardt trials (Algorithm 1 with the Sec. 4.6 control, the same
 * algebra as cp_dgn_step) until its stop rule fires or `trials` trials have
 * run in this launch, then takes the next problem.  probs_dev: device copy of
 * the laid-out problems; Y: packed float32 tensors; a: packed float64 factors,
 * updated in place; status: `count` cp_status, zero-filled by the caller
 * before the first launch and carried across launches; ws: workspace of
 * cp_batch_layout's size.  A later launch continues every problem that has not
 * stopped.  The first 256 bytes of ws are the queue counter (reset here).
 * tile: fibres per tile of the in-CTA pass over a tensor (8, 16 or 32; 0 =
 * 16), a tuning knob that does not change results beyond rounding.  order
 * (device, may be NULL): a permutation of 0..count-1 giving the queue order
 * (e.g. most expensive first); results are always indexed by problem. */
int cp_batch_run(const cp_batch_problem* probs_dev, int count, const float* Y, double* a, void* ws,
                 cp_status* status, const cp_opts* opts, int trials, int ctas, int tile,
                 const int* order, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CPDGN_H */
