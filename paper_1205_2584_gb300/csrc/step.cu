// One damped Gauss-Newton / Levenberg-Marquardt trial on the device
// (Algorithm 1 with the damping control of Sec. 4.6), and the stand-alone
// core-system calls of the C ABI.
//
// Kernel sequence of cp_dgn_step (no host synchronisation; graph-capturable):
//   k_step_begin      clear per-trial flags, zero the trial MTTKRP
//   k_gram_cp/_had    C^(n), P^(n) = A^(n)T M_n, Gamma^(n,m), Gamma
//   k_mode_prep       Gt^(n), U_n, L_n, w                 (Algorithm 1 steps 5-7)
//   k_core_w/_fill    core = I + S^T K S                   (step 8-9, SPD form)
//   chol_factor       core = L L^T (float64 form), or
//   gj_invert         core^{-1} in float32 (mixed form; Gauss-Jordan, the
//                     pivot chain on a second stream; meanwhile a third
//                     stream forms b = S^T K w)
//   solve             f = K w - K S core^{-1} S^T K w      (step 9): triangular
//                     solves, or float64 refinement sweeps with the inverse
//   k_update          Delta A^(n) = (G_n - A^(n) F_n) Gt^(n), trial factors,
//                     Delta^T (g + mu Delta) and column norms (steps 10-11)
//   mttkrp            M_n and ||E||^2 at the trial factors (one pass over Y)
//   k_control         gain ratio, accept iff the error decreased, Nielsen's
//                     mu update, equal-energy scales, stop test (Sec. 4.6)
//   k_commit          on acceptance: A <- scaled trial factors, M <- rescaled
//                     trial MTTKRP (normalisation does not need a new pass:
//                     column r of M_n scales by 1/s_r^(n) when prod_n s_r^(n) = 1)
#include <new>

#include "common.cuh"

namespace cpdgn {

int launch_mttkrp(const Dims& d, const void* Y, const double* a, double* m, double* resid2,
                  const int* skip, cudaStream_t s, int grad);
int launch_gram(const Dims& d, const double* a, const double* m, double* part, double* C, double* P,
                double* Gnm, double* Gall, const int* skip, cudaStream_t s);
int launch_mode_prep(const Dims& d, const double* C, const double* P, const double* mu, double* Gnm,
                     double* Gt, double* U, double* LC, double* w, int* info, const int* skip,
                     cudaStream_t s);
int launch_core_w(const Dims& d, const double* Gnm, const double* LC, const double* U, double* Wp,
                  const int* skip, cudaStream_t s);
template <typename T>
int launch_core_fill(const Dims& d, const double* LC, const double* U, const double* Wp, T* core, int full,
                     const int* skip, cudaStream_t s);
int launch_apply_K(const Dims& d, const double* Gnm, const double* x, const double* base, double* out,
                   const int* skip, cudaStream_t s);
int launch_apply_S(const Dims& d, const double* LC, const double* U, const double* x, double* out,
                   const int* skip, cudaStream_t s);
int launch_apply_ST(const Dims& d, const double* LC, const double* U, const double* Gnm, const double* x,
                    int kx, const double* b, const double* y, double* out, double* kw, double* norm2,
                    const int* skip, cudaStream_t s);
int chol64_factor(double* A, int64_t n, double* dinv, int* info, void* sync, int* tmo, const int* skip,
                  cudaStream_t s);
int chol64_solve(const double* L, const double* dinv, int64_t n, const double* b, double* z, double* y,
                 void* sync, int* info, int* tmo, const int* skip, cudaStream_t s);
template <typename T>
int gj_invert(T* A, T* B, T* pinv, int64_t n, int64_t ident, int* info, const int* skip, cudaStream_t s,
              cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join, T** result, int tc_mode = -1);
int tc_timeout_counter(int** out);
int launch_gemv_acc(const float* X, int64_t n, const double* r, double* y, const double* b2, const double* r2,
                    const double* r2prev, int* done, double tol2, const int* skip, cudaStream_t s);

// scalar slots (doubles) inside S_SCAL
enum { SC_R2T = 0, SC_YN2 = 1, SC_R2 = 2, SC_REFN = 3, SC_NRM = 8 };   // SC_NRM..: ||b||^2, ||res_k||^2
constexpr int kMaxRefine = 48;
// int slots inside S_INFO
// IN_INFO: first failed pivot of the trial (per-mode factors or the float64
// core factor: the trial is rejected); IN_INFO32: first failed pivot of the
// float32 core inverse (the mixed solve then falls back to float64);
// IN_SKIP64: 1 unless the mixed solve needs its float64 fallback
enum { IN_INFO = 0, IN_COMMIT = 1, IN_ZERO = 2, IN_RDONE = 3, IN_TOBASE = 4, IN_SKIP64 = 5, IN_INFO32 = 6 };

struct Bufs {
  double *C, *Gnm, *Gall, *P, *LC, *U, *Gt, *w, *Kw, *b, *y, *Z, *res, *dcor, *f, *Wp;
  float *core32, *core32b, *pinv;
  double *gpart, *part, *scal;
  int* info;
  cp_status* status;
  double *m, *mt, *at, *delta, *scale, *mu;
  double* core64;
  double* dinv;
  void* sync;
};

static Bufs carve(const Layout& L, void* ws, int64_t ncore) {
  char* base = static_cast<char*>(ws);
  Bufs b;
  b.C = reinterpret_cast<double*>(base + L.off[S_C]);
  b.Gnm = reinterpret_cast<double*>(base + L.off[S_GNM]);
  b.Gall = reinterpret_cast<double*>(base + L.off[S_GALL]);
  b.P = reinterpret_cast<double*>(base + L.off[S_P]);
  b.LC = reinterpret_cast<double*>(base + L.off[S_LC]);
  b.U = reinterpret_cast<double*>(base + L.off[S_U]);
  b.Gt = reinterpret_cast<double*>(base + L.off[S_GT]);
  b.w = reinterpret_cast<double*>(base + L.off[S_W]);
  b.Kw = reinterpret_cast<double*>(base + L.off[S_KW]);
  b.b = reinterpret_cast<double*>(base + L.off[S_B]);
  b.y = reinterpret_cast<double*>(base + L.off[S_Y]);
  b.Z = reinterpret_cast<double*>(base + L.off[S_Z]);
  b.res = reinterpret_cast<double*>(base + L.off[S_RES]);
  b.dcor = reinterpret_cast<double*>(base + L.off[S_D]);
  b.f = reinterpret_cast<double*>(base + L.off[S_F]);
  b.Wp = reinterpret_cast<double*>(base + L.off[S_WP]);
  b.core32 = reinterpret_cast<float*>(base + L.off[S_CORE32]);
  b.core32b = b.core32 + size_t(0);   // set by carve_core2()
  b.gpart = reinterpret_cast<double*>(base + L.off[S_GPART]);
  b.pinv = reinterpret_cast<float*>(base + L.off[S_PINV]);
  b.part = reinterpret_cast<double*>(base + L.off[S_PART]);
  b.scal = reinterpret_cast<double*>(base + L.off[S_SCAL]);
  b.info = reinterpret_cast<int*>(base + L.off[S_INFO]);
  b.status = reinterpret_cast<cp_status*>(base + L.off[S_STATUS]);
  b.m = reinterpret_cast<double*>(base + L.off[S_M]);
  b.mt = reinterpret_cast<double*>(base + L.off[S_MT]);
  b.at = reinterpret_cast<double*>(base + L.off[S_AT]);
  b.delta = reinterpret_cast<double*>(base + L.off[S_DELTA]);
  b.scale = reinterpret_cast<double*>(base + L.off[S_SCALE]);
  b.mu = reinterpret_cast<double*>(base + L.off[S_MU]);
  b.core64 = reinterpret_cast<double*>(base + L.off[S_CORE64]);
  b.core32b = b.core32 + size_t(ncore) * size_t(ncore);
  b.dinv = reinterpret_cast<double*>(base + L.off[S_DINV]);
  b.sync = base + L.off[S_SYNC];
  return b;
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

__global__ void k_step_begin(int64_t nm, double* mt, double* scal, int* info, const cp_status* st) {
  pdl_enter();
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i == 0) {
    info[IN_INFO] = 0;
    info[IN_INFO32] = 0;
    info[IN_SKIP64] = 1;
    info[IN_COMMIT] = 0;
    info[IN_RDONE] = (st->stop != CP_RUNNING) ? 1 : 0;
    scal[SC_R2T] = 0.0;
  }
  if (i < kMaxRefine + 2) scal[SC_NRM + i] = 0.0;
  for (; i < nm; i += int64_t(gridDim.x) * blockDim.x) mt[i] = 0.0;
}

// Delta A and trial factors; CTA = (mode n, block of kUpdRows rows); thread = (row, r).
__global__ void __launch_bounds__(kUpdRows * 32) k_update(Dims d, const double* a, const double* m,
                                                          const double* Gnm, const double* Gt,
                                                          const double* f, const double* mu,
                                                          double* delta, double* at, double* part,
                                                          const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double Gam[CP_MAX_R * CP_MAX_R], Fn[CP_MAX_R * CP_MAX_R], Gtn[CP_MAX_R * CP_MAX_R];
  __shared__ double Arow[kUpdRows][CP_MAX_R], H[kUpdRows][CP_MAX_R], Q[kUpdRows][CP_MAX_R];
  __shared__ double red[kUpdRows * 32];
  const int R = d.R, RR = d.RR, N = d.N;
  int b = blockIdx.x, n = 0;
  for (; n < N; ++n) {
    const int nb = int((d.I[n] + kUpdRows - 1) / kUpdRows);
    if (b < nb) break;
    b -= nb;
  }
  const int64_t In = d.I[n];
  const int64_t i0 = int64_t(b) * kUpdRows;
  const int tid = threadIdx.x;
  const int row = tid / 32, r = tid % 32;
  const int64_t i = i0 + row;
  const bool act = (r < R) && (i < In);
  for (int e = tid; e < RR; e += blockDim.x) {
    Gam[e] = Gnm[(int64_t(n) * N + n) * RR + e];
    Fn[e] = f[int64_t(n) * RR + e];
    Gtn[e] = Gt[int64_t(n) * RR + e];
  }
  const double* An = a + d.aoff[n];
  const double* Mn = m + d.aoff[n];
  Arow[row][r] = act ? An[i + In * r] : 0.0;
  __syncthreads();
  double g = 0.0;
  if (act) {
    double s1 = 0.0, s2 = 0.0;
    for (int s = 0; s < R; ++s) {
      s1 = fma(Arow[row][s], Gam[s + R * r], s1);
      s2 = fma(Arow[row][s], Fn[s + R * r], s2);
    }
    // gradient block G_n = M_n - A^(n) Gamma^(n), or G_n itself from the pass
    g = d.mg ? Mn[i + In * r] : Mn[i + In * r] - s1;
    H[row][r] = g - s2;               // G_n - A^(n) F_n
  }
  __syncthreads();
  double dl = 0.0, contrib = 0.0, at2 = 0.0;
  if (act) {
    double s = 0.0;
    for (int c = 0; c < R; ++c) s = fma(H[row][c], Gtn[c + R * r], s);
    dl = s;
    const double muv = *mu;
    contrib = dl * (g + muv * dl);
    const double av = Arow[row][r] + dl;
    at2 = av * av;
    delta[d.aoff[n] + i + In * r] = dl;
    at[d.aoff[n] + i + In * r] = av;
  }
  Q[row][r] = at2;
  const double den = block_sum<kUpdRows * 32>(contrib, red);
  double* pc = part + int64_t(blockIdx.x) * (1 + R);
  if (tid == 0) pc[0] = den;
  if (tid < R) {
    double s = 0.0;
    for (int q = 0; q < kUpdRows; ++q) s += Q[q][tid];
    pc[1 + tid] = s;
  }
}

__global__ void k_control(Dims d, cp_opts o, double* part, int64_t nparts, cp_status* st,
                          double* scal, int* info, double* scale, const int* tmo) {
  pdl_enter();
  // One CTA of 256 threads.  The float64 square roots, divides and roots
  // below are long dependent operations on this part (hundreds of cycles
  // each), so independent ones run on different threads: the two relative
  // errors and the refinement residual on three threads, the column norms
  // on one thread per (mode, column), the accept / damping decision on a
  // thread of the last warp, while the equal-energy targets are formed for
  // every column and applied only if the step is accepted.
  constexpr int kT = 256;
  __shared__ double sh[kT];
  __shared__ double qs[kT];
  __shared__ double nrm[CP_MAX_N * CP_MAX_R], rnm[CP_MAX_N * CP_MAX_R], tgt[CP_MAX_R];
  __shared__ double e_s[2], rr_s;
  __shared__ int sweeps_s, s_acc;
  if (st->stop != CP_RUNNING) return;
  const int tid = threadIdx.x;
  const int R = d.R, N = d.N, NR = d.N * d.R;
  double v = 0.0;
  for (int64_t c = tid; c < nparts; c += kT) v += part[c * (1 + R)];
  const double den = block_sum<kT>(v, sh);
  // squared column norms of the trial factors, tp threads per (mode, column),
  // each summing every tp-th block of its mode
  int tp = 1;
  while (tp * 2 * NR <= kT) tp *= 2;
  if (tid < NR * tp) {
    const int pr = tid / tp, sub = tid % tp, n = pr / R, r = pr % R;
    int64_t c0 = 0;
    for (int k = 0; k < n; ++k) c0 += (d.I[k] + kUpdRows - 1) / kUpdRows;
    const int64_t c1 = c0 + (d.I[n] + kUpdRows - 1) / kUpdRows;
    double sq = 0.0;
    for (int64_t c = c0 + sub; c < c1; c += tp) sq += part[c * (1 + R) + 1 + r];
    qs[tid] = sq;
  }
  const int tdec = kT - 1;   // decision thread, last warp
  if (tid == kT - 32) e_s[0] = sqrt(st->resid2 / st->y_norm2);
  if (tid == kT - 64) e_s[1] = sqrt(scal[SC_R2T] / st->y_norm2);
  if (tid == kT - 96) {
    double rr = 0.0;   // relative residual of the last refinement sweep that ran
    int sweeps = 0;
    for (int k = kMaxRefine; k >= 1; --k)
      if (scal[SC_NRM + k] > 0.0) {
        rr = sqrt(scal[SC_NRM + k] / scal[SC_NRM]);
        sweeps = k;
        break;
      }
    rr_s = rr;
    sweeps_s = sweeps;
  }
  __syncthreads();
  if (tid < NR) {
    double sq = 0.0;
    for (int q = 0; q < tp; ++q) sq += qs[tid * tp + q];
    nrm[tid] = sqrt(sq);
    rnm[tid] = rsqrt(sq);
  }
  if (tid == tdec) {
    const double r2 = st->resid2;
    const double r2t = scal[SC_R2T];
    const int bad = info[IN_INFO];
    const bool finite = isfinite(r2t) && isfinite(den);
    const bool accept = (bad == 0) && finite && (r2t < r2);
    // a trial whose core factorisation failed, or whose step or residual is
    // not finite, is rejected and counts as rho = 0, so mu always grows then
    const double rho = (bad == 0 && finite && den > 0.0) ? (r2 - r2t) / den : 0.0;
    // (a failed factorisation leaves undefined values behind it; only a trial
    // whose factorisations succeeded reports non-finite numbers as an error)
    if (bad == 0 && !finite && st->error == 0) st->error = CP_ENONFINITE;
    // a bounded device wait of the tensor-core pass ran out since cp_state_init
    // (its outputs were poisoned, so this trial is rejected): stop with an error
    const bool timed_out = tmo && (*reinterpret_cast<const volatile int*>(tmo) != info[IN_TOBASE]);
    double mu = st->mu, nu = st->nu;
    if (rho > 0.0) {
      const double t = 2.0 * rho - 1.0;
      const double fac = 1.0 - t * t * t;
      mu *= (fac > 1.0 / 3.0) ? fac : 1.0 / 3.0;
      nu = 2.0;
    } else {
      mu *= nu;
      nu *= 2.0;
    }
    st->iters += 1;
    st->rho = rho;
    st->denom = den;
    st->resid2_trial = r2t;
    st->info = bad;
    st->refine_resid = rr_s;
    st->refine_sweeps = sweeps_s;
    st->core_f64 = info[IN_SKIP64] ? 0 : 1;
    st->mu = mu;
    st->nu = nu;
    st->last_accepted = accept ? 1 : 0;
    if (accept) {
      const double e_old = e_s[0], e_new = e_s[1];
      st->accepted += 1;
      st->resid2 = r2t;
      st->rel_err = e_new;
      if (e_old > 0.0 && fabs(e_old - e_new) < o.tol * e_old) st->stop = CP_STOP_TOL;
    }
    if (timed_out) {
      st->error = CP_ETIMEOUT;
      st->stop = CP_STOP_ERROR;
    }
    if (st->stop == CP_RUNNING && mu > o.mu_max) st->stop = CP_STOP_MU;
    if (st->stop == CP_RUNNING && st->iters >= o.max_iter) st->stop = CP_STOP_MAXIT;
    info[IN_COMMIT] = accept ? 1 : 0;
    s_acc = accept ? 1 : 0;
  }
  __syncthreads();
  // equal-energy scales: s_r^(n) = lambda_r^(1/N) / ||a_r^(n)||, lambda_r = prod_n ||a_r^(n)||
  if (tid < R) {
    double lam = 1.0;
    bool pos = true;
    for (int n = 0; n < N; ++n) {
      const double nr = nrm[n * R + tid];
      if (!(nr > 0.0)) pos = false;
      lam *= nr;
    }
    tgt[tid] = !pos ? 0.0 : (N == 2 ? sqrt(lam) : (N == 3 ? cbrt(lam) : pow(lam, 1.0 / N)));
  }
  __syncthreads();
  if (tid < NR) {
    const int r = tid % R;
    const bool ok = (o.normalize != 0) && s_acc && tgt[r] > 0.0;
    scale[tid] = ok ? tgt[r] * rnm[tid] : 1.0;
  }
}

__global__ void k_commit(Dims d, const int* commit, const double* at, const double* mt,
                         const double* scale, double* a, double* m) {
  pdl_enter();
  if (!*commit) return;
  const int64_t tot = d.T * d.R;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < tot;
       idx += int64_t(gridDim.x) * blockDim.x) {
    int n = 0;
    while (n + 1 < d.N && idx >= d.aoff[n + 1]) ++n;
    const int r = int((idx - d.aoff[n]) / d.I[n]);
    const double s = scale[n * d.R + r];
    a[idx] = at[idx] * s;
    m[idx] = mt[idx] / s;
  }
}

__global__ void k_sumsq(const void* Y, int dtype, int64_t J, double* out) {
  pdl_enter();
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < J; i += int64_t(gridDim.x) * 256) {
    double v;
    if (dtype == CP_F64) v = static_cast<const double*>(Y)[i];
    else if (dtype == CP_F32) v = static_cast<const float*>(Y)[i];
    else if (dtype == CP_BF16X2)
      v = double(__bfloat162float(static_cast<const __nv_bfloat16*>(Y)[i])) +
          double(__bfloat162float(static_cast<const __nv_bfloat16*>(Y)[J + i]));
    else v = __bfloat162float(static_cast<const __nv_bfloat16*>(Y)[i]);
    s = fma(v, v, s);
  }
  const double t = block_sum<256>(s, sh);
  if (threadIdx.x == 0) atomicAdd(out, t);
}

__global__ void k_init_status(Dims d, cp_opts o, const double* Gnm, const double* scal, cp_status* st,
                              double* mu_copy, const int* tmo, int* info) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = 0.0;
  for (int n = 0; n < d.N; ++n)
    for (int r = 0; r < d.R; ++r) {
      const double v = Gnm[(int64_t(n) * d.N + n) * d.RR + r + d.R * r];
      mx = v > mx ? v : mx;
    }
  cp_status s;
  s.mu = (o.mu0 > 0.0) ? o.mu0 : o.tau * mx;
  s.nu = 2.0;
  s.resid2 = scal[SC_R2];
  s.resid2_trial = scal[SC_R2];
  s.y_norm2 = scal[SC_YN2];
  s.rel_err = sqrt(scal[SC_R2] / scal[SC_YN2]);
  s.rho = 0.0;
  s.denom = 0.0;
  s.refine_resid = 0.0;
  s.reserved_d[0] = s.reserved_d[1] = s.reserved_d[2] = 0.0;
  s.iters = 0;
  s.accepted = 0;
  s.stop = CP_RUNNING;
  s.error = 0;
  s.last_accepted = 0;
  s.info = 0;
  s.refine_sweeps = 0;
  s.core_f64 = 0;
  // a tensor or factors with NaN / Inf entries give a non-finite ||Y||^2 or
  // residual: nothing can be decided from them, so the run stops at once
  if (!isfinite(s.y_norm2) || !isfinite(s.resid2) || !isfinite(s.mu) || !(s.y_norm2 > 0.0)) {
    s.error = isfinite(s.y_norm2) && isfinite(s.resid2) && isfinite(s.mu) ? CP_EINVAL : CP_ENONFINITE;
    s.stop = CP_STOP_ERROR;
  }
  *st = s;
  *mu_copy = s.mu;
  // the timeout counter of the tensor-core pass as it stands now; k_control
  // reports CP_ETIMEOUT once it moves
  info[IN_TOBASE] = tmo ? *reinterpret_cast<const volatile int*>(tmo) : 0;
}

// ---------------------------------------------------------------------------
// shared pieces of the core solve
// ---------------------------------------------------------------------------

// f = K w - K S y with y = core^{-1} b, b = S^T K w.
// CP_CORE_F64: L64 holds the float64 Cholesky factor, two triangular solves.
// CP_CORE_MIXED: X32 holds the float32 inverse of the core; y = X b, then up
// to refine_iters sweeps y += X (b - y - S^T K S y) with the float64
// operator, stopping once ||b - core y|| <= 1e-15 ||b|| (1e-12 ||b|| for
// float32 and bfloat16 tensors) or the residual stops shrinking (kernels of later sweeps return at once; the graph is fixed).
// b = S^T (K w), ||b||^2 (nrm[0]) and K w, the right-hand side of the core
// system; it needs the per-mode preparation only, not the core.
static int core_rhs(const Dims& d, const Bufs& B, const int* skip, cudaStream_t s) {
  return launch_apply_ST(d, B.LC, B.U, B.Gnm, B.w, 1, nullptr, nullptr, B.b, B.Kw, B.scal + SC_NRM, skip, s);
}

// Decide whether the mixed solve must fall back to float64: skip64 = 1 when
// the run has stopped or a refinement residual met ||r|| <= tol ||b|| (and
// the float32 inverse had no bad pivot); else 0, and the float64 Cholesky
// path below runs for this trial.
__global__ void k_refine_verdict(const double* nrm, int K, double tol2, const int* stop, const int* info32,
                                 int* skip64) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int out = 1;
  if (*stop == CP_RUNNING) {
    bool conv = !(nrm[0] > 0.0);                  // b = 0: y = 0 is exact
    for (int k = 1; k <= K && !conv; ++k) {
      const double v = nrm[k];
      if (v > 0.0 && v <= tol2 * nrm[0]) conv = true;
    }
    if (*info32 != 0) conv = false;
    out = conv ? 1 : 0;
  }
  *skip64 = out;
}

// y = core^{-1} b by the float64 Cholesky factor of `core` (lower triangle
// filled here from the per-mode factors), skipped while *skip is set.
static int solve_core_f64(const Dims& d, const Bufs& B, double* core, int* tmo, const int* skip, cudaStream_t s,
                          bool fill) {
  if (fill) CP_TRY(launch_core_fill<double>(d, B.LC, B.U, B.Wp, core, 0, skip, s));
  CP_TRY(chol64_factor(core, d.ncore, B.dinv, B.info + IN_INFO, B.sync, tmo, skip, s));
  CP_TRY(chol64_solve(core, B.dinv, d.ncore, B.b, B.dcor, B.y, B.sync, B.info + IN_INFO, tmo, skip, s));
  return CP_OK;
}

// core64: the float64 core (CP_CORE_F64: filled and factored by the caller's
// sequence here; CP_CORE_MIXED: storage for the fallback, may alias the
// float32 buffers, which are dead by then).
static int solve_core(const Dims& d, const Bufs& B, double* core64, const float* X32, int mode,
                      int refine_iters, int* tmo, const int* skip, cudaStream_t s, bool rhs_ready = false) {
  const int64_t n = d.ncore;
  double* nrm = B.scal + SC_NRM;
  if (!rhs_ready) CP_TRY(core_rhs(d, B, skip, s));
  if (mode == CP_CORE_F64) {
    CP_TRY(chol64_solve(core64, B.dinv, n, B.b, B.dcor, B.y, B.sync, B.info + IN_INFO, tmo, skip, s));
  } else {
    int* rdone = B.info + IN_RDONE;
    const int K = refine_iters < kMaxRefine ? refine_iters : kMaxRefine;
    // refinement target: 1e-15 ||b|| for a float64 tensor; 1e-12 ||b|| for
    // float32 and bfloat16 tensors, whose gradient blocks carry float32
    // rounding (relative 1e-7 and more), so that a tighter solve changes the
    // step by less than its own rounding error while costing 1-2 more sweeps
    const double rtol2 = (d.y_dtype == CP_F64) ? 1e-30 : 1e-24;
    CP_CUDA(cudaMemsetAsync(B.y, 0, n * sizeof(double), s));
    CP_TRY(launch_gemv_acc(X32, n, B.b, B.y, nullptr, nullptr, nullptr, nullptr, 0.0, skip, s));
    for (int it = 1; it <= K; ++it) {
      CP_TRY(launch_apply_S(d, B.LC, B.U, B.y, B.Z, rdone, s));
      CP_TRY(launch_apply_ST(d, B.LC, B.U, B.Gnm, B.Z, 1, B.b, B.y, B.res, nullptr, nrm + it, rdone, s));
      CP_TRY(launch_gemv_acc(X32, n, B.res, B.y, nrm, nrm + it, it > 1 ? nrm + it - 1 : nullptr, rdone, rtol2,
                             rdone, s));
    }
    if (core64) {
      // the refinement missed its target (an ill-conditioned core: collinear
      // factors at small mu) or the float32 inverse failed: float64 Cholesky.
      // Target: 1e-14 ||b|| for a float64 tensor; 1e-8 ||b|| for float32 and
      // bfloat16 tensors, whose gradient blocks carry float32-level rounding
      // already (a tighter core solve would not make the step more accurate)
      const double tol2 = (d.y_dtype == CP_F64) ? 1e-28 : 1e-16;
      CP_CUDA(launch_pdl(k_refine_verdict, 1, 32, 0, s, nrm, K, tol2, skip, B.info + IN_INFO32, B.info + IN_SKIP64));
      CP_TRY(solve_core_f64(d, B, core64, tmo, B.info + IN_SKIP64, s, true));
    }
  }
  CP_TRY(launch_apply_S(d, B.LC, B.U, B.y, B.Z, skip, s));                        // Z = S y
  CP_TRY(launch_apply_K(d, B.Gnm, B.Z, B.Kw, B.f, skip, s));                      // f = Kw - K Z
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn

using namespace cpdgn;

struct cp_state {
  Dims d;
  cp_opts o;
  double* a;
  void* ws;
  Layout L;
  Bufs B;
  cudaStream_t side = nullptr;           // second stream for the pivot chain of the core inversion
  cudaStream_t rhs = nullptr;            // third stream: the core system's right-hand side
  cudaEvent_t ev_rhs_fork = nullptr, ev_rhs_join = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int* tmo = nullptr;                    // device counter of timed-out waits of the tensor-core pass
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_steps = 0;
  int graph_kernels = 0;
};

static void drop_graph(cp_state* st) {
  if (st->exec) cudaGraphExecDestroy(st->exec);
  if (st->graph) cudaGraphDestroy(st->graph);
  st->exec = nullptr;
  st->graph = nullptr;
  st->graph_steps = 0;
  st->graph_kernels = 0;
}

extern "C" int cp_workspace_bytes(const cp_shape* shape, int core_mode, int what, size_t* bytes) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!bytes || (core_mode != CP_CORE_F64 && core_mode != CP_CORE_MIXED)) return CP_EINVAL;
  Layout L;
  make_layout(d, core_mode, what ? 1 : 0, &L);
  *bytes = L.total;
  return CP_OK;
}

extern "C" int cp_dgn_core_build(const cp_shape* shape, const double* a, const double* m,
                                 const double* mu, double* core, double* Gt, double* w, int* info,
                                 void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !m || !mu || !core || !Gt || !w || !ws) return CP_EINVAL;
  Layout L;
  make_layout(d, CP_CORE_F64, 0, &L);
  if (ws_bytes < L.total) return CP_ENOMEM;
  Bufs B = carve(L, ws, d.ncore);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (info) CP_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
  CP_TRY(launch_gram(d, a, m, B.gpart, B.C, B.P, nullptr, nullptr, nullptr, s));
  CP_TRY(launch_mode_prep(d, B.C, B.P, mu, B.Gnm, Gt, B.U, B.LC, w, info, nullptr, s));
  CP_TRY(launch_core_w(d, B.Gnm, B.LC, B.U, B.Wp, nullptr, s));
  CP_TRY(launch_core_fill<double>(d, B.LC, B.U, B.Wp, core, 0, nullptr, s));
  return CP_OK;
}

extern "C" int cp_dgn_solve(const cp_shape* shape, const double* a, const double* mu, double* core,
                            const double* w, double* f, int* info, void* ws, size_t ws_bytes,
                            void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !mu || !core || !w || !f || !info || !ws) return CP_EINVAL;
  Layout L;
  make_layout(d, CP_CORE_F64, 0, &L);
  if (ws_bytes < L.total) return CP_ENOMEM;
  Bufs B = carve(L, ws, d.ncore);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CP_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
  // S and K need the Gramians and the damped factors at (a, mu)
  CP_TRY(launch_gram(d, a, nullptr, B.gpart, B.C, nullptr, nullptr, nullptr, nullptr, s));
  CP_TRY(launch_mode_prep(d, B.C, nullptr, mu, B.Gnm, B.Gt, B.U, B.LC, nullptr, nullptr, nullptr, s));
  int* tmo = nullptr;
  CP_TRY(tc_timeout_counter(&tmo));
  CP_TRY(chol64_factor(core, d.ncore, B.dinv, info, B.sync, tmo, nullptr, s));
  CP_CUDA(cudaMemcpyAsync(B.w, w, d.ncore * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CP_TRY(core_rhs(d, B, nullptr, s));
  CP_TRY(chol64_solve(core, B.dinv, d.ncore, B.b, B.dcor, B.y, B.sync, info, tmo, nullptr, s));
  CP_TRY(launch_apply_S(d, B.LC, B.U, B.y, B.Z, nullptr, s));
  CP_TRY(launch_apply_K(d, B.Gnm, B.Z, B.Kw, B.f, nullptr, s));
  CP_CUDA(cudaMemcpyAsync(f, B.f, d.ncore * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return CP_OK;
}

extern "C" int cp_state_destroy(cp_state* st);

extern "C" int cp_state_create(const cp_shape* shape, const cp_opts* opts, double* a, void* ws,
                               size_t ws_bytes, cp_state** out) {
  if (!opts || !a || !ws || !out) return CP_EINVAL;
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (opts->core_mode != CP_CORE_F64 && opts->core_mode != CP_CORE_MIXED) return CP_EINVAL;
  if (opts->max_iter < 0 || opts->refine_iters < 0 || opts->refine_iters > 64) return CP_EINVAL;
  Layout L;
  make_layout(d, opts->core_mode, 1, &L);
  if (ws_bytes < L.total) return CP_ENOMEM;
  cp_state* st = new (std::nothrow) cp_state;
  if (!st) return CP_ENOMEM;
  // the pass gives the gradient blocks directly (from the residual tensor,
  // accurate relative to the gradient rather than to the MTTKRP) wherever
  // the kernel for the shape can; the two-plane tensor-core pass gives M_n
  d.mg = (d.y_dtype == CP_BF16X2) ? 0 : 1;
  st->d = d;
  st->o = *opts;
  st->a = a;
  st->ws = ws;
  st->L = L;
  st->B = carve(L, ws, d.ncore);
  if (tc_timeout_counter(&st->tmo) != CP_OK) {
    delete st;
    return CP_ECUDA;
  }
  if (opts->core_mode == CP_CORE_MIXED) {
    if (cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st->rhs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev_rhs_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev_rhs_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cp_state_destroy(st);
      return CP_ECUDA;
    }
  }
  *out = st;
  return CP_OK;
}

extern "C" int cp_state_destroy(cp_state* st) {
  if (st) {
    drop_graph(st);
    if (st->ev_fork) cudaEventDestroy(st->ev_fork);
    if (st->ev_join) cudaEventDestroy(st->ev_join);
    if (st->side) cudaStreamDestroy(st->side);
    if (st->rhs) cudaStreamDestroy(st->rhs);
    if (st->ev_rhs_fork) cudaEventDestroy(st->ev_rhs_fork);
    if (st->ev_rhs_join) cudaEventDestroy(st->ev_rhs_join);
  }
  delete st;
  return CP_OK;
}

extern "C" cp_status* cp_state_status(cp_state* st) { return st ? st->B.status : nullptr; }

// ---------------------------------------------------------------------------
// ALS sweeps (Sec. 3, Eq. ALS) on a state's factors: for n = 1..N in turn,
// A^(n) <- M_n (Gamma^(n))^{-1} with M_n from a pass over Y at the current
// factors and Gamma^(n) = Hadamard_{k != n} C^(k) from their Gramians.
// ---------------------------------------------------------------------------
namespace cpdgn {

constexpr int kAlsThreads = 128;

// Rows of A^(n) = M_n Gamma^{-1}.  Every CTA factors Gamma = L L^T (at most
// 32 x 32; one warp, lane i owning row i) in shared memory, then each thread
// solves x Gamma = m for one row by two triangular solves.  A non-positive or
// non-finite pivot leaves A^(n) unchanged and records CP_ENOTSPD with the
// pivot (1-based) in the status, unless an error is recorded already.
__global__ void __launch_bounds__(kAlsThreads) k_als_mode(Dims d, int n, const double* G, const double* Mn,
                                                         double* An, cp_status* st) {
  __shared__ double L[CP_MAX_R * CP_MAX_R];
  __shared__ int bad;
  const int R = d.R, tid = threadIdx.x;
  for (int e = tid; e < R * R; e += blockDim.x) L[e] = G[e];
  if (tid == 0) bad = 0;
  __syncthreads();
  if (tid < 32) {
    for (int j = 0; j < R; ++j) {
      if (tid == j) {
        double p = L[j + R * j];
        if (!(p > 0.0) || !isfinite(p)) {
          if (bad == 0) bad = j + 1;
          p = 1.0;
        }
        L[j + R * j] = sqrt(p);
      }
      __syncwarp();
      if (tid > j && tid < R) L[tid + R * j] /= L[j + R * j];
      __syncwarp();
      if (tid > j && tid < R)
        for (int k = j + 1; k <= tid; ++k) L[tid + R * k] = fma(-L[tid + R * j], L[k + R * j], L[tid + R * k]);
      __syncwarp();
    }
  }
  __syncthreads();
  if (bad) {
    if (blockIdx.x == 0 && tid == 0 && atomicCAS(&st->error, 0, CP_ENOTSPD) == 0) st->info = bad;
    return;
  }
  const int64_t In = d.I[n];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + tid; i < In; i += int64_t(gridDim.x) * blockDim.x) {
    double x[CP_MAX_R];
    for (int r = 0; r < R; ++r) x[r] = Mn[i + In * r];
    for (int r = 0; r < R; ++r) {                 // L y = m^T
      double v = x[r];
      for (int k = 0; k < r; ++k) v = fma(-L[r + R * k], x[k], v);
      x[r] = v / L[r + R * r];
    }
    for (int r = R - 1; r >= 0; --r) {            // L^T x = y
      double v = x[r];
      for (int k = r + 1; k < R; ++k) v = fma(-L[k + R * r], x[k], v);
      x[r] = v / L[r + R * r];
    }
    for (int r = 0; r < R; ++r) An[i + In * r] = x[r];
  }
}

}  // namespace cpdgn

extern "C" int cp_als_sweep(cp_state* st, const void* Y, int sweeps, void* stream) {
  if (!st || !Y || sweeps < 1) return CP_EINVAL;
  const Dims& d = st->d;
  const Bufs& B = st->B;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int it = 0; it < sweeps; ++it)
    for (int n = 0; n < d.N; ++n) {
      CP_CUDA(cudaMemsetAsync(B.m, 0, size_t(d.T) * d.R * sizeof(double), s));
      CP_TRY(launch_mttkrp(d, Y, st->a, B.m, nullptr, nullptr, s, 0));
      CP_TRY(launch_gram(d, st->a, nullptr, B.gpart, B.C, nullptr, B.Gnm, nullptr, nullptr, s));
      int64_t g = (d.I[n] + kAlsThreads - 1) / kAlsThreads;
      if (g > 4 * kSMs) g = 4 * kSMs;
      k_als_mode<<<unsigned(g), kAlsThreads, 0, s>>>(d, n, B.Gnm + (int64_t(n) * d.N + n) * d.RR,
                                                      B.m + d.aoff[n], st->a + d.aoff[n], B.status);
    }
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" double* cp_state_buffer(cp_state* st, int id) {
  if (!st) return nullptr;
  switch (id) {
    case 0: return st->B.m;
    case 1: return st->B.delta;
    case 2: return st->B.Gt;
    case 3: return st->B.w;
    case 4: return st->B.f;
    case 5: return st->B.at;
    default: return nullptr;
  }
}

extern "C" int cp_state_init(cp_state* st, const void* Y, void* stream) {
  if (!st || !Y) return CP_EINVAL;
  const Dims& d = st->d;
  const Bufs& B = st->B;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CP_CUDA(cudaMemsetAsync(B.m, 0, size_t(d.T) * d.R * sizeof(double), s));
  CP_CUDA(cudaMemsetAsync(B.scal, 0, 64 * sizeof(double), s));
  CP_CUDA(cudaMemsetAsync(B.info, 0, 64 * sizeof(int), s));
  CP_TRY(launch_mttkrp(d, Y, st->a, B.m, B.scal + SC_R2, nullptr, s, d.mg));
  int64_t g = (d.J + 255) / 256;
  if (g > 4 * kSMs) g = 4 * kSMs;
  CP_CUDA(launch_pdl(k_sumsq, unsigned(g), 256, 0, s, Y, d.y_dtype, d.J, B.scal + SC_YN2));
  CP_TRY(launch_gram(d, st->a, nullptr, B.gpart, B.C, nullptr, B.Gnm, B.Gall, nullptr, s));
  CP_CUDA(launch_pdl(k_init_status, 1, 32, 0, s, d, st->o, B.Gnm, B.scal, B.status, B.mu, st->tmo, B.info));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" int cp_dgn_step(cp_state* st, const void* Y, void* stream) {
  if (!st || !Y) return CP_EINVAL;
  const Dims& d = st->d;
  const Bufs& B = st->B;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int* skip = &B.status->stop;
  const double* mu = &B.status->mu;
  const int64_t nm = d.T * d.R;
  CP_CUDA(launch_pdl(k_step_begin, unsigned((nm + 255) / 256 < 64 ? (nm + 255) / 256 : 64), 256, 0, s, nm, B.mt, B.scal,
                                                                                       B.info, B.status));
  CP_TRY(launch_gram(d, st->a, B.m, B.gpart, B.C, B.P, nullptr, nullptr, skip, s));
  CP_TRY(launch_mode_prep(d, B.C, B.P, mu, B.Gnm, B.Gt, B.U, B.LC, B.w, B.info + IN_INFO, skip, s));
  CP_TRY(launch_core_w(d, B.Gnm, B.LC, B.U, B.Wp, skip, s));
  if (st->o.core_mode == CP_CORE_F64) {
    CP_TRY(launch_core_fill<double>(d, B.LC, B.U, B.Wp, B.core64, 0, skip, s));
    CP_TRY(chol64_factor(B.core64, d.ncore, B.dinv, B.info + IN_INFO, B.sync, st->tmo, skip, s));
    CP_TRY(solve_core(d, B, B.core64, nullptr, CP_CORE_F64, 0, st->tmo, skip, s));
  } else {
    // the right-hand side runs on a third stream while the core is filled and
    // inverted (the inversion's pivot chain leaves most SMs idle)
    CP_CUDA(cudaEventRecord(st->ev_rhs_fork, s));
    CP_CUDA(cudaStreamWaitEvent(st->rhs, st->ev_rhs_fork, 0));
    CP_TRY(core_rhs(d, B, skip, st->rhs));
    CP_CUDA(cudaEventRecord(st->ev_rhs_join, st->rhs));
    CP_TRY(launch_core_fill<float>(d, B.LC, B.U, B.Wp, B.core32, 1, skip, s));
    float* inv = nullptr;
    // the core's first R^2 x R^2 diagonal block is the identity
    CP_TRY(gj_invert<float>(B.core32, B.core32b, B.pinv, d.ncore, d.RR, B.info + IN_INFO32, skip, s, st->side,
                            st->ev_fork, st->ev_join, &inv));
    CP_CUDA(cudaStreamWaitEvent(s, st->ev_rhs_join, 0));
    // the float64 fallback's core reuses the float32 buffers (2 n^2 floats = n^2 doubles)
    CP_TRY(solve_core(d, B, reinterpret_cast<double*>(B.core32), inv, CP_CORE_MIXED, st->o.refine_iters, st->tmo,
                      skip, s, true));
  }
  const int64_t nupd = update_ctas(d);
  CP_CUDA(launch_pdl(k_update, unsigned(nupd), kUpdRows * 32, 0, s, d, st->a, B.m, B.Gnm, B.Gt, B.f, mu, B.delta, B.at,
                                                    B.part, skip));
  CP_TRY(launch_mttkrp(d, Y, B.at, B.mt, B.scal + SC_R2T, skip, s, d.mg));
  CP_CUDA(launch_pdl(k_control, 1, 256, 0, s, d, st->o, B.part, nupd, B.status, B.scal, B.info, B.scale, st->tmo));
  int64_t gc = (nm + 255) / 256;
  if (gc > 4 * kSMs) gc = 4 * kSMs;
  CP_CUDA(launch_pdl(k_commit, unsigned(gc), 256, 0, s, d, B.info + IN_COMMIT, B.at, B.mt, B.scale, st->a, B.m));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" int cp_dgn_step(cp_state* st, const void* Y, void* stream);

extern "C" int cp_state_capture(cp_state* st, const void* Y, int steps, void* stream) {
  if (!st || !Y || steps < 1) return CP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  drop_graph(st);
  CP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = CP_OK;
  for (int i = 0; i < steps && rc == CP_OK; ++i) rc = cp_dgn_step(st, Y, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc != CP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != CP_OK ? rc : CP_ECUDA;
  }
  size_t nn = 0;
  CP_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  int kernels = 0;
  if (nn) {
    cudaGraphNode_t* nodes = new (std::nothrow) cudaGraphNode_t[nn];
    if (!nodes) { cudaGraphDestroy(g); return CP_ENOMEM; }
    if (cudaGraphGetNodes(g, nodes, &nn) == cudaSuccess) {
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
    }
    delete[] nodes;
  }
  cudaGraphExec_t x = nullptr;
  if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return CP_ECUDA;
  }
  st->graph = g;
  st->exec = x;
  st->graph_steps = steps;
  st->graph_kernels = kernels;
  return CP_OK;
}

extern "C" int cp_state_launch(cp_state* st, void* stream) {
  if (!st || !st->exec) return CP_EINVAL;
  CP_CUDA(cudaGraphLaunch(st->exec, static_cast<cudaStream_t>(stream)));
  return CP_OK;
}

extern "C" int cp_state_graph_kernels(cp_state* st) { return st ? st->graph_kernels : -1; }
