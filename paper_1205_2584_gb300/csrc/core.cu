// Damped per-mode inverses, w, and the symmetric positive definite core system.
//
// Theorem 3 writes (H + mu I)^{-1} = Gt - L_mu B_mu L_mu^T with
// B_mu = K (I + Psi_mu K)^{-1} (Eq. inverse_f1a).  With Psi_mu = S S^T,
// S = blkdiag(S_n), S_n = U_n kron L_n, where Gamma^(n) + mu I = L_G L_G^T,
// U_n = L_G^{-T} (U_n U_n^T = Gt^(n)) and C^(n) = L_n L_n^T, the push-through
// identity gives
//     B_mu w = K w - K S (I + S^T K S)^{-1} S^T K w,
// and core = I + S^T K S is symmetric positive definite whenever H + mu I is
// and every A^(n) has full column rank (x^T core x = v^T (H + mu I) v for
// v = Gt Z Psi^{-1} S x).  This replaces the paper's non-symmetric Phi_1 and
// the indefinite Phi_2 of Sec. 4.4 by a matrix that needs no pivoting.
//
// Block (n, m), n != m, of S^T K S, entry (i + R j, k + R l):
//     sum_a L_n[a,i] U_m[a,l] W_nm[a, (k,j)],
//     W_nm[a, (k,j)] = sum_b Gamma^(n,m)[a,b] L_m[b,k] U_n[b,j],
// which costs O(R^5) per block instead of the O(R^6) of the dense product.
//
// The matrix-free operators apply S, S^T and K in O(N R^3) and O(N^2 R^2)
// float64 operations (Kronecker identity (U kron L) vec X = vec(L X U^T);
// K^(n,m) vec X = vec((Gamma^(n,m) * X)^T)).
//
// Every kernel stages its operands in shared memory with coalesced loads
// before computing: float64 runs at 2 FMA/clock/SM on GB300, and a dependent
// global load inside an FMA loop would dominate these small kernels.
#include "common.cuh"
#include "small.cuh"

namespace cpdgn {

constexpr int kRR = CP_MAX_R * CP_MAX_R;

constexpr int kPrepThreads = 128;
constexpr int kPrepWarps = kPrepThreads / 32;
static_assert(kPrepWarps == 4, "the partial sums of k_mode_prep are added as four terms");

// CTA (n, j), j < R: column j of Gt^(n), U_n and w_n.
//   Gt[:, j] = L_G^{-T} L_G^{-1} e_j;  U[:, j] = L_G^{-T} e_j
//   w_n[:, j] = P^(n) Gt[:, j] - C^(n) (Gamma^(n) Gt[:, j])     (Appendix D)
//   (P^(n) = A^(n)T M_n; when the state's pass gives the gradient blocks,
//   P^(n) = A^(n)T G_n and w_n[:, j] = P^(n) Gt[:, j])
// CTA (n, 0) also writes Gamma^(n,m) for every m.
// CTA N R + n: L_n = chol(C^(n)) (independent of mu).
__global__ void __launch_bounds__(kPrepThreads) k_mode_prep(Dims d, const double* C, const double* P,
                                                            const double* mu, double* Gnm, double* Gt,
                                                            double* U, double* LC, double* w, int* info,
                                                            const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double G[kRR], Gam[kRR], Cn[kRR], Pn[kRR];
  __shared__ double z[CP_MAX_R], u[CP_MAX_R], v[CP_MAX_R], rinv[CP_MAX_R];
  __shared__ double part[2][kPrepWarps][CP_MAX_R];
  __shared__ int okc;
  const int R = d.R, RR = d.RR, N = d.N;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (int(blockIdx.x) >= N * R) {                 // Cholesky of C^(n)
    const int n = blockIdx.x - N * R;
    for (int e = tid; e < RR; e += kPrepThreads) G[e] = C[int64_t(n) * RR + e];
    const bool ok = cta_chol(G, rinv, R, &okc);
    if (tid == 0 && info && !ok) atomicCAS(info, 0, n + 1);
    for (int e = tid; e < RR; e += kPrepThreads) {
      const int i = e % R, jj = e / R;
      LC[int64_t(n) * RR + e] = (i >= jj) ? G[e] : 0.0;
    }
    return;
  }
  const int n = blockIdx.x / R, j = blockIdx.x % R;
  const double muv = *mu;
  for (int e = tid; e < RR; e += kPrepThreads) {
    double g = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != n) g *= C[int64_t(k) * RR + e];
    Gam[e] = g;
    G[e] = g + ((e % R) == (e / R) ? muv : 0.0);
    Cn[e] = C[int64_t(n) * RR + e];
    Pn[e] = P ? P[int64_t(n) * RR + e] : 0.0;
    if (j == 0 && Gnm) {
      for (int m = 0; m < N; ++m) {
        double h = 1.0;
        for (int k = 0; k < N; ++k)
          if (k != n && k != m) h *= C[int64_t(k) * RR + e];
        Gnm[(int64_t(n) * N + m) * RR + e] = h;
      }
    }
  }
  const bool okG = cta_chol(G, rinv, R, &okc);
  if (tid == 0 && j == 0 && info && !okG) atomicCAS(info, 0, n + 1);
  if (warp < 2) {                 // warp 0: z = Gt e_j; warp 1: u = L_G^{-T} e_j, concurrently
    const double rl = lane < R ? rinv[lane] : 1.0;
    double x = (lane == j) ? 1.0 : 0.0;
    if (warp == 0) x = warp_fwd_reg(G, rl, x, R);
    x = warp_bwd_reg(G, rl, x, R);
    if (lane < R) (warp == 0 ? z : u)[lane] = x;
  }
  __syncthreads();
  // the three length-R dot products per entry below are float64 chains of
  // ~40-cycle dependent multiply-adds; each is split over the four warps
  // (warp w takes every fourth term) and the partial sums added in order
  if (lane < R) {
    double s = 0.0;
    for (int c = warp; c < R; c += kPrepWarps) s = fma(Gam[lane + R * c], z[c], s);
    part[0][warp][lane] = s;
  }
  __syncthreads();
  if (tid < R) v[tid] = (part[0][0][tid] + part[0][1][tid]) + (part[0][2][tid] + part[0][3][tid]);
  __syncthreads();
  if (lane < R) {
    double s = 0.0, t = 0.0;
    for (int c = warp; c < R; c += kPrepWarps) {
      s = fma(Pn[lane + R * c], z[c], s);
      t = fma(Cn[lane + R * c], v[c], t);
    }
    part[0][warp][lane] = s;
    part[1][warp][lane] = t;
  }
  __syncthreads();
  if (tid < R) {
    const int64_t o = int64_t(n) * RR + tid + int64_t(R) * j;
    const double s = (part[0][0][tid] + part[0][1][tid]) + (part[0][2][tid] + part[0][3][tid]);
    const double t = (part[1][0][tid] + part[1][1][tid]) + (part[1][2][tid] + part[1][3][tid]);
    Gt[o] = z[tid];
    U[o] = u[tid];
    // with gradient blocks in P (P = A^T G, G = M - A Gamma) the C Gamma term is already in it
    if (w) w[o] = d.mg ? s : s - t;
  }
}

int launch_mode_prep(const Dims& d, const double* C, const double* P, const double* mu, double* Gnm,
                     double* Gt, double* U, double* LC, double* w, int* info, const int* skip,
                     cudaStream_t s) {
  CP_CUDA(launch_pdl(k_mode_prep, d.N * d.R + d.N, kPrepThreads, 0, s, d, C, P, mu, Gnm, Gt, U, LC, w, info, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

// ---------------------------------------------------------------------------
// core = I + S^T K S
// ---------------------------------------------------------------------------

// pair p -> (n, m) with n > m, enumerated row by row: (1,0), (2,0), (2,1), ...
__device__ __forceinline__ void pair_of(int p, int* n, int* m) {
  int nn = 1;
  while ((nn * (nn + 1)) / 2 <= p) ++nn;
  *n = nn;
  *m = p - (nn * (nn - 1)) / 2;
}

// CTA (pair p, j): W_nm[a + R (k + R j)] = sum_b Gamma^(n,m)[a,b] L_m[b,k] U_n[b,j].
__global__ void __launch_bounds__(256) k_core_w(Dims d, const double* Gnm, const double* LC,
                                                const double* U, double* Wp, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double G[kRR], Lm[kRR], un[CP_MAX_R];
  const int R = d.R, RR = d.RR, N = d.N;
  const int p = blockIdx.x / R, j = blockIdx.x % R;
  int n, m;
  pair_of(p, &n, &m);
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    G[e] = Gnm[(int64_t(n) * N + m) * RR + e];
    Lm[e] = LC[int64_t(m) * RR + e];
  }
  if (threadIdx.x < R) un[threadIdx.x] = U[int64_t(n) * RR + threadIdx.x + R * j];
  __syncthreads();
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    const int a = e % R, k = e / R;
    double s = 0.0;
    // L_m[b,k] = 0 for b < k and U_n[b,j] = 0 for b > j
    for (int b = k; b <= j; ++b) s = fma(G[a + R * b], Lm[b + R * k] * un[b], s);
    Wp[int64_t(p) * RR * R + a + R * (k + R * j)] = s;
  }
}

// One CTA per column of a lower block (n > m) or of a diagonal block; thread
// = row i + R j inside the block.  full != 0 also writes the mirrored upper
// block (the Gauss-Jordan inversion reads the full matrix).
template <typename T>
__global__ void k_core_fill(Dims d, const double* LC, const double* U, const double* Wp, T* core,
                            int64_t ld, int full, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR, N = d.N;
  const int npairs = N * (N - 1) / 2;
  const int blk = blockIdx.x / RR;
  const int kap = blockIdx.x % RR;
  const int rho = threadIdx.x;
  if (blk >= npairs) {
    const int n = blk - npairs;
    if (rho < RR && (full || rho >= kap))
      core[(int64_t(n) * RR + rho) + ld * (int64_t(n) * RR + kap)] = T(rho == kap ? 1 : 0);
    return;
  }
  int n, m;
  pair_of(blk, &n, &m);
  __shared__ T Ln[kRR];
  __shared__ T Uml[CP_MAX_R];
  __shared__ T Wk[kRR];
  const int k = kap % R, l = kap / R;
  const double* W = Wp + int64_t(blk) * RR * R;
  for (int e = rho; e < RR; e += blockDim.x) {
    Ln[e] = T(LC[int64_t(n) * RR + e]);
    const int a = e % R, jj = e / R;
    Wk[e] = T(W[a + R * (k + R * jj)]);
  }
  if (rho < R) Uml[rho] = T(U[int64_t(m) * RR + rho + R * l]);
  __syncthreads();
  if (rho >= RR) return;
  const int i = rho % R, j = rho / R;
  T s = T(0);
  // L_n[a,i] = 0 for a < i and U_m[a,l] = 0 for a > l
  for (int a = i; a <= l; ++a) s = fma(Ln[a + R * i] * Uml[a], Wk[a + R * j], s);
  const int64_t row = int64_t(n) * RR + rho, col = int64_t(m) * RR + kap;
  core[row + ld * col] = s;
  if (full) core[col + ld * row] = s;
}

int launch_core_w(const Dims& d, const double* Gnm, const double* LC, const double* U, double* Wp,
                  const int* skip, cudaStream_t s) {
  const int npairs = d.N * (d.N - 1) / 2;
  if (npairs == 0) return CP_OK;
  CP_CUDA(launch_pdl(k_core_w, npairs * d.R, 256, 0, s, d, Gnm, LC, U, Wp, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

template <typename T>
int launch_core_fill(const Dims& d, const double* LC, const double* U, const double* Wp, T* core, int full,
                     const int* skip, cudaStream_t s) {
  const int npairs = d.N * (d.N - 1) / 2;
  int threads = ((d.RR + 31) / 32) * 32;
  CP_CUDA(launch_pdl(k_core_fill<T>, (npairs + d.N) * d.RR, threads, 0, s, d, LC, U, Wp, core, d.ncore, full, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
template int launch_core_fill<double>(const Dims&, const double*, const double*, const double*, double*,
                                      int, const int*, cudaStream_t);
template int launch_core_fill<float>(const Dims&, const double*, const double*, const double*, float*,
                                     int, const int*, cudaStream_t);

// ---------------------------------------------------------------------------
// Matrix-free float64 operators on vectors of length N R^2
// ---------------------------------------------------------------------------
constexpr int kOpThreads = 128;

// Columns 0..jmax of V = (K x)_n into shared memory:
// V[i + R j] = sum_{m != n} Gamma^(n,m)[i,j] X_m[j,i]
__device__ void stage_Kx(const Dims& d, int n, int jmax, const double* Gnm, const double* x, double* V) {
  const int R = d.R, RR = d.RR, N = d.N;
  for (int e = threadIdx.x; e < R * (jmax + 1); e += blockDim.x) {
    const int i = e % R, j = e / R;
    double s = 0.0;
    for (int m = 0; m < N; ++m)
      if (m != n) s = fma(Gnm[(int64_t(n) * N + m) * RR + e], x[int64_t(m) * RR + j + R * i], s);
    V[e] = s;
  }
}

// out = K x (base == null) or out = base - K x; one thread per entry.
__global__ void k_apply_K(Dims d, const double* Gnm, const double* x, const double* base, double* out,
                          const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR, N = d.N;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= d.ncore) return;
  const int n = int(idx / RR), e = int(idx % RR);
  const int i = e % R, j = e / R;
  double s = 0.0;
  for (int m = 0; m < N; ++m)
    if (m != n) s = fma(Gnm[(int64_t(n) * N + m) * RR + e], x[int64_t(m) * RR + j + R * i], s);
  out[idx] = base ? base[idx] - s : s;
}

// The two small products of a column of S x / S^T x are float64 dot products
// of length <= R.  Each is split over the CTA's four warps (thread (w, p)
// takes every fourth term, starting at w) so that all four sub-partitions of
// the SM feed its float64 pipe; the four partial sums are then added in a
// fixed order.
constexpr int kOpWarps = kOpThreads / 32;
static_assert(kOpWarps == 4, "the partial sums below are added as four terms");

// out_m = vec(L_m X_m U_m^T): CTA (m, q) computes column q.
__global__ void __launch_bounds__(kOpThreads) k_apply_S(Dims d, const double* LC, const double* U,
                                                        const double* x, double* out, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double X[kRR], L[kRR], uq[CP_MAX_R], t[CP_MAX_R];
  __shared__ double part[2][kOpWarps][CP_MAX_R];
  const int R = d.R, RR = d.RR;
  const int m = blockIdx.x / R, q = blockIdx.x % R;
  const int tid = threadIdx.x, w = tid / 32, p = tid % 32;
  for (int e = tid; e < RR; e += kOpThreads) {
    X[e] = x[int64_t(m) * RR + e];
    L[e] = LC[int64_t(m) * RR + e];
  }
  if (tid < R) uq[tid] = U[int64_t(m) * RR + q + R * tid];   // row q of U_m
  __syncthreads();
  if (p < R) {   // t = X U_m[q, :]^T ; U_m upper: U_m[q,l] = 0 for l < q
    double s = 0.0;
    for (int l = q + w; l < R; l += kOpWarps) s = fma(X[p + R * l], uq[l], s);
    part[0][w][p] = s;
  }
  __syncthreads();
  if (tid < R) t[tid] = (part[0][0][tid] + part[0][1][tid]) + (part[0][2][tid] + part[0][3][tid]);
  __syncthreads();
  if (p < R) {   // out[:, q] = L_m t ; L_m[p,k] = 0 for k > p
    double s = 0.0;
    for (int k = w; k <= p; k += kOpWarps) s = fma(L[p + R * k], t[k], s);
    part[1][w][p] = s;
  }
  __syncthreads();
  if (tid < R)
    out[int64_t(m) * RR + tid + R * q] = (part[1][0][tid] + part[1][1][tid]) + (part[1][2][tid] + part[1][3][tid]);
}

// out_n = vec(L_n^T V_n U_n) with V_n = x_n (kx = 0) or V_n = (K x)_n (kx = 1).
// b != null: out = b - y - (that)  (refinement residual b - y - S^T K S y).
// kw != null (kx = 1): CTA q also stores column q of V_n = (K x)_n into kw.
// Column q needs columns 0..q of V_n only (U_n is upper triangular).
__global__ void __launch_bounds__(kOpThreads) k_apply_ST(Dims d, const double* LC, const double* U,
                                                         const double* Gnm, const double* x, int kx,
                                                         const double* b, const double* y, double* out,
                                                         double* kw, double* norm2, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double V[kRR], L[kRR], uq[CP_MAX_R], t[CP_MAX_R];
  __shared__ double part[2][kOpWarps][CP_MAX_R];
  const int R = d.R, RR = d.RR;
  const int n = blockIdx.x / R, q = blockIdx.x % R;
  const int tid = threadIdx.x, w = tid / 32, p = tid % 32;
  if (kx) {
    stage_Kx(d, n, q, Gnm, x, V);
  } else {
    for (int e = tid; e < R * (q + 1); e += kOpThreads) V[e] = x[int64_t(n) * RR + e];
  }
  for (int e = tid; e < RR; e += kOpThreads) L[e] = LC[int64_t(n) * RR + e];
  if (tid < R) uq[tid] = U[int64_t(n) * RR + tid + R * q];   // column q of U_n
  __syncthreads();
  if (kw && tid < R) kw[int64_t(n) * RR + tid + R * q] = V[tid + R * q];
  if (p < R) {   // t = V U_n[:, q] ; U_n[l,q] = 0 for l > q
    double s = 0.0;
    for (int l = w; l <= q; l += kOpWarps) s = fma(V[p + R * l], uq[l], s);
    part[0][w][p] = s;
  }
  __syncthreads();
  if (tid < R) t[tid] = (part[0][0][tid] + part[0][1][tid]) + (part[0][2][tid] + part[0][3][tid]);
  __syncthreads();
  if (p < R) {   // out[:, q] = L_n^T t ; L_n[k,p] = 0 for k < p
    double s = 0.0;
    for (int k = p + w; k < R; k += kOpWarps) s = fma(L[k + R * p], t[k], s);
    part[1][w][p] = s;
  }
  __syncthreads();
  if (tid < R) {
    const double s = (part[1][0][tid] + part[1][1][tid]) + (part[1][2][tid] + part[1][3][tid]);
    const int64_t o = int64_t(n) * RR + tid + R * q;
    const double val = b ? (b[o] - y[o] - s) : s;
    out[o] = val;
    t[tid] = val * val;
  }
  if (norm2) {   // ||out||^2 accumulated over the CTAs by warp 0
    __syncthreads();
    if (tid < 32) {
      double sq = (tid < R) ? t[tid] : 0.0;
      for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
      if (tid == 0) atomicAdd(norm2, sq);
    }
  }
}

int launch_apply_K(const Dims& d, const double* Gnm, const double* x, const double* base, double* out,
                   const int* skip, cudaStream_t s) {
  CP_CUDA(launch_pdl(k_apply_K, unsigned((d.ncore + 127) / 128), 128, 0, s, d, Gnm, x, base, out, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
int launch_apply_S(const Dims& d, const double* LC, const double* U, const double* x, double* out,
                   const int* skip, cudaStream_t s) {
  CP_CUDA(launch_pdl(k_apply_S, d.N * d.R, kOpThreads, 0, s, d, LC, U, x, out, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
int launch_apply_ST(const Dims& d, const double* LC, const double* U, const double* Gnm, const double* x,
                    int kx, const double* b, const double* y, double* out, double* kw, double* norm2,
                    const int* skip, cudaStream_t s) {
  CP_CUDA(launch_pdl(k_apply_ST, d.N * d.R, kOpThreads, 0, s, d, LC, U, Gnm, x, kx, b, y, out, kw, norm2, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn
