// The damped Hessian's inverse in Theorem 4's block form, and the squared
// angular errors of Sec. 6 (Eq. MedSAE).
//
// Theorem 4:  (H + mu I)^{-1} block (n, m) =
//     delta_nm (Gt^(n) kron I_{I_n}) - (I_R kron A^(n)) St^(n,m) (I_R kron A^(m)T),
//     St = D B_mu D,  D = blkdiag(Gt^(n) kron I_R),  B_mu = K (I + Psi_mu K)^{-1},
// stored as N R x R matrices Gt^(n) and the N R^2 x N R^2 matrix St instead
// of the R T x R T inverse.  With the symmetric positive definite core
// M = I + S^T K S of the step (Psi_mu = S S^T, S = blkdiag(U_n kron L_n)),
// B_mu = K - K S M^{-1} S^T K = K - X^T X with X = L_M^{-1} (S^T K), M = L_M L_M^T:
//   k_stk        W = S^T K, entry by entry: block (n, m), n != m, entry
//                (i + R j, k + R l) = Gamma^(n,m)[k, l] L_n[l, i] U_n[k, j]
//                (K^(n,m) maps e_(k + R l) to Gamma^(n,m)[k, l] e_(l + R k), and
//                (U_n kron L_n)^T vec(E_lk) = vec(L_n^T E_lk U_n));
//   chol64       M = L_M L_M^T (the step's float64 Cholesky);
//   k_trsm_fwd   X = L_M^{-1} W, one warp per right-hand side column;
//   k_kmxtx      B = K - X^T X (32 x 32 tiles);
//   k_scale_l/r  St = D (B D).
// k_hinv_diag gives the diagonal of the inverse from (Gt, St); k_sae the
// squared angular errors after matching the components (Hungarian method).
// Every kernel is plain float64 SIMT code.
#include "common.cuh"

namespace cpdgn {

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
int chol64_factor(double* A, int64_t n, double* dinv, int* info, void* sync, int* tmo, const int* skip,
                  cudaStream_t s);
int tc_timeout_counter(int** out);

constexpr int kTW = 4;            // warps (right-hand sides) per CTA of k_trsm_fwd

// W = S^T K (n x n, column-major); thread = entry.
__global__ void k_stk(Dims d, const double* Gnm, const double* LC, const double* U, double* W) {
  const int64_t n = d.ncore;
  const int R = d.R, RR = d.RR, N = d.N;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = e % n, col = e / n;
    const int bn = int(row / RR), bm = int(col / RR);
    double v = 0.0;
    if (bn != bm) {
      const int x = int(row % RR), y = int(col % RR);
      const int i = x % R, j = x / R, k = y % R, l = y / R;
      const double g = Gnm[(int64_t(bn) * N + bm) * RR + k + R * l];
      v = g * LC[int64_t(bn) * RR + l + R * i] * U[int64_t(bn) * RR + k + R * j];
    }
    W[e] = v;
  }
}

// X = L^{-1} W for the lower Cholesky factor L (n x n) with the inverses of
// its 32 x 32 diagonal tiles in dinv (chol64); one warp per column of W,
// the column held in shared memory.
__global__ void __launch_bounds__(kTW * 32) k_trsm_fwd(const double* L, const double* dinv, int64_t n,
                                                      const double* W, double* X, int64_t ncols) {
  extern __shared__ double xs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t col = int64_t(blockIdx.x) * kTW + warp;
  if (col >= ncols) return;
  double* x = xs + int64_t(warp) * n;
  for (int64_t i = lane; i < n; i += 32) x[i] = W[i + n * col];
  __syncwarp();
  const int nb = int((n + 31) / 32);
  for (int k = 0; k < nb; ++k) {
    const int64_t k0 = int64_t(k) * 32;
    const int64_t row = k0 + lane;
    double r = 0.0;
    if (row < n) {
      double s0 = x[row], s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int64_t j = 0;
      for (; j + 3 < k0; j += 4) {
        s0 = fma(-L[row + n * j], x[j], s0);
        s1 = fma(-L[row + n * (j + 1)], x[j + 1], s1);
        s2 = fma(-L[row + n * (j + 2)], x[j + 2], s2);
        s3 = fma(-L[row + n * (j + 3)], x[j + 3], s3);
      }
      for (; j < k0; ++j) s0 = fma(-L[row + n * j], x[j], s0);
      r = (s0 + s1) + (s2 + s3);
    }
    const double* Xc = dinv + int64_t(k) * 32 * 32;
    double z = 0.0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) z = fma(Xc[lane + 32 * l], __shfl_sync(0xffffffffu, r, l), z);
    __syncwarp();
    if (row < n) x[row] = z;
    __syncwarp();
  }
  for (int64_t i = lane; i < n; i += 32) X[i + n * col] = x[i];
}

// B = K - X^T X (n x n), K from Gamma^(n,m) (see k_stk); 32 x 32 tiles,
// 256 threads, each 2 x 2 entries.
__global__ void __launch_bounds__(256) k_kmxtx(Dims d, const double* Gnm, const double* X, double* B) {
  __shared__ double Xa[32][33], Xb[32][33];
  const int64_t n = d.ncore;
  const int R = d.R, RR = d.RR, N = d.N;
  const int64_t r0 = int64_t(blockIdx.x) * 32, c0 = int64_t(blockIdx.y) * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      const int kk = e & 31, q = e >> 5;
      const int64_t k = k0 + kk;
      Xa[kk][q] = (k < n && r0 + q < n) ? X[k + n * (r0 + q)] : 0.0;
      Xb[kk][q] = (k < n && c0 + q < n) ? X[k + n * (c0 + q)] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double a0 = Xa[kk][tx], a1 = Xa[kk][tx + 16], b0 = Xb[kk][ty], b1 = Xb[kk][ty + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int64_t row = r0 + tx + 16 * u, col = c0 + ty + 16 * v;
      if (row >= n || col >= n) continue;
      const int bn = int(row / RR), bm = int(col / RR);
      double kv = 0.0;
      if (bn != bm) {
        const int x = int(row % RR), y = int(col % RR);
        const int k = y % R, l = y / R;
        if (x == l + R * k) kv = Gnm[(int64_t(bn) * N + bm) * RR + k + R * l];
      }
      B[row + n * col] = kv - acc[u][v];
    }
}

// Right factor: Out = In D, D = blkdiag(Gt^(m) kron I_R):
// Out[row, (m, c + R dd)] = sum_e In[row, (m, c + R e)] Gt^(m)[e, dd].
__global__ void k_scale_r(Dims d, const double* Gt, const double* In, double* Out) {
  const int64_t n = d.ncore;
  const int R = d.R, RR = d.RR;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = e % n, col = e / n;
    const int m = int(col / RR), y = int(col % RR), c = y % R, dd = y / R;
    const double* g = Gt + int64_t(m) * RR;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(In[row + n * (int64_t(m) * RR + c + R * k)], g[k + R * dd], s);
    Out[e] = s;
  }
}

// Left factor: Out = D In: Out[(n, a + R b), col] = sum_e Gt^(n)[b, e] In[(n, a + R e), col].
__global__ void k_scale_l(Dims d, const double* Gt, const double* In, double* Out) {
  const int64_t n = d.ncore;
  const int R = d.R, RR = d.RR;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = e % n, col = e / n;
    const int bn = int(row / RR), x = int(row % RR), a = x % R, b = x / R;
    const double* g = Gt + int64_t(bn) * RR;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(g[b + R * k], In[(int64_t(bn) * RR + a + R * k) + n * col], s);
    Out[e] = s;
  }
}

// diag(H_mu^{-1}) entry for parameter (mode n, row i, column r):
// Gt^(n)[r, r] - sum_{s, s'} A[i, s] St[(n, s + R r), (n, s' + R r)] A[i, s'].
__global__ void k_hinv_diag(Dims d, const double* a, const double* Gt, const double* St, double* out) {
  const int64_t n = d.ncore;
  const int R = d.R, RR = d.RR;
  const int64_t tot = d.T * R;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < tot; e += int64_t(gridDim.x) * blockDim.x) {
    int m = 0;
    while (m + 1 < d.N && e >= d.aoff[m + 1]) ++m;
    const int64_t In = d.I[m];
    const int64_t q = e - d.aoff[m];
    const int64_t i = q % In;
    const int r = int(q / In);
    const double* A = a + d.aoff[m];
    const int64_t base = int64_t(m) * RR + int64_t(R) * r;
    double s = 0.0;
    for (int s1 = 0; s1 < R; ++s1) {
      double t = 0.0;
      for (int s2 = 0; s2 < R; ++s2) t = fma(St[(base + s1) + n * (base + s2)], A[i + In * s2], t);
      s = fma(A[i + In * s1], t, s);
    }
    out[e] = Gt[int64_t(m) * RR + r + R * r] - s;
  }
}

// Squared angular errors after matching (Eq. MedSAE).  One CTA: the
// absolute cosines |cos(a_r^(n), ahat_c^(n))| of every mode, their sum over
// the modes as the assignment score, the permutation pi maximising the total
// score by the Hungarian method (Kuhn-Munkres with row and column
// potentials, O(R^3), one thread), then alpha^2[n, r] = arccos(|cos|)^2 of
// the matched pairs.  alpha2: N x R (mode-major), pi: R ints.
__device__ __forceinline__ double abs_cos(const Dims& d, const double* at, const double* ae, int n, int r, int c,
                                          const double (*nt)[CP_MAX_R], const double (*ne)[CP_MAX_R]) {
  const int64_t In = d.I[n];
  const double* x = at + d.aoff[n] + In * r;
  const double* y = ae + d.aoff[n] + In * c;
  double s = 0.0;
  for (int64_t i = 0; i < In; ++i) s = fma(x[i], y[i], s);
  const double v = fabs(s) / (nt[n][r] * ne[n][c]);
  return v > 1.0 ? 1.0 : v;
}

__global__ void __launch_bounds__(256) k_sae(Dims d, const double* at, const double* ae, double* alpha2, int* pi) {
  __shared__ double score[CP_MAX_R][CP_MAX_R];
  __shared__ double nt[CP_MAX_N][CP_MAX_R], ne[CP_MAX_N][CP_MAX_R];
  __shared__ int match[CP_MAX_R];
  const int R = d.R, N = d.N, tid = threadIdx.x;
  for (int e = tid; e < N * R; e += blockDim.x) {
    const int n = e / R, r = e % R;
    const int64_t In = d.I[n];
    const double* x = at + d.aoff[n] + In * r;
    const double* y = ae + d.aoff[n] + In * r;
    double sx = 0.0, sy = 0.0;
    for (int64_t i = 0; i < In; ++i) {
      sx = fma(x[i], x[i], sx);
      sy = fma(y[i], y[i], sy);
    }
    nt[n][r] = sqrt(sx);
    ne[n][r] = sqrt(sy);
  }
  __syncthreads();
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e % R;
    double sc = 0.0;
    for (int n = 0; n < N; ++n) sc += abs_cos(d, at, ae, n, r, c, nt, ne);
    score[r][c] = sc;
  }
  __syncthreads();
  if (tid == 0) {
    // minimise cost[r][c] = -score[r][c]; rows r = true components, columns c = estimates
    double u[CP_MAX_R + 1], v[CP_MAX_R + 1], minv[CP_MAX_R + 1];
    int p[CP_MAX_R + 1], way[CP_MAX_R + 1];
    bool used[CP_MAX_R + 1];
    for (int j = 0; j <= R; ++j) { u[j] = 0.0; v[j] = 0.0; p[j] = 0; way[j] = 0; }
    for (int i = 1; i <= R; ++i) {
      p[0] = i;
      int j0 = 0;
      for (int j = 0; j <= R; ++j) { minv[j] = 1e300; used[j] = false; }
      do {
        used[j0] = true;
        const int i0 = p[j0];
        double delta = 1e300;
        int j1 = 0;
        for (int j = 1; j <= R; ++j) {
          if (used[j]) continue;
          const double cur = -score[i0 - 1][j - 1] - u[i0] - v[j];
          if (cur < minv[j]) { minv[j] = cur; way[j] = j0; }
          if (minv[j] < delta) { delta = minv[j]; j1 = j; }
        }
        for (int j = 0; j <= R; ++j) {
          if (used[j]) { u[p[j]] += delta; v[j] -= delta; }
          else minv[j] -= delta;
        }
        j0 = j1;
      } while (p[j0] != 0);
      do {
        const int j1 = way[j0];
        p[j0] = p[j1];
        j0 = j1;
      } while (j0);
    }
    for (int j = 1; j <= R; ++j) match[p[j] - 1] = j - 1;
  }
  __syncthreads();
  for (int e = tid; e < N * R; e += blockDim.x) {
    const int n = e / R, r = e % R;
    const double ang = acos(abs_cos(d, at, ae, n, r, match[r], nt, ne));
    alpha2[e] = ang * ang;
  }
  if (tid < R) pi[tid] = match[tid];
}

static size_t hinv_extra(int64_t n) { return 3 * align256(size_t(n) * size_t(n) * sizeof(double)); }

}  // namespace cpdgn

using namespace cpdgn;

extern "C" int cp_hinv_workspace_bytes(const cp_shape* shape, size_t* bytes) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!bytes) return CP_EINVAL;
  Layout L;
  make_layout(d, CP_CORE_F64, 0, &L);
  *bytes = L.total + hinv_extra(d.ncore);
  return CP_OK;
}

extern "C" int cp_hinv_blocks(const cp_shape* shape, const double* a, const double* mu, double* Gt, double* St,
                              int* info, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !mu || !Gt || !St || !info || !ws) return CP_EINVAL;
  Layout L;
  make_layout(d, CP_CORE_F64, 0, &L);
  const int64_t n = d.ncore;
  if (ws_bytes < L.total + hinv_extra(n)) return CP_ENOMEM;
  if (size_t(kTW) * size_t(n) * sizeof(double) > 200 * 1024) return CP_EINVAL;   // n <= 6400
  char* base = static_cast<char*>(ws);
  double* C = reinterpret_cast<double*>(base + L.off[S_C]);
  double* Gnm = reinterpret_cast<double*>(base + L.off[S_GNM]);
  double* LC = reinterpret_cast<double*>(base + L.off[S_LC]);
  double* U = reinterpret_cast<double*>(base + L.off[S_U]);
  double* Wp = reinterpret_cast<double*>(base + L.off[S_WP]);
  double* gpart = reinterpret_cast<double*>(base + L.off[S_GPART]);
  double* dinv = reinterpret_cast<double*>(base + L.off[S_DINV]);
  void* sync = base + L.off[S_SYNC];
  const size_t nn = align256(size_t(n) * size_t(n) * sizeof(double));
  double* M = reinterpret_cast<double*>(base + L.total);
  double* W = reinterpret_cast<double*>(base + L.total + nn);
  double* X = reinterpret_cast<double*>(base + L.total + 2 * nn);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* tmo = nullptr;
  CP_TRY(tc_timeout_counter(&tmo));
  CP_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
  CP_TRY(launch_gram(d, a, nullptr, gpart, C, nullptr, nullptr, nullptr, nullptr, s));
  CP_TRY(launch_mode_prep(d, C, nullptr, mu, Gnm, Gt, U, LC, nullptr, info, nullptr, s));
  CP_TRY(launch_core_w(d, Gnm, LC, U, Wp, nullptr, s));
  CP_TRY(launch_core_fill<double>(d, LC, U, Wp, M, 0, nullptr, s));
  CP_TRY(chol64_factor(M, n, dinv, info, sync, tmo, nullptr, s));
  int64_t g = (n * n + 255) / 256;
  if (g > 8 * kSMs) g = 8 * kSMs;
  k_stk<<<unsigned(g), 256, 0, s>>>(d, Gnm, LC, U, W);
  const size_t smem = size_t(kTW) * size_t(n) * sizeof(double);
  CP_CUDA(cudaFuncSetAttribute(k_trsm_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  k_trsm_fwd<<<unsigned((n + kTW - 1) / kTW), kTW * 32, smem, s>>>(M, dinv, n, W, X, n);
  const unsigned nt = unsigned((n + 31) / 32);
  k_kmxtx<<<dim3(nt, nt), 256, 0, s>>>(d, Gnm, X, W);                   // W <- B
  k_scale_r<<<unsigned(g), 256, 0, s>>>(d, Gt, W, X);                   // X <- B D
  k_scale_l<<<unsigned(g), 256, 0, s>>>(d, Gt, X, St);                  // St <- D B D
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" int cp_hinv_diag(const cp_shape* shape, const double* a, const double* Gt, const double* St,
                            double* diag, void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !Gt || !St || !diag) return CP_EINVAL;
  int64_t g = (d.T * d.R + 255) / 256;
  if (g > 8 * kSMs) g = 8 * kSMs;
  k_hinv_diag<<<unsigned(g), 256, 0, static_cast<cudaStream_t>(stream)>>>(d, a, Gt, St, diag);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" int cp_sae(const cp_shape* shape, const double* a_true, const double* a_est, double* alpha2, int* perm,
                      void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a_true || !a_est || !alpha2 || !perm) return CP_EINVAL;
  k_sae<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(d, a_true, a_est, alpha2, perm);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
