// Blocked right-looking Cholesky of the N R^2 x N R^2 core system and the two
// triangular solves, for T = double (float64 core mode) and T = float (mixed
// mode, refined in float64 by the caller).  Column-major, lower triangle;
// the upper triangle is never read and is left unspecified.
//
// Per panel step k0 (block width NB):
//   k_chol_panel : every CTA factors the diagonal block in shared memory;
//                  CTA 0 writes it, CTA b > 0 solves row block b of the panel
//                  (X <- X L_kk^{-T}) and writes it;
//   k_chol_update: trailing update A_ij -= L_ik L_jk^T over 64 x 64 tiles of
//                  the lower triangle.
// A non-positive or non-finite pivot records its 1-based index in *info
// (first one wins) and the factorisation continues with NaNs; nothing traps.
#include "common.cuh"

namespace cpdgn {

constexpr int NB = 32;        // panel width
constexpr int TB = 64;        // trailing-update tile
constexpr int PT = 256;       // threads of the panel / update kernels

template <typename T>
__device__ void factor_diag(T (*D)[NB + 1], int kb, int* bad) {
  const int tid = threadIdx.x;
  for (int c = 0; c < kb; ++c) {
    __syncthreads();
    const T piv = D[c][c];
    if (tid == 0 && (!(piv > T(0)) || !isfinite(double(piv))) && *bad == 0) *bad = c + 1;
    const T dc = sqrt(piv);
    __syncthreads();
    if (tid == 0) D[c][c] = dc;
    for (int i = c + 1 + tid; i < kb; i += PT) D[i][c] /= dc;
    __syncthreads();
    const int m = kb - c - 1;   // trailing size
    for (int e = tid; e < m * m; e += PT) {
      const int i = c + 1 + e % m, l = c + 1 + e / m;
      if (l <= i) D[i][l] -= D[i][c] * D[l][c];
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(PT) k_chol_panel(T* A, int64_t n, int64_t k0, int* info,
                                                   const int* skip) {
  if (skip && *skip) return;
  __shared__ T D[NB][NB + 1];
  __shared__ T X[NB][NB + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int kb = int((n - k0) < NB ? (n - k0) : NB);
  if (tid == 0) bad = 0;
  for (int e = tid; e < kb * kb; e += PT) {
    const int i = e % kb, l = e / kb;
    D[i][l] = A[(k0 + i) + n * (k0 + l)];
  }
  factor_diag<T>(D, kb, &bad);
  if (blockIdx.x == 0) {
    if (tid == 0 && bad && info) atomicCAS(info, 0, int(k0) + bad);
    for (int e = tid; e < kb * kb; e += PT) {
      const int i = e % kb, l = e / kb;
      if (i >= l) A[(k0 + i) + n * (k0 + l)] = D[i][l];
    }
    return;
  }
  const int64_t i0 = k0 + int64_t(blockIdx.x) * NB;
  if (i0 >= n) return;
  const int ib = int((n - i0) < NB ? (n - i0) : NB);
  for (int e = tid; e < ib * kb; e += PT) {
    const int i = e % ib, l = e / ib;
    X[i][l] = A[(i0 + i) + n * (k0 + l)];
  }
  __syncthreads();
  // X <- X D^{-T}: column c of the result depends on columns < c
  for (int c = 0; c < kb; ++c) {
    for (int i = tid; i < ib; i += PT) X[i][c] /= D[c][c];
    __syncthreads();
    const int m = kb - c - 1;
    for (int e = tid; e < ib * m; e += PT) {
      const int i = e % ib, l = c + 1 + e / ib;
      X[i][l] -= X[i][c] * D[l][c];
    }
    __syncthreads();
  }
  for (int e = tid; e < ib * kb; e += PT) {
    const int i = e % ib, l = e / ib;
    A[(i0 + i) + n * (k0 + l)] = X[i][l];
  }
}

// Trailing update of the lower triangle of A[k1:n, k1:n], k1 = k0 + kb.
template <typename T>
__global__ void __launch_bounds__(PT) k_chol_update(T* A, int64_t n, int64_t k0, int kb,
                                                    const int* skip) {
  if (skip && *skip) return;
  __shared__ T Pi[TB][NB + 1];
  __shared__ T Pj[TB][NB + 1];
  const int64_t k1 = k0 + kb;
  // tile (ti, tj), ti >= tj, from the linear block index
  int ti = 0;
  {
    const int b = blockIdx.x;
    ti = int((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while (ti * (ti + 1) / 2 > b) --ti;
  }
  const int tj = blockIdx.x - ti * (ti + 1) / 2;
  const int64_t r0 = k1 + int64_t(ti) * TB, c0 = k1 + int64_t(tj) * TB;
  const int tid = threadIdx.x;
  for (int e = tid; e < TB * kb; e += PT) {
    const int i = e % TB, l = e / TB;
    const int64_t ri = r0 + i, cj = c0 + i;
    Pi[i][l] = (ri < n) ? A[ri + n * (k0 + l)] : T(0);
    Pj[i][l] = (cj < n) ? A[cj + n * (k0 + l)] : T(0);
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int l = 0; l < kb; ++l) {
    T a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = Pi[tx + 16 * u][l];
#pragma unroll
    for (int v = 0; v < 4; ++v) b[v] = Pj[ty + 16 * v][l];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t r = r0 + tx + 16 * u, c = c0 + ty + 16 * v;
      if (r < n && c < n && r >= c) A[r + n * c] -= acc[u][v];
    }
  }
}

template <typename T>
int chol_factor(T* A, int64_t n, int* info, const int* skip, cudaStream_t s) {
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int kb = int((n - k0) < NB ? (n - k0) : NB);
    const int64_t nbr = (n - k0 + NB - 1) / NB;
    k_chol_panel<T><<<unsigned(nbr), PT, 0, s>>>(A, n, k0, info, skip);
    const int64_t rest = n - k0 - kb;
    if (rest > 0) {
      const int64_t nt = (rest + TB - 1) / TB;
      k_chol_update<T><<<unsigned(nt * (nt + 1) / 2), PT, 0, s>>>(A, n, k0, kb, skip);
    }
  }
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
template int chol_factor<double>(double*, int64_t, int*, const int*, cudaStream_t);
template int chol_factor<float>(float*, int64_t, int*, const int*, cudaStream_t);

// ---------------------------------------------------------------------------
// Triangular solves, one launch per block of TS rows.
//   forward : L z = x   (x is consumed: rows below the block are updated)
//   backward: L^T y = x (x is consumed: rows above the block are updated)
// TX is the type of the right-hand side / solution vectors.
// ---------------------------------------------------------------------------
constexpr int TS = 64;
constexpr int TRows = 256;   // rows updated per CTA

template <typename T, typename TX>
__global__ void __launch_bounds__(TS) k_trsv_fwd(const T* L, int64_t n, int64_t k0, TX* x, TX* z,
                                                 const int* skip) {
  if (skip && *skip) return;
  __shared__ T D[TS][TS + 1];
  __shared__ T zk[TS];
  const int tid = threadIdx.x;
  const int kb = int((n - k0) < TS ? (n - k0) : TS);
  for (int e = tid; e < kb * kb; e += TS) {
    const int i = e % kb, l = e / kb;
    D[i][l] = (i >= l) ? L[(k0 + i) + n * (k0 + l)] : T(0);
  }
  if (tid < kb) zk[tid] = T(x[k0 + tid]);
  __syncthreads();
  for (int p = 0; p < kb; ++p) {
    const T zp = zk[p] / D[p][p];
    __syncthreads();
    if (tid == p) zk[p] = zp;
    if (tid > p && tid < kb) zk[tid] -= D[tid][p] * zp;
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    if (tid < kb) z[k0 + tid] = TX(zk[tid]);
    return;
  }
  const int64_t rbeg = k0 + kb + int64_t(blockIdx.x - 1) * TRows;
  for (int64_t r = rbeg + tid; r < rbeg + TRows && r < n; r += TS) {
    T s = T(0);
    for (int l = 0; l < kb; ++l) s = fma(L[r + n * (k0 + l)], zk[l], s);
    x[r] = TX(T(x[r]) - s);
  }
}

template <typename T, typename TX>
__global__ void __launch_bounds__(TS) k_trsv_bwd(const T* L, int64_t n, int64_t k0, TX* x, TX* y,
                                                 const int* skip) {
  if (skip && *skip) return;
  __shared__ T D[TS][TS + 1];
  __shared__ T yk[TS];
  const int tid = threadIdx.x;
  const int kb = int((n - k0) < TS ? (n - k0) : TS);
  for (int e = tid; e < kb * kb; e += TS) {
    const int i = e % kb, l = e / kb;
    D[i][l] = (i >= l) ? L[(k0 + i) + n * (k0 + l)] : T(0);
  }
  if (tid < kb) yk[tid] = T(x[k0 + tid]);
  __syncthreads();
  for (int p = kb - 1; p >= 0; --p) {
    const T yp = yk[p] / D[p][p];
    __syncthreads();
    if (tid == p) yk[p] = yp;
    if (tid < p) yk[tid] -= D[p][tid] * yp;
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    if (tid < kb) y[k0 + tid] = TX(yk[tid]);
    return;
  }
  // rows r < k0: x[r] -= sum_l L[k0 + l, r] y_l
  const int64_t rbeg = int64_t(blockIdx.x - 1) * TRows;
  for (int64_t r = rbeg + tid; r < rbeg + TRows && r < k0; r += TS) {
    T s = T(0);
    for (int l = 0; l < kb; ++l) s = fma(L[(k0 + l) + n * r], yk[l], s);
    x[r] = TX(T(x[r]) - s);
  }
}

// y = (L L^T)^{-1} x; x is destroyed, tmp has length n.
template <typename T, typename TX>
int chol_solve(const T* L, int64_t n, TX* x, TX* tmp, TX* y, const int* skip, cudaStream_t s) {
  for (int64_t k0 = 0; k0 < n; k0 += TS) {
    const int kb = int((n - k0) < TS ? (n - k0) : TS);
    const int64_t rest = n - k0 - kb;
    const int64_t g = 1 + (rest + TRows - 1) / TRows;
    k_trsv_fwd<T, TX><<<unsigned(g), TS, 0, s>>>(L, n, k0, x, tmp, skip);
  }
  const int64_t last = ((n - 1) / TS) * TS;
  for (int64_t k0 = last; k0 >= 0; k0 -= TS) {
    const int64_t g = 1 + (k0 + TRows - 1) / TRows;
    k_trsv_bwd<T, TX><<<unsigned(g), TS, 0, s>>>(L, n, k0, tmp, y, skip);
  }
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
template int chol_solve<double, double>(const double*, int64_t, double*, double*, double*, const int*,
                                        cudaStream_t);
template int chol_solve<float, float>(const float*, int64_t, float*, float*, float*, const int*,
                                      cudaStream_t);

}  // namespace cpdgn
