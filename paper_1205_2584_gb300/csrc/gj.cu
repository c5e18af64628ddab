// Blocked Gauss-Jordan inversion of the symmetric positive definite core
// system (float32 in the mixed mode), and the accumulate-GEMV used by the
// float64 iterative refinement.
//
// With pivot block P = A[k,k] of panel k (width GJB), one sweep maps A -> B:
//     B[k,k] = P^{-1}
//     B[k,j] = P^{-1} A[k,j]                (j != k)      k_gj_rowpanel
//     B[i,k] = -A[i,k] P^{-1}               (i != k)      k_gj_update
//     B[i,j] = A[i,j] - A[i,k] B[k,j]       (i, j != k)   k_gj_update
// and after the last panel B = A^{-1}.  No pivoting is needed for an SPD
// matrix (each pivot block is a Schur complement of an SPD matrix).  P^{-1}
// is computed once per sweep by one CTA that keeps the block in registers;
// for sweeps after the first, the CTA of k_gj_update that produces the next
// pivot tile inverts it before it exits.  A and B alternate between sweeps.
// A non-positive or non-finite pivot sets *info (1-based row); nothing traps.
#include "common.cuh"

namespace cpdgn {

constexpr int GJB = 64;           // panel / tile width
constexpr int GJT = 256;          // threads per CTA: a 16 x 16 grid of 4 x 4 blocks
constexpr int GJL = GJB + 1;      // padded leading dimension in shared memory

// Gauss-Jordan inversion (no pivoting) of the kb x kb block held as 4 x 4
// register blocks: thread (tx, ty) owns rows tx + 16 u and columns ty + 16 v
// (u, v < 4).  Rows/columns >= kb must hold the identity.  One barrier per
// elimination step; the pivot row and column go through shared memory,
// double-buffered by step parity.
template <typename T>
__device__ void gj_invert_regs(T (&x)[4][4], int kb, T (*prow)[GJB], T (*pcol)[GJB], int* bad) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  for (int p = 0; p < kb; ++p) {
    const int par = p & 1;
    // publish the current row p and column p
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (tx + 16 * u == p) {
#pragma unroll
        for (int v = 0; v < 4; ++v) prow[par][ty + 16 * v] = x[u][v];
      }
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (ty + 16 * v == p) {
#pragma unroll
        for (int u = 0; u < 4; ++u) pcol[par][tx + 16 * u] = x[u][v];
      }
    __syncthreads();
    const T piv = prow[par][p];
    if (tid == 0 && !(piv > T(0) && isfinite(double(piv))) && *bad == 0) *bad = p + 1;
    const T d = T(1) / piv;
    T cu[4], rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) cu[u] = pcol[par][tx + 16 * u];
#pragma unroll
    for (int v = 0; v < 4; ++v) rv[v] = prow[par][ty + 16 * v] * d;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ip = (tx + 16 * u == p);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const bool jp = (ty + 16 * v == p);
        const T upd = fma(-cu[u], rv[v], x[u][v]);
        x[u][v] = ip ? (jp ? d : rv[v]) : (jp ? -cu[u] * d : upd);
      }
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void load_tile(const T* A, int64_t n, int ti, int tj, T (*S)[GJL]) {
  for (int e = threadIdx.x; e < GJB * GJB; e += GJT) {
    const int i = e % GJB, j = e / GJB;
    const int64_t r = int64_t(ti) * GJB + i, c = int64_t(tj) * GJB + j;
    S[i][j] = (r < n && c < n) ? A[r + n * c] : T(0);
  }
}

template <typename T>
__device__ void store_regs(const T (&x)[4][4], T* B, int64_t n, int ti, int tj) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t r = int64_t(ti) * GJB + tx + 16 * u, c = int64_t(tj) * GJB + ty + 16 * v;
      if (r < n && c < n) B[r + n * c] = x[u][v];
    }
}

// Invert the pivot tile (kk, kk) of Bsrc (already in registers as x) and write
// P^{-1} to Pinv (GJB x GJB, column-major) and into tile (kk, kk) of Bdst.
template <typename T>
__device__ void pivot_from_regs(T (&x)[4][4], int64_t n, int kk, T* Pinv, T* Bdst, int* info,
                                T (*prow)[GJB], T (*pcol)[GJB], int* bad) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int kb = int((n - int64_t(kk) * GJB) < GJB ? (n - int64_t(kk) * GJB) : GJB);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = tx + 16 * u, j = ty + 16 * v;
      if (i >= kb || j >= kb) x[u][v] = (i == j) ? T(1) : T(0);
    }
  if (threadIdx.x == 0) *bad = 0;
  __syncthreads();
  gj_invert_regs<T>(x, kb, prow, pcol, bad);
  if (threadIdx.x == 0 && *bad && info) atomicCAS(info, 0, kk * GJB + *bad);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) Pinv[(tx + 16 * u) + GJB * (ty + 16 * v)] = x[u][v];
  store_regs(x, Bdst, n, kk, kk);
}

// First pivot: one CTA.
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_pivot0(const T* A, T* B, int64_t n, T* Pinv, int* info,
                                                   const int* skip) {
  if (skip && *skip) return;
  __shared__ T prow[2][GJB], pcol[2][GJB];
  __shared__ int bad;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T x[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t r = tx + 16 * u, c = ty + 16 * v;
      x[u][v] = (r < n && c < n) ? A[r + n * c] : T(0);
    }
  pivot_from_regs<T>(x, n, 0, Pinv, B, info, prow, pcol, &bad);
}

// Row panel: B[k,j] = P^{-1} A[k,j] for j != k; CTA = tile column j.
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_rowpanel(const T* A, T* B, int64_t n, int k, const T* Pinv,
                                                     const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ps[GJB][GJL], Xs[GJB][GJL];
  const int nt = int((n + GJB - 1) / GJB);
  const int tj = blockIdx.x >= k ? blockIdx.x + 1 : blockIdx.x;
  if (tj >= nt) return;
  for (int e = threadIdx.x; e < GJB * GJB; e += GJT) Ps[e % GJB][e / GJB] = Pinv[e];
  load_tile(A, n, k, tj, Xs);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int l = 0; l < GJB; ++l) {
    T a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = Ps[tx + 16 * u][l];
#pragma unroll
    for (int v = 0; v < 4; ++v) b[v] = Xs[l][ty + 16 * v];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
  store_regs(acc, B, n, k, tj);
}

// Update of every tile outside row k; the CTA of tile (k+1, k+1) then inverts
// it as the next pivot.
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_update(const T* A, T* B, int64_t n, int k, const T* Pinv,
                                                   T* Pinv_next, int* info, const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ls[GJB][GJL], Rs[GJB][GJL];
  __shared__ T prow[2][GJB], pcol[2][GJB];
  __shared__ int bad;
  const int nt = int((n + GJB - 1) / GJB);
  const int ti = blockIdx.x % (nt - 1) >= k ? blockIdx.x % (nt - 1) + 1 : blockIdx.x % (nt - 1);
  const int tj = blockIdx.x / (nt - 1);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  load_tile(A, n, ti, k, Ls);                        // A[i,k]
  if (tj == k) {
    for (int e = threadIdx.x; e < GJB * GJB; e += GJT) Rs[e % GJB][e / GJB] = Pinv[e];
  } else {
    load_tile(B, n, k, tj, Rs);                      // B[k,j] from the row panel
  }
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t r = int64_t(ti) * GJB + tx + 16 * u, c = int64_t(tj) * GJB + ty + 16 * v;
      acc[u][v] = (tj == k || r >= n || c >= n) ? T(0) : A[r + n * c];
    }
  __syncthreads();
  for (int l = 0; l < GJB; ++l) {
    T a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = Ls[tx + 16 * u][l];
#pragma unroll
    for (int v = 0; v < 4; ++v) b[v] = Rs[l][ty + 16 * v];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(-a[u], b[v], acc[u][v]);
  }
  if (Pinv_next && ti == k + 1 && tj == k + 1) {
    // the next sweep writes into this sweep's source buffer: its pivot tile
    // (k+1, k+1) is read by this CTA only, so P^{-1} goes there
    pivot_from_regs<T>(acc, n, k + 1, Pinv_next, const_cast<T*>(A), info, prow, pcol, &bad);
    return;
  }
  store_regs(acc, B, n, ti, tj);
}

// Invert the n x n SPD matrix A (full storage, column-major); B is the second
// buffer and pinv holds 2 GJB x GJB blocks.  *result receives the buffer
// with the inverse.
template <typename T>
int gj_invert(T* A, T* B, T* pinv, int64_t n, int* info, const int* skip, cudaStream_t s, T** result) {
  const int nt = int((n + GJB - 1) / GJB);
  T* src = A;
  T* dst = B;
  k_gj_pivot0<T><<<1, GJT, 0, s>>>(src, dst, n, pinv, info, skip);
  for (int k = 0; k < nt; ++k) {
    T* pk = pinv + size_t(k & 1) * GJB * GJB;
    T* pn = pinv + size_t((k + 1) & 1) * GJB * GJB;
    if (nt > 1) {
      k_gj_rowpanel<T><<<nt - 1, GJT, 0, s>>>(src, dst, n, k, pk, skip);
      k_gj_update<T><<<(nt - 1) * nt, GJT, 0, s>>>(src, dst, n, k, pk, (k + 1 < nt) ? pn : nullptr, info,
                                                    skip);
    }
    T* t = src;
    src = dst;
    dst = t;
  }
  *result = src;
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
template int gj_invert<float>(float*, float*, float*, int64_t, int*, const int*, cudaStream_t, float**);

// y += X r  (X n x n float32 column-major, r and y float64).  CTA = (row block,
// column slice); partial sums of the slice are added with atomics.  When b2
// and r2 are given the sweep first checks convergence of the refinement:
// with ||b||^2 = *b2, ||r||^2 = *r2 and the previous sweep's *r2prev, it sets
// *done and returns if ||r||^2 <= tol2 ||b||^2 or the residual stopped
// shrinking (||r||^2 > ||r_prev||^2 / 16).
constexpr int GVT = 256;
constexpr int GVS = 64;     // columns per slice

__global__ void __launch_bounds__(GVT) k_gemv_acc(const float* X, int64_t n, const double* r, double* y,
                                                  const double* b2, const double* r2, const double* r2prev,
                                                  int* done, double tol2, const int* skip) {
  if (skip && *skip) return;
  if (b2 && r2) {
    const double vb = *b2, vr = *r2, vp = r2prev ? *r2prev : 0.0;
    const bool conv = (vr <= tol2 * vb) || (vp > 0.0 && vr > 0.0625 * vp);
    if (conv) {
      if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *done = 1;
      return;
    }
  }
  __shared__ float rs[GVS];
  const int64_t row = int64_t(blockIdx.x) * GVT + threadIdx.x;
  const int64_t c0 = int64_t(blockIdx.y) * GVS;
  const int nc = int((n - c0) < GVS ? (n - c0) : GVS);
  if (threadIdx.x < nc) rs[threadIdx.x] = float(r[c0 + threadIdx.x]);
  __syncthreads();
  if (row >= n) return;
  const float* x = X + row + n * c0;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  int c = 0;
  for (; c + 3 < nc; c += 4) {
    s0 = fmaf(x[n * c], rs[c], s0);
    s1 = fmaf(x[n * (c + 1)], rs[c + 1], s1);
    s2 = fmaf(x[n * (c + 2)], rs[c + 2], s2);
    s3 = fmaf(x[n * (c + 3)], rs[c + 3], s3);
  }
  for (; c < nc; ++c) s0 = fmaf(x[n * c], rs[c], s0);
  atomicAdd(y + row, double((s0 + s1) + (s2 + s3)));
}

int launch_gemv_acc(const float* X, int64_t n, const double* r, double* y, const double* b2, const double* r2,
                    const double* r2prev, int* done, double tol2, const int* skip, cudaStream_t s) {
  dim3 g(unsigned((n + GVT - 1) / GVT), unsigned((n + GVS - 1) / GVS));
  k_gemv_acc<<<g, GVT, 0, s>>>(X, n, r, y, b2, r2, r2prev, done, tol2, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn
