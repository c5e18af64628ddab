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

// Reciprocal of a pivot.  The float32 inverse only preconditions the float64
// refinement, so the fast intrinsic division (about 2 ulp) is accurate enough.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <typename T>
__device__ void load_tile(const T* A, int64_t n, int ti, int tj, T (*S)[GJL]) {
  constexpr int K = GJB * GJB / GJT;
  T v[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int e = int(threadIdx.x) + q * GJT;
    const int i = e % GJB, j = e / GJB;
    const int64_t r = int64_t(ti) * GJB + i, c = int64_t(tj) * GJB + j;
    v[q] = (r < n && c < n) ? A[r + n * c] : T(0);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int e = int(threadIdx.x) + q * GJT;
    S[e % GJB][e / GJB] = v[q];
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

// Row panel: B[k,j] = P^{-1} A[k,j] for j != k; CTA = tile column j.
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_rowpanel(const T* A, T* B, int64_t n, int k, const T* Pinv,
                                                     const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ps[GJB][GJL], Xs[GJB][GJL];
  const int nt = int((n + GJB - 1) / GJB);
  const int tj = blockIdx.x >= k ? blockIdx.x + 1 : blockIdx.x;
  if (tj >= nt) return;
  load_tile(Pinv, GJB, 0, 0, Ps);
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

// Update of every tile outside row k.  When skip_pivot is set, tile
// (k+1, k+1) is left to k_gj_pivot_next (which runs concurrently).
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_update(const T* A, T* B, int64_t n, int k, const T* Pinv,
                                                   int skip_pivot, const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ls[GJB][GJL], Rs[GJB][GJL];
  const int nt = int((n + GJB - 1) / GJB);
  const int b = int(blockIdx.x);
  const int ti = b % (nt - 1) >= k ? b % (nt - 1) + 1 : b % (nt - 1);
  const int tj = b / (nt - 1);
  if (skip_pivot && ti == k + 1 && tj == k + 1) return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  load_tile(A, n, ti, k, Ls);                        // A[i,k]
  if (tj == k) {
    load_tile(Pinv, GJB, 0, 0, Rs);
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
    T a[4], bb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = Ls[tx + 16 * u][l];
#pragma unroll
    for (int v = 0; v < 4; ++v) bb[v] = Rs[l][ty + 16 * v];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(-a[u], bb[v], acc[u][v]);
  }
  store_regs(acc, B, n, ti, tj);
}

// The first kb0 tiles of the core lie inside its leading identity block
// (the core's diagonal R^2 x R^2 blocks are I).  Eliminating them at once
// (pivot I of size kb0 * GJB) maps A -> B as
//     B[0:,0:] = I, B[0:, j] = A[0:, j], B[i, 0:] = -A[i, 0:],
//     B[i, j] = A[i, j] - A[i, 0:] A[0:, j]      (tiles i, j >= kb0)
// which replaces kb0 sweeps by one launch.  CTA = one output tile.
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_identity(const T* A, T* B, int64_t n, int kb0, const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ls[GJB][GJL], Rs[GJB][GJL];
  const int nt = int((n + GJB - 1) / GJB);
  const int ti = blockIdx.x % nt, tj = blockIdx.x / nt;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
  if (ti < kb0 || tj < kb0) {
    const T sgn = (ti >= kb0) ? T(-1) : T(1);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int64_t r = int64_t(ti) * GJB + tx + 16 * u, c = int64_t(tj) * GJB + ty + 16 * v;
        if (ti < kb0 && tj < kb0) acc[u][v] = (r == c) ? T(1) : T(0);
        else acc[u][v] = (r < n && c < n) ? sgn * A[r + n * c] : T(0);
      }
    store_regs(acc, B, n, ti, tj);
    return;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t r = int64_t(ti) * GJB + tx + 16 * u, c = int64_t(tj) * GJB + ty + 16 * v;
      acc[u][v] = (r < n && c < n) ? A[r + n * c] : T(0);
    }
  for (int kk = 0; kk < kb0; ++kk) {
    __syncthreads();
    load_tile(A, n, ti, kk, Ls);
    load_tile(A, n, kk, tj, Rs);
    __syncthreads();
    for (int l = 0; l < GJB; ++l) {
      T a[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ls[tx + 16 * u][l];
#pragma unroll
      for (int v = 0; v < 4; ++v) bb[v] = Rs[l][ty + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(-a[u], bb[v], acc[u][v]);
    }
  }
  store_regs(acc, B, n, ti, tj);
}

// ---------------------------------------------------------------------------
// The pivot chain is the sequential part of the inversion, so each pivot is
// inverted by one 1024-thread CTA (32 x 32 threads, a 2 x 2 register block
// each: ~20 instructions and 8 resident warps per scheduler per elimination
// step).  For sweep k + 1 the same CTA first forms its pivot tile
// X = A[k+1,k+1] - A[k+1,k] B[k,k+1] (B[k,:] is sweep k's row panel), so it
// can run concurrently with sweep k's update of every other tile.
// ---------------------------------------------------------------------------
constexpr int PVT = 1024;

template <typename T>
__device__ void gj_invert_2x2(T (&x)[2][2], int kb, T (*prow)[GJB], T (*pcol)[GJB], int* bad) {
  __shared__ T pv[GJB];                                          // pivots, checked at the end
  const int tid = threadIdx.x, bi = tid % 32, bj = tid / 32;   // rows 2 bi + u, cols 2 bj + v
#pragma unroll 2
  for (int p = 0; p < kb; ++p) {
    const int par = p & 1;
    const int hp = p >> 1, lp = p & 1;
    if (bi == hp) {
      prow[par][2 * bj] = lp ? x[1][0] : x[0][0];
      prow[par][2 * bj + 1] = lp ? x[1][1] : x[0][1];
    }
    if (bj == hp) {
      pcol[par][2 * bi] = lp ? x[0][1] : x[0][0];
      pcol[par][2 * bi + 1] = lp ? x[1][1] : x[1][0];
    }
    __syncthreads();
    const T piv = prow[par][p];
    if (tid == 0) pv[p] = piv;
    const T dinv = recip(piv);
    const T c0 = pcol[par][2 * bi], c1 = pcol[par][2 * bi + 1];
    const T r0 = prow[par][2 * bj] * dinv, r1 = prow[par][2 * bj + 1] * dinv;
    x[0][0] = fma(-c0, r0, x[0][0]);
    x[0][1] = fma(-c0, r1, x[0][1]);
    x[1][0] = fma(-c1, r0, x[1][0]);
    x[1][1] = fma(-c1, r1, x[1][1]);
    if (bi == hp) {                  // row p -> scaled pivot row
      if (lp) { x[1][0] = r0; x[1][1] = r1; }
      else { x[0][0] = r0; x[0][1] = r1; }
    }
    if (bj == hp) {                  // column p -> -col / piv; the pivot itself -> 1 / piv
      if (lp) {
        x[0][1] = -c0 * dinv;
        x[1][1] = (bi == hp) ? dinv : -c1 * dinv;
      } else {
        x[0][0] = (bi == hp) ? dinv : -c0 * dinv;
        x[1][0] = -c1 * dinv;
      }
    }
  }
  // check the recorded pivots once, after the elimination
  __syncthreads();
  if (tid < kb && !(pv[tid] > T(0) && isfinite(pv[tid]))) atomicMin(bad, tid + 1);
  __syncthreads();
}

// Tile (ti, tj) of A as 2 x 2 register blocks (identity beyond kb).
template <typename T>
__device__ void load_2x2(const T* A, int64_t n, int ti, int tj, int kb, T (&x)[2][2]) {
  const int bi = threadIdx.x % 32, bj = threadIdx.x / 32;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = 2 * bi + u, j = 2 * bj + v;
      const int64_t r = int64_t(ti) * GJB + i, c = int64_t(tj) * GJB + j;
      x[u][v] = (i < kb && j < kb) ? A[r + n * c] : (i == j ? T(1) : T(0));
    }
}

// Invert x (pivot tile kk) and write P^{-1} to Pinv and into tile (kk, kk) of D.
template <typename T>
__device__ void pivot_store(T (&x)[2][2], int64_t n, int kk, int kb, T* Pinv, T* D, int* info,
                            T (*prow)[GJB], T (*pcol)[GJB], int* bad) {
  const int bi = threadIdx.x % 32, bj = threadIdx.x / 32;
  if (threadIdx.x == 0) *bad = GJB + 1;
  __syncthreads();
  gj_invert_2x2<T>(x, kb, prow, pcol, bad);
  if (threadIdx.x == 0 && *bad <= GJB && info) atomicCAS(info, 0, kk * GJB + *bad);
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = 2 * bi + u, j = 2 * bj + v;
      Pinv[i + GJB * j] = x[u][v];
      if (i < kb && j < kb) D[(int64_t(kk) * GJB + i) + n * (int64_t(kk) * GJB + j)] = x[u][v];
    }
}

// Pivot of sweep k (tile (k, k) of A as it stands); P^{-1} also into D's tile.
template <typename T>
__global__ void __launch_bounds__(PVT) k_gj_pivot(const T* A, T* D, int64_t n, int k, T* Pinv, int* info,
                                                  const int* skip) {
  if (skip && *skip) return;
  __shared__ T prow[2][GJB], pcol[2][GJB];
  __shared__ int bad;
  const int kb = int((n - int64_t(k) * GJB) < GJB ? (n - int64_t(k) * GJB) : GJB);
  T x[2][2];
  load_2x2(A, n, k, k, kb, x);
  pivot_store<T>(x, n, k, kb, Pinv, D, info, prow, pcol, &bad);
}

// Pivot of sweep k + 1 during sweep k: X = A[k+1,k+1] - A[k+1,k] B[k,k+1],
// inverted; P^{-1} goes to Pinv_next and into A's tile (k+1, k+1), which sweep
// k + 1 writes into and which nobody else reads during sweep k.
template <typename T>
__global__ void __launch_bounds__(PVT) k_gj_pivot_next(T* A, const T* B, int64_t n, int k, T* Pinv_next,
                                                       int* info, const int* skip) {
  if (skip && *skip) return;
  __shared__ T Ls[GJB][GJL], Rs[GJB][GJL];
  __shared__ T prow[2][GJB], pcol[2][GJB];
  __shared__ int bad;
  const int k1 = k + 1;
  const int kb = int((n - int64_t(k1) * GJB) < GJB ? (n - int64_t(k1) * GJB) : GJB);
  for (int e = threadIdx.x; e < GJB * GJB; e += PVT) {
    const int i = e % GJB, j = e / GJB;
    const int64_t r = int64_t(k1) * GJB + i, c = int64_t(k) * GJB + j, rr = int64_t(k) * GJB + i,
                  cc = int64_t(k1) * GJB + j;
    Ls[i][j] = (r < n) ? A[r + n * c] : T(0);          // A[k+1, k]
    Rs[i][j] = (cc < n) ? B[rr + n * cc] : T(0);       // B[k, k+1]
  }
  T x[2][2];
  load_2x2(A, n, k1, k1, kb, x);
  __syncthreads();
  const int bi = threadIdx.x % 32, bj = threadIdx.x / 32;
#pragma unroll 8
  for (int l = 0; l < GJB; ++l) {
    const T a0 = Ls[2 * bi][l], a1 = Ls[2 * bi + 1][l];
    const T b0 = Rs[l][2 * bj], b1 = Rs[l][2 * bj + 1];
    x[0][0] = fma(-a0, b0, x[0][0]);
    x[0][1] = fma(-a0, b1, x[0][1]);
    x[1][0] = fma(-a1, b0, x[1][0]);
    x[1][1] = fma(-a1, b1, x[1][1]);
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v)
      if (2 * bi + u >= kb || 2 * bj + v >= kb) x[u][v] = (2 * bi + u == 2 * bj + v) ? T(1) : T(0);
  pivot_store<T>(x, n, k1, kb, Pinv_next, A, info, prow, pcol, &bad);
}

// Invert the n x n SPD matrix A (full storage, column-major); B is the second
// buffer and pinv holds 2 GJB x GJB blocks.  *result receives the buffer with
// the inverse.  When the leading `ident` rows/columns of A are the identity,
// the first ident / GJB sweeps are replaced by one block elimination.  With
// side != null the pivot of sweep k + 1 is inverted on `side` while sweep k's
// update runs on s (fork/join through ev_fork / ev_join, graph-capturable).
template <typename T>
int gj_invert(T* A, T* B, T* pinv, int64_t n, int64_t ident, int* info, const int* skip, cudaStream_t s,
              cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join, T** result) {
  const int nt = int((n + GJB - 1) / GJB);
  T* src = A;
  T* dst = B;
  int k0 = int(ident / GJB);
  if (k0 >= nt) k0 = nt - 1;
  if (k0 > 0) {
    k_gj_identity<T><<<nt * nt, GJT, 0, s>>>(src, dst, n, k0, skip);
    T* t = src;
    src = dst;
    dst = t;
  }
  k_gj_pivot<T><<<1, PVT, 0, s>>>(src, dst, n, k0, pinv + size_t(k0 & 1) * GJB * GJB, info, skip);
  for (int k = k0; k < nt; ++k) {
    T* pk = pinv + size_t(k & 1) * GJB * GJB;
    T* pn = pinv + size_t((k + 1) & 1) * GJB * GJB;
    if (nt > 1) {
      k_gj_rowpanel<T><<<nt - 1, GJT, 0, s>>>(src, dst, n, k, pk, skip);
      const bool next = (k + 1 < nt);
      if (next && side) {
        if (cudaEventRecord(ev_fork, s) != cudaSuccess) return CP_ECUDA;
        if (cudaStreamWaitEvent(side, ev_fork, 0) != cudaSuccess) return CP_ECUDA;
        k_gj_pivot_next<T><<<1, PVT, 0, side>>>(src, dst, n, k, pn, info, skip);
        if (cudaEventRecord(ev_join, side) != cudaSuccess) return CP_ECUDA;
      }
      k_gj_update<T><<<(nt - 1) * nt, GJT, 0, s>>>(src, dst, n, k, pk, (next && side) ? 1 : 0, skip);
      if (next && side) {
        if (cudaStreamWaitEvent(s, ev_join, 0) != cudaSuccess) return CP_ECUDA;
      } else if (next) {
        k_gj_pivot<T><<<1, PVT, 0, s>>>(dst, src, n, k + 1, pn, info, skip);
      }
    }
    T* t = src;
    src = dst;
    dst = t;
  }
  *result = src;
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
template int gj_invert<float>(float*, float*, float*, int64_t, int64_t, int*, const int*, cudaStream_t,
                               cudaStream_t, cudaEvent_t, cudaEvent_t, float**);

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
