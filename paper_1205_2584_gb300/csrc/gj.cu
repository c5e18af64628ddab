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
// matrix (each pivot block is a Schur complement of an SPD matrix).  A and B
// alternate between sweeps.  A non-positive or non-finite pivot sets *info
// (1-based row); nothing traps.
//
// The sequential part is the chain of pivot inverses.  P^{-1} of sweep k + 1
// is formed and inverted during sweep k from sweep k's input alone, so it
// overlaps sweep k's row panel and update: by one CTA (k_gj_pivot_next) on a
// side stream that reserves nearly all of its SM's shared memory (so no tile
// CTA shares the SM with it), or, on the tensor-core path while the grid fits
// on the GPU, by CTA 0 of the sweep's single launch (k_gj_sweep_tc), whose
// other CTAs form their slices of the row panel themselves.  The kernels by
// path (n = N R^2):
//   n % 4 != 0 or n < 1024: k_gj_identity, k_gj_pivot, then per sweep
//     k_gj_pivot_next (side stream), k_gj_rowpanel, k_gj_update;
//   1024 <= n, 1 + ceil(n / 128)^2 CTAs fit: k_gj_identity + k_gj_update_tc
//     (identity block) with k_gj_pivot_ident (side stream), then one
//     k_gj_sweep_tc per sweep;
//   larger n: k_gj_identity + k_gj_update_tc, k_gj_pivot, then per sweep
//     k_gj_pivot_next (side stream), k_gj_rowpanel, k_gj_update2_tc.
//
// Tile products.  The pivot kernels (128 threads on a 64 x 64 tile): thread
// (bi, bj) owns rows 4 bi .. 4 bi + 3 and columns 8 bj .. 8 bj + 7, so each
// k-step reads one float4 of the left operand (stored column by column, rows
// contiguous) and two float4 of the right operand (stored row by row) for 32
// multiply-adds.  The row panel, the update and the identity elimination work
// on 64 x 32 half tiles (twice as many CTAs as tiles, which spreads a sweep
// evenly over the SMs) with 64 threads: thread (bi, bj) owns rows
// 4 bi .. 4 bi + 3 and 32 + 4 bi .. 32 + 4 bi + 3 and columns 4 bj .. 4 bj + 3,
// so each k-step reads two float4 of the left operand and one of the right
// operand for 32 multiply-adds; eight consecutive lanes read eight
// consecutive float4, free of shared-memory bank conflicts.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace cpdgn {

constexpr int GJB = 64;           // panel / tile height
constexpr int GJT = 128;          // threads of a 64 x 64 tile CTA: 16 x 8 threads, 4 x 8 entries each
constexpr int GJH = 32;           // width of a half tile
constexpr int GJTH = 64;          // threads of a 64 x 32 half-tile CTA: 8 x 8 threads, 8 x 4 entries each
constexpr int GJP = GJB + 4;      // padded row length in shared memory (keeps float4 alignment)
// shared memory reserved by k_gj_pivot_next on top of its static arrays
// (56 KB): with it the CTA holds 224 KB of the SM's 228 KB, so no half-tile
// CTA (about 27 KB) fits beside it; the sum stays under the 227 KB per-block
// limit
constexpr int kPivotReserve = 168 * 1024;

// Reciprocal of a pivot.  The float32 inverse only preconditions the float64
// refinement, so the fast intrinsic division (about 2 ulp) is accurate enough.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }


// S[c][r] = sgn * A(r0 + r, c0 + c) for r, c < 64 (zero outside n x n): a
// 64 x 64 left operand stored column by column.  Global reads are coalesced
// along r.  NT threads.
template <int NT>
__device__ __forceinline__ void load_cols(const float* A, int64_t n, int64_t r0, int64_t c0, float (*S)[GJP],
                                          float sgn) {
#pragma unroll
  for (int q = 0; q < GJB * GJB / NT; ++q) {
    const int e = int(threadIdx.x) + q * NT;
    const int r = e % GJB, c = e / GJB;
    const int64_t gr = r0 + r, gc = c0 + c;
    S[c][r] = (gr < n && gc < n) ? sgn * A[gr + n * gc] : 0.f;
  }
}

// the thread's 4 x 8 block of the 64 x 64 tile at (r0, c0); entries outside n x n read as 0
__device__ __forceinline__ void load_block(const float* A, int64_t n, int64_t r0, int64_t c0, float (&x)[4][8]) {
  const int bi = threadIdx.x % 16, bj = threadIdx.x / 16;
  const int64_t rr = r0 + 4 * bi;
  const bool vec = (n % 4 == 0) && (rr + 3 < n);
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int64_t c = c0 + 8 * bj + v;
    if (c >= n) {
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u][v] = 0.f;
    } else if (vec) {
      const float4 t = *reinterpret_cast<const float4*>(A + rr + n * c);
      x[0][v] = t.x;
      x[1][v] = t.y;
      x[2][v] = t.z;
      x[3][v] = t.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u][v] = (rr + u < n) ? A[rr + u + n * c] : 0.f;
    }
  }
}

__device__ __forceinline__ void store_block(const float (&x)[4][8], float* B, int64_t n, int64_t r0, int64_t c0) {
  const int bi = threadIdx.x % 16, bj = threadIdx.x / 16;
  const int64_t rr = r0 + 4 * bi;
  const bool vec = (n % 4 == 0) && (rr + 3 < n);
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int64_t c = c0 + 8 * bj + v;
    if (c >= n) continue;
    if (vec) {
      *reinterpret_cast<float4*>(B + rr + n * c) = make_float4(x[0][v], x[1][v], x[2][v], x[3][v]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (rr + u < n) B[rr + u + n * c] = x[u][v];
    }
  }
}

__device__ __forceinline__ void zero_block(float (&x)[4][8]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) x[u][v] = 0.f;
}

// ---- half-tile kernels (64 threads, 8 x 4 entries per thread) ----

// Ls[l][r] = sgn * A(r0 + r, c0 + l) for r, l < 64 (zero outside n x n).
// With n % 4 == 0 the reads are float4 along r (tile origins are multiples of
// 64, so they are 16-byte aligned).
__device__ __forceinline__ void h_load_left(const float* A, int64_t n, int64_t r0, int64_t c0, float (*Ls)[GJP],
                                            float sgn) {
  if (n % 4 == 0) {
#pragma unroll 4
    for (int q = 0; q < GJB * GJB / 4 / GJTH; ++q) {
      const int e = int(threadIdx.x) + q * GJTH;
      const int r = 4 * (e % 16), l = e / 16;
      const int64_t gr = r0 + r, gc = c0 + l;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < n && gc < n) v = *reinterpret_cast<const float4*>(A + gr + n * gc);
      *reinterpret_cast<float4*>(&Ls[l][r]) = make_float4(sgn * v.x, sgn * v.y, sgn * v.z, sgn * v.w);
    }
  } else {
#pragma unroll 4
    for (int q = 0; q < GJB * GJB / GJTH; ++q) {
      const int e = int(threadIdx.x) + q * GJTH;
      const int r = e % GJB, l = e / GJB;
      const int64_t gr = r0 + r, gc = c0 + l;
      Ls[l][r] = (gr < n && gc < n) ? sgn * A[gr + n * gc] : 0.f;
    }
  }
}

// Rs[l][c] = A(r0 + l, c0 + c) for l < 64, c < 32.  With n % 4 == 0 each
// thread reads a float4 along l and scatters it over 4 rows (consecutive
// lanes take consecutive columns: no bank conflicts).
__device__ __forceinline__ void h_load_right(const float* A, int64_t n, int64_t r0, int64_t c0,
                                             float (*Rs)[GJH + 4]) {
  if (n % 4 == 0) {
#pragma unroll 4
    for (int q = 0; q < GJB * GJH / 4 / GJTH; ++q) {
      const int e = int(threadIdx.x) + q * GJTH;
      const int c = e % GJH, l = 4 * (e / GJH);
      const int64_t gr = r0 + l, gc = c0 + c;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < n && gc < n) v = *reinterpret_cast<const float4*>(A + gr + n * gc);
      Rs[l][c] = v.x;
      Rs[l + 1][c] = v.y;
      Rs[l + 2][c] = v.z;
      Rs[l + 3][c] = v.w;
    }
  } else {
#pragma unroll 4
    for (int q = 0; q < GJB * GJH / GJTH; ++q) {
      const int e = int(threadIdx.x) + q * GJTH;
      const int c = e % GJH, l = e / GJH;
      const int64_t gr = r0 + l, gc = c0 + c;
      Rs[l][c] = (gr < n && gc < n) ? A[gr + n * gc] : 0.f;
    }
  }
}

// row of entry (u, .) of thread bi: u < 4 -> 4 bi + u, u >= 4 -> 32 + 4 bi + u - 4
__device__ __forceinline__ int h_row(int bi, int hh) { return 4 * bi + 32 * hh; }

__device__ __forceinline__ void h_load_block(const float* A, int64_t n, int64_t r0, int64_t c0, float (&x)[8][4]) {
  const int bi = threadIdx.x % 8, bj = threadIdx.x / 8;
  const bool vec = (n % 4 == 0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int64_t c = c0 + 4 * bj + v;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int64_t r = r0 + h_row(bi, hh);
      if (vec) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < n && r < n) t = *reinterpret_cast<const float4*>(A + r + n * c);
        x[4 * hh][v] = t.x;
        x[4 * hh + 1][v] = t.y;
        x[4 * hh + 2][v] = t.z;
        x[4 * hh + 3][v] = t.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) x[4 * hh + u][v] = (c < n && r + u < n) ? A[r + u + n * c] : 0.f;
      }
    }
  }
}

__device__ __forceinline__ void h_store_block(const float (&x)[8][4], float* B, int64_t n, int64_t r0, int64_t c0) {
  const int bi = threadIdx.x % 8, bj = threadIdx.x / 8;
  const bool vec = (n % 4 == 0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int64_t c = c0 + 4 * bj + v;
    if (c >= n) continue;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int64_t r = r0 + h_row(bi, hh);
      if (vec) {
        if (r < n)
          *reinterpret_cast<float4*>(B + r + n * c) =
              make_float4(x[4 * hh][v], x[4 * hh + 1][v], x[4 * hh + 2][v], x[4 * hh + 3][v]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (r + u < n) B[r + u + n * c] = x[4 * hh + u][v];
      }
    }
  }
}

__device__ __forceinline__ void h_zero(float (&x)[8][4]) {
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) x[u][v] = 0.f;
}

// x += L R with L = Ls (64 x 64, k-major) and R = Rs (64 x 32, k-major).
__device__ __forceinline__ void h_fma(const float (*Ls)[GJP], const float (*Rs)[GJH + 4], float (&x)[8][4]) {
  const int bi = threadIdx.x % 8, bj = threadIdx.x / 8;
#pragma unroll 8
  for (int l = 0; l < GJB; ++l) {
    const float4 a0 = *reinterpret_cast<const float4*>(&Ls[l][4 * bi]);
    const float4 a1 = *reinterpret_cast<const float4*>(&Ls[l][32 + 4 * bi]);
    const float4 b = *reinterpret_cast<const float4*>(&Rs[l][4 * bj]);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) x[u][v] = fmaf(av[u], bv[v], x[u][v]);
  }
}

// ---- asynchronous operand copies (n % 4 == 0) ----

// 16-byte global -> shared copy that bypasses registers; when !pred the
// destination is zero-filled and nothing is read.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Ls[l][r] = A(r0 + r, c0 + l) and Rc[c][l] = A(k0 + l, c1 + c) (both copied
// column by column, rows contiguous), r, l < 64, c < 32; 64 threads.
__device__ __forceinline__ void h_copy_operands(const float* A, int64_t n, int64_t r0, int64_t c0, int64_t k0,
                                                int64_t c1, float (*Ls)[GJP], float (*Rc)[GJP]) {
#pragma unroll 4
  for (int q = 0; q < GJB * GJB / 4 / GJTH; ++q) {
    const int e = int(threadIdx.x) + q * GJTH;
    const int r = 4 * (e % 16), l = e / 16;
    const int64_t gr = r0 + r, gc = c0 + l;
    const bool in = gr < n && gc < n;
    cp_async16(&Ls[l][r], in ? A + gr + n * gc : A, in);
  }
#pragma unroll 4
  for (int q = 0; q < GJB * GJH / 4 / GJTH; ++q) {
    const int e = int(threadIdx.x) + q * GJTH;
    const int l = 4 * (e % 16), c = e / 16;
    const int64_t gr = k0 + l, gc = c1 + c;
    const bool in = gr < n && gc < n;
    cp_async16(&Rc[c][l], in ? A + gr + n * gc : A, in);
  }
}

// x += SGN L R with L = Ls (64 x 64, k-major) and R stored by columns in Rc
// (Rc[c][l] = R[l][c]); four k-steps per float4 of R.
template <int SGN>
__device__ __forceinline__ void h_fma_rc(const float (*Ls)[GJP], const float (*Rc)[GJP], float (&x)[8][4]) {
  const int bi = threadIdx.x % 8, bj = threadIdx.x / 8;
#pragma unroll 2
  for (int l4 = 0; l4 < GJB; l4 += 4) {
    float rv[4][4];                  // rv[v][dl] = R[l4 + dl][4 bj + v]
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float4 t = *reinterpret_cast<const float4*>(&Rc[4 * bj + v][l4]);
      rv[v][0] = t.x;
      rv[v][1] = t.y;
      rv[v][2] = t.z;
      rv[v][3] = t.w;
    }
#pragma unroll
    for (int dl = 0; dl < 4; ++dl) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Ls[l4 + dl][4 * bi]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Ls[l4 + dl][32 + 4 * bi]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) x[u][v] = fmaf(SGN > 0 ? av[u] : -av[u], rv[v][dl], x[u][v]);
    }
  }
}

// Row panel: B[k,j] = P^{-1} A[k,j] for j != k; CTA = one half tile of row k.
// ASYNC (n % 4 == 0): operands copied with cp.async, R kept by columns.
constexpr int kTileSmem = 2 * GJB * GJP * 4;   // (Ls, Rc) or (Ls, Rs)
template <typename T, bool ASYNC>
__global__ void __launch_bounds__(GJTH) k_gj_rowpanel(const T* A, T* B, int64_t n, int k, const T* Pinv,
                                                      const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(16) float dsm[];
  float (*Ps)[GJP] = reinterpret_cast<float (*)[GJP]>(dsm);
  const int nt = int((n + GJB - 1) / GJB);
  const int jj = int(blockIdx.x) / 2, h = int(blockIdx.x) % 2;
  const int tj = jj >= k ? jj + 1 : jj;
  const int64_t c0 = int64_t(tj) * GJB + h * GJH;
  if (tj >= nt || c0 >= n) return;
  float acc[8][4];
  h_zero(acc);
  if (ASYNC) {
    float (*Rc)[GJP] = Ps + GJB;
#pragma unroll 4
    for (int q = 0; q < GJB * GJB / 4 / GJTH; ++q) {          // Ps[l][r] = P^{-1}(r, l)
      const int e = int(threadIdx.x) + q * GJTH;
      const int r = 4 * (e % 16), l = e / 16;
      cp_async16(&Ps[l][r], Pinv + r + GJB * l, true);
    }
#pragma unroll 4
    for (int q = 0; q < GJB * GJH / 4 / GJTH; ++q) {          // Rc[c][l] = A(64 k + l, c0 + c)
      const int e = int(threadIdx.x) + q * GJTH;
      const int l = 4 * (e % 16), c = e / 16;
      const int64_t gr = int64_t(k) * GJB + l, gc = c0 + c;
      const bool in = gr < n && gc < n;
      cp_async16(&Rc[c][l], in ? A + gr + n * gc : A, in);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    h_fma_rc<1>(Ps, Rc, acc);
  } else {
    float (*Xs)[GJH + 4] = reinterpret_cast<float (*)[GJH + 4]>(dsm + GJB * GJP);
    h_load_left(Pinv, GJB, 0, 0, Ps, 1.f);
    h_load_right(A, n, int64_t(k) * GJB, c0, Xs);
    __syncthreads();
    h_fma(Ps, Xs, acc);
  }
  h_store_block(acc, B, n, int64_t(k) * GJB, c0);
}

// Update of every half tile outside row k.  When skip_pivot is set, tile
// (k+1, k+1) is left to k_gj_pivot_next (which runs concurrently).
template <typename T, bool ASYNC>
__global__ void __launch_bounds__(GJTH) k_gj_update(const T* A, T* B, int64_t n, int k, const T* Pinv,
                                                    int skip_pivot, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(16) float dsm[];
  float (*Ls)[GJP] = reinterpret_cast<float (*)[GJP]>(dsm);
  const int nt = int((n + GJB - 1) / GJB);
  const int h = int(blockIdx.x) % 2, b = int(blockIdx.x) / 2;
  const int ti = b % (nt - 1) >= k ? b % (nt - 1) + 1 : b % (nt - 1);
  const int tj = b / (nt - 1);
  if (skip_pivot && ti == k + 1 && tj == k + 1) return;
  const int64_t r0 = int64_t(ti) * GJB, c0 = int64_t(tj) * GJB + h * GJH;
  if (c0 >= n) return;
  const int64_t ko = int64_t(k) * GJB;
  float acc[8][4];
  if (ASYNC) {
    float (*Rc)[GJP] = Ls + GJB;
#pragma unroll 4
    for (int q = 0; q < GJB * GJB / 4 / GJTH; ++q) {          // Ls[l][r] = A(r0 + r, 64 k + l)
      const int e = int(threadIdx.x) + q * GJTH;
      const int r = 4 * (e % 16), l = e / 16;
      const int64_t gr = r0 + r, gc = ko + l;
      const bool in = gr < n && gc < n;
      cp_async16(&Ls[l][r], in ? A + gr + n * gc : A, in);
    }
#pragma unroll 4
    for (int q = 0; q < GJB * GJH / 4 / GJTH; ++q) {          // Rc[c][l] = B(64 k + l, c0 + c) or P^{-1}
      const int e = int(threadIdx.x) + q * GJTH;
      const int l = 4 * (e % 16), c = e / 16;
      if (tj == k) {
        cp_async16(&Rc[c][l], Pinv + l + GJB * (h * GJH + c), true);
      } else {
        const int64_t gr = ko + l, gc = c0 + c;
        const bool in = gr < n && gc < n;
        cp_async16(&Rc[c][l], in ? B + gr + n * gc : B, in);
      }
    }
    cp_async_commit();
    if (tj == k) h_zero(acc);
    else h_load_block(A, n, r0, c0, acc);
    cp_async_wait<0>();
    __syncthreads();
    h_fma_rc<-1>(Ls, Rc, acc);                               // - A[i,k] B[k,j]
  } else {
    float (*Rs)[GJH + 4] = reinterpret_cast<float (*)[GJH + 4]>(dsm + GJB * GJP);
    h_load_left(A, n, r0, ko, Ls, -1.f);                      // -A[i,k]
    if (tj == k) {
      h_load_right(Pinv, GJB, 0, h * GJH, Rs);
      h_zero(acc);
    } else {
      h_load_right(B, n, ko, c0, Rs);                         // B[k,j] from the row panel
      h_load_block(A, n, r0, c0, acc);
    }
    __syncthreads();
    h_fma(Ls, Rs, acc);
  }
  h_store_block(acc, B, n, r0, c0);
}

// ---- rank-64 k updates on the tensor cores (tcgen05) ----
//
// k_gj_update_tc: one CTA (256 threads) per 128 x 128 output tile of the
// trailing part of the one-launch elimination of the leading identity block,
// a rank-(64 nkb) update over the tiles of [base, n)^2 (base = 64 nkb):
//     B[i, j] = A[i, j] - sum_{l < 64 nkb} A[i, l] A[l, j].
// Per K block of 64 the two operand slices (128 x 64 of the column panel,
// 64 x 128 of the row panel) are copied to a float32 staging area by
// cp.async; each thread splits half a row of each into three bfloat16
// pieces (x = x0 + x1 + x2, 24 significant bits) in the no-swizzle K-major
// layout of 8 x 16-byte core matrices (8-row groups 1024 bytes apart); one
// thread issues the six piece products down to 2^-16 relative (x0 y0, x0 y1,
// x1 y0, x1 y1, x0 y2, x2 y0: float32-level products), 4 MMAs of K = 16
// each, accumulating in 128 TMEM columns, while the next block's slices are
// copied.  Then the tile of A to subtract from is staged the same way, each
// warp reads 32 lanes (rows) x 64 columns of the accumulator back into it,
// and the CTA stores the result along the columns with 16-byte stores.
// The sweeps use the same pieces and layout in k_gj_sweep_tc and
// k_gj_update2_tc (below).
// Every wait for the MMAs is bounded: when one runs out the tile is not
// written, *info is set to n + 1 (the inverse is then rejected like one with
// a bad pivot), the timeout counter grows, and the CTA waits once more
// (bounded) before it frees its tensor memory.
constexpr int kUtM = 128;                          // rows (i) per tile
constexpr int kUtN = 128;                          // columns (j) per tile
constexpr int kUtPiece = 128 * GJB * 2;            // one bfloat16 piece of a 128 x 64 operand: 16 KB
constexpr int kUtSmem = 6 * kUtPiece;              // three pieces of each operand
constexpr int64_t kUtMinN = 1024;                  // smallest core inverted with tensor-core updates (measured: 768 and 900 are faster on the SIMT update)
int tc_timeout_counter(int** out);

__device__ __forceinline__ uint32_t ut_off(int row, int col) {
  return uint32_t((row >> 3) * 1024 + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2);
}

// the three bfloat16 pieces of 32 values of operand row `row`, inner index
// l0 .. l0 + 31 (pieces PS bytes apart)
template <int PS = kUtPiece>
__device__ __forceinline__ void ut_store_half(unsigned char* base, int row, int l0, const float (&v)[32]) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) tc::split3x2(v[8 * g + 2 * h], v[8 * g + 2 * h + 1], w0[h], w1[h], w2[h]);
    const uint32_t o = ut_off(row, l0 + 8 * g);
    *reinterpret_cast<uint4*>(base + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(base + PS + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(base + 2 * PS + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
}

// Shared memory of k_gj_update_tc: the six bfloat16 pieces, then a float32
// staging area that holds the two operand slices of a K block as copied
// (column panel [l][row], row panel [j][l] with rows padded to GJP floats so
// that the split reads no bank twice) and at the end the 128 x 128 tile of A
// to subtract from.
constexpr int kUtStage = (GJB * kUtM + kUtN * GJP) * 4;                  // 66.8 KB >= 128 x 128 x 4
constexpr int kUtSmemAll = kUtSmem + kUtStage;

// 16-byte copies of K block kb's operand slices into the staging area;
// n % 4 == 0, so a copy is wholly inside or wholly outside the matrix
template <typename T>
__device__ __forceinline__ void ut_copy_slices(const T* A, int64_t n, int64_t i0, int64_t j0, int64_t kc,
                                               float (*sa)[kUtM], float (*sr)[GJP]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < GJB * kUtM / 4 / 256; ++q) {           // A(i0 + r, kc + l)
    const int e = tid + 256 * q, l = e / 32, r = 4 * (e % 32);
    const bool in = i0 + r < n && kc + l < n;
    cp_async16(&sa[l][r], in ? A + (i0 + r) + n * (kc + l) : A, in);
  }
#pragma unroll
  for (int q = 0; q < kUtN * GJB / 4 / 256; ++q) {           // A(kc + l, j0 + j)
    const int e = tid + 256 * q, j = e / 16, l = 4 * (e % 16);
    const bool in = j0 + j < n && kc + l < n;
    cp_async16(&sr[j][l], in ? A + (kc + l) + n * (j0 + j) : A, in);
  }
  cp_async_commit();
}

template <typename T>
__global__ void __launch_bounds__(256) k_gj_update_tc(const T* A, T* B, int64_t n, int64_t base, int nkb,
                                                      const int* skip, int* info, int* tmo) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(1024) unsigned char ut_smem[];
  unsigned char* apc = ut_smem;                    // column-panel slice pieces, rows = i
  unsigned char* rpc = ut_smem + 3 * kUtPiece;     // row-panel slice pieces, rows = j
  float (*sa)[kUtM] = reinterpret_cast<float (*)[kUtM]>(ut_smem + kUtSmem);              // [l][row]
  float (*sr)[GJP] = reinterpret_cast<float (*)[GJP]>(ut_smem + kUtSmem + GJB * kUtM * 4); // [j][l]
  float (*si)[kUtM] = reinterpret_cast<float (*)[kUtM]>(ut_smem + kUtSmem);              // [c][row], at the end
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = base + int64_t(blockIdx.x) * kUtM, j0 = base + int64_t(blockIdx.y) * kUtN;
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tbase_s, 128);
    tc::tmem_relinquish();
  }
  ut_copy_slices(A, n, i0, j0, 0, sa, sr);
  const uint32_t id = tc::idesc_bf16(kUtM, kUtN, false, false);
  bool ok = true;
  int kb = 0;
  for (; kb < nkb; ++kb) {
    cp_async_wait<0>();
    __syncthreads();                               // staging holds block kb
    if (kb > 0) {                                  // the pieces are free once block kb - 1's MMAs are done
      ok = __syncthreads_and(tc::mbar_wait(&bar, uint32_t(kb - 1) & 1u) ? 1 : 0) != 0;
      if (!ok) break;
    }
    {
      const int row = tid & 127, l0 = 32 * (tid >> 7);        // one operand row, half of the inner index
      float v[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) v[l] = sa[l0 + l][row];
      ut_store_half(apc, row, l0, v);
#pragma unroll
      for (int l = 0; l < 32; l += 4) {
        const float4 t = *reinterpret_cast<const float4*>(&sr[row][l0 + l]);
        v[l] = t.x;
        v[l + 1] = t.y;
        v[l + 2] = t.z;
        v[l + 3] = t.w;
      }
      ut_store_half(rpc, row, l0, v);
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0) {
      const uint32_t tb = tbase_s;
      const uint32_t sa_ = tc::smem_u32(apc), sr_ = tc::smem_u32(rpc);
      constexpr int pa[6] = {0, 0, 1, 1, 0, 2}, pr[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int ks = 0; ks < GJB / 16; ++ks)
          tc::mma_bf16(tb, tc::sdesc(sa_ + pa[c] * kUtPiece + ks * 256, 128, 1024),
                       tc::sdesc(sr_ + pr[c] * kUtPiece + ks * 256, 128, 1024), id,
                       (kb | c | ks) ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    if (kb + 1 < nkb) {
      ut_copy_slices(A, n, i0, j0, int64_t(kb + 1) * GJB, sa, sr);
    } else {                                       // the tile of A to subtract from, while the MMAs run
#pragma unroll
      for (int q = 0; q < kUtN * kUtM / 4 / 256; ++q) {
        const int e = tid + 256 * q, c = e / 32, r = 4 * (e % 32);
        const bool in = i0 + r < n && j0 + c < n;
        cp_async16(&si[c][r], in ? A + (i0 + r) + n * (j0 + c) : A, in);
      }
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
  const uint32_t tb = tbase_s;
  if (ok) ok = __syncthreads_and(tc::mbar_wait(&bar, uint32_t(nkb - 1) & 1u) ? 1 : 0) != 0;
  if (ok) {
    tc::tc_fence_after();
    // warp w: TMEM lanes (rows) 32 (w % 4) .., columns 64 (w / 4) .. + 63;
    // the result replaces the staged tile in shared memory (lanes = rows:
    // no bank is read twice), then the CTA stores it along the columns
    const int qr = warp & 3, cbase = 64 * (warp >> 2), r = 32 * qr + lane;
#pragma unroll 1
    for (int c0 = cbase; c0 < cbase + 64; c0 += 32) {
      float d[32];
      tc::tmem_ld32(tb + (uint32_t(32 * qr) << 16) + uint32_t(c0), d);
#pragma unroll
      for (int c = 0; c < 32; ++c) si[c0 + c][r] -= d[c];
    }
  }
  __syncthreads();
  if (ok) {
#pragma unroll 4
    for (int q = 0; q < kUtN * kUtM / 4 / 256; ++q) {
      const int e = tid + 256 * q, c = e / 32, rr = 4 * (e % 32);
      const int64_t i = i0 + rr, j = j0 + c;
      if (i < n && j < n) *reinterpret_cast<float4*>(B + i + n * j) = *reinterpret_cast<const float4*>(&si[c][rr]);
    }
  } else {
    if (tid == 0) {
      if (tmo) atomicAdd(tmo, 1);
      if (info) atomicCAS(info, 0, int(n + 1));
    }
    // the MMAs last committed may still run: bounded drain
    tc::mbar_wait(&bar, uint32_t((kb < nkb ? kb : nkb) - 1) & 1u);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 128);
}

// The rank-64 update of one sweep above the one-launch size (the row panel
// already in B): B[i, j] = init - sum_l A[i, k0 + l] B[k0 + l, j] with init
// 0 in column block k, else A[i, j]; rows of block k and, with skip_pivot,
// tile (k + 1, k + 1) are not written.  Same products as k_gj_update_tc,
// but with only the bfloat16 pieces in shared memory (96 KB), so that two
// CTAs share an SM and one's loads and split overlap the other's products
// and stores: each thread splits its operand half-rows straight from global
// memory (a warp's loads of the column panel are 128-byte rows), the tile of
// A to subtract from is read per 32-column chunk into registers, and the
// result is staged for the 16-byte stores where the pieces were.
template <typename T>
__global__ void __launch_bounds__(256, 2) k_gj_update2_tc(const T* A, T* B, int64_t n, int k, int skip_pivot,
                                                          const int* skip, int* info, int* tmo) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(1024) unsigned char u2_smem[];
  unsigned char* apc = u2_smem;                    // column-panel pieces, rows = i
  unsigned char* rpc = u2_smem + 3 * kUtPiece;     // row-panel pieces, rows = j
  float (*st)[kUtM] = reinterpret_cast<float (*)[kUtM]>(u2_smem);   // [j][i], the result, at the end
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t i0 = int64_t(blockIdx.x) * kUtM, j0 = int64_t(blockIdx.y) * kUtN, k0 = int64_t(k) * GJB;
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tbase_s, 128);
    tc::tmem_relinquish();
  }
  {
    const int row = tid & 127, l0 = 32 * (tid >> 7);
    float v[32];
    const int64_t i = i0 + row;
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = (i < n && k0 + l0 + c < n) ? A[i + n * (k0 + l0 + c)] : 0.f;
    ut_store_half(apc, row, l0, v);
    const int64_t j = j0 + row;
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < n && k0 + l0 + c < n) q = *reinterpret_cast<const float4*>(B + (k0 + l0 + c) + n * j);
      v[c] = q.x;
      v[c + 1] = q.y;
      v[c + 2] = q.z;
      v[c + 3] = q.w;
    }
    ut_store_half(rpc, row, l0, v);
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tb = tbase_s;
  if (tid == 0) {
    const uint32_t id = tc::idesc_bf16(kUtM, kUtN, false, false);
    const uint32_t sa_ = tc::smem_u32(apc), sr_ = tc::smem_u32(rpc);
    constexpr int pa[6] = {0, 0, 1, 1, 0, 2}, pr[6] = {0, 1, 0, 1, 2, 0};
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int ks = 0; ks < GJB / 16; ++ks)
        tc::mma_bf16(tb, tc::sdesc(sa_ + pa[c] * kUtPiece + ks * 256, 128, 1024),
                     tc::sdesc(sr_ + pr[c] * kUtPiece + ks * 256, 128, 1024), id, (c | ks) ? 1u : 0u);
    tc::mma_commit(&bar);
  }
  __syncwarp();
  // warp w: TMEM lanes (rows) 32 (w % 4) .., columns 64 (w / 4) .. + 63
  const int qr = warp & 3, cbase = 64 * (warp >> 2), r = 32 * qr + lane;
  const int64_t i = i0 + r;
  float cv[32];                                    // the first chunk of A's tile, while the products run
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const int64_t j = j0 + cbase + c;
    cv[c] = (i < n && j < n && j / GJB != k) ? A[i + n * j] : 0.f;
  }
  const bool ok = __syncthreads_and(tc::mbar_wait(&bar, 0u) ? 1 : 0) != 0;
  if (ok) {
    tc::tc_fence_after();
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int c0 = cbase + 32 * h;
      if (h == 1) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int64_t j = j0 + c0 + c;
          cv[c] = (i < n && j < n && j / GJB != k) ? A[i + n * j] : 0.f;
        }
      }
      float d[32];
      tc::tmem_ld32(tb + (uint32_t(32 * qr) << 16) + uint32_t(c0), d);
#pragma unroll
      for (int c = 0; c < 32; ++c) st[c0 + c][r] = cv[c] - d[c];   // the pieces are dead: the products are done
    }
  }
  __syncthreads();
  if (ok) {
#pragma unroll 4
    for (int q = 0; q < kUtN * kUtM / 4 / 256; ++q) {   // four rows per copy: a 64-row block never splits one
      const int e = tid + 256 * q, c = e / 32, rr = 4 * (e % 32);
      const int64_t ii = i0 + rr, j = j0 + c;
      const int64_t bi = ii / GJB, bj = j / GJB;
      if (ii < n && j < n && bi != k && !(skip_pivot && bi == k + 1 && bj == k + 1))
        *reinterpret_cast<float4*>(B + ii + n * j) = *reinterpret_cast<const float4*>(&st[c][rr]);
    }
  } else {
    if (tid == 0) {
      if (tmo) atomicAdd(tmo, 1);
      if (info) atomicCAS(info, 0, int(n + 1));
    }
    tc::mbar_wait(&bar, 0u);                       // bounded drain of the products
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 128);
}

// The first kb0 tiles of the core lie inside its leading identity block
// (the core's diagonal R^2 x R^2 blocks are I).  Eliminating them at once
// (pivot I of size kb0 * GJB) maps A -> B as
//     B[0:,0:] = I, B[0:, j] = A[0:, j], B[i, 0:] = -A[i, 0:],
//     B[i, j] = A[i, j] - A[i, 0:] A[0:, j]      (tiles i, j >= kb0)
// which replaces kb0 sweeps by one launch.  CTA = one output half tile.
// ASYNC (n % 4 == 0): the K loop of an interior tile copies the operands of
// step kk + 1 (cp.async, two shared-memory stages in dynamic shared memory)
// while it multiplies those of step kk.
constexpr int kIdentSmem = 2 * 2 * GJB * GJP * 4;   // two stages of (Ls, Rc)
template <typename T, bool ASYNC>
__global__ void __launch_bounds__(GJTH) k_gj_identity(const T* A, T* B, int64_t n, int kb0, int border_only,
                                                      const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(16) float dsm[];
  const int nt = int((n + GJB - 1) / GJB);
  const int h = int(blockIdx.x) % 2, b = int(blockIdx.x) / 2;
  const int ti = b % nt, tj = b / nt;
  if (border_only && ti >= kb0 && tj >= kb0) return;   // the trailing tiles: k_gj_update_tc
  const int bi = threadIdx.x % 8, bj = threadIdx.x / 8;
  const int64_t r0 = int64_t(ti) * GJB, c0 = int64_t(tj) * GJB + h * GJH;
  if (c0 >= n) return;
  float acc[8][4];
  if (ti < kb0 || tj < kb0) {
    if (ti < kb0 && tj < kb0) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = (r0 + h_row(bi, u / 4) + u % 4 == c0 + 4 * bj + v) ? 1.f : 0.f;
    } else {
      h_load_block(A, n, r0, c0, acc);
      if (ti >= kb0) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = -acc[u][v];
      }
    }
    h_store_block(acc, B, n, r0, c0);
    return;
  }
  if (ASYNC) {
    float (*Ls0)[GJP] = reinterpret_cast<float (*)[GJP]>(dsm);
    float (*Rc0)[GJP] = Ls0 + GJB;
    float (*Ls1)[GJP] = Rc0 + GJB;
    float (*Rc1)[GJP] = Ls1 + GJB;
    h_copy_operands(A, n, r0, 0, 0, c0, Ls0, Rc0);
    cp_async_commit();
    h_load_block(A, n, r0, c0, acc);
    for (int kk = 0; kk < kb0; ++kk) {
      const bool odd = kk & 1;
      if (kk + 1 < kb0) {
        h_copy_operands(A, n, r0, int64_t(kk + 1) * GJB, int64_t(kk + 1) * GJB, c0, odd ? Ls0 : Ls1,
                        odd ? Rc0 : Rc1);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      h_fma_rc<-1>(odd ? Ls1 : Ls0, odd ? Rc1 : Rc0, acc);
      __syncthreads();
    }
  } else {
    float (*Ls)[GJP] = reinterpret_cast<float (*)[GJP]>(dsm);
    float (*Rs)[GJH + 4] = reinterpret_cast<float (*)[GJH + 4]>(dsm + GJB * GJP);
    h_load_block(A, n, r0, c0, acc);
    for (int kk = 0; kk < kb0; ++kk) {
      __syncthreads();
      h_load_left(A, n, r0, int64_t(kk) * GJB, Ls, -1.f);
      h_load_right(A, n, int64_t(kk) * GJB, c0, Rs);
      __syncthreads();
      h_fma(Ls, Rs, acc);
    }
  }
  h_store_block(acc, B, n, r0, c0);
}

// ---------------------------------------------------------------------------
// The pivot chain is the sequential part of the inversion.  Each pivot block
// is inverted by one 128-thread CTA that keeps the block in registers (4 x 8
// entries per thread); an elimination step broadcasts the pivot row (two
// float4 per owning thread) and column (one float4) through shared memory,
// double-buffered, so one barrier per step.  A step is about 160 cycles of
// dependent latency (store, barrier, load, reciprocal, multiply-add): 10.4K
// cycles a tile, measured.  Eliminating four pivots per barrier (each thread
// inverting the 4 x 4 pivot block itself, then a rank-4 update) took 13.4K
// cycles, and the 256-thread 4 x 4 layout about 240 cycles a step: the extra
// instructions lie on the chain.  For sweep k + 1 the pivot tile
// X = A[k+1,k+1] - A[k+1,k] (P_k^{-1} A[k,k+1]) is first formed from sweep
// k's input, so that it is inverted concurrently with sweep k's row panel
// and update.
// ---------------------------------------------------------------------------
// Barrier of the 128 pivot threads: the whole CTA, or (NB) named barrier 1
// over warps 0-3 when the pivot runs inside a larger CTA whose other warps
// have left.
template <bool NB>
__device__ __forceinline__ void gj_sync() {
  if constexpr (NB) asm volatile("bar.sync 1, 128;\n" ::: "memory");
  else __syncthreads();
}

// All 64 steps run, in groups of 8 so that the row and column a step reads
// sit at compile-time offsets of the owning threads' registers.  Rows and
// columns beyond kb hold the identity (pad_identity), and a step on such a
// unit row/column leaves the tile unchanged; only the first kb pivots are
// checked.
template <bool NB>
__device__ void gj_invert_tile(float (&x)[4][8], int kb, float (*prow)[GJB], float (*pcol)[GJB], int* bad) {
  __shared__ float pv[GJB];                                    // pivots, checked at the end
  const int bi = threadIdx.x % 16, bj = threadIdx.x / 16;
  for (int g = 0; g < GJB / 8; ++g) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int p = 8 * g + q, par = q & 1, lr = q & 3;
      const bool orow = (bi == (p >> 2)), ocol = (bj == g);   // owners of row p / column p
      if (orow) {
        *reinterpret_cast<float4*>(&prow[par][8 * bj]) = make_float4(x[lr][0], x[lr][1], x[lr][2], x[lr][3]);
        *reinterpret_cast<float4*>(&prow[par][8 * bj + 4]) = make_float4(x[lr][4], x[lr][5], x[lr][6], x[lr][7]);
      }
      if (ocol) *reinterpret_cast<float4*>(&pcol[par][4 * bi]) = make_float4(x[0][q], x[1][q], x[2][q], x[3][q]);
      gj_sync<NB>();
      const float piv = prow[par][p];
      if (threadIdx.x == 0) pv[p] = piv;
      const float dinv = recip(piv);
      const float4 c4 = *reinterpret_cast<const float4*>(&pcol[par][4 * bi]);
      const float4 r0 = *reinterpret_cast<const float4*>(&prow[par][8 * bj]);
      const float4 r1 = *reinterpret_cast<const float4*>(&prow[par][8 * bj + 4]);
      const float c[4] = {c4.x, c4.y, c4.z, c4.w};
      const float r[8] = {r0.x * dinv, r0.y * dinv, r0.z * dinv, r0.w * dinv,
                          r1.x * dinv, r1.y * dinv, r1.z * dinv, r1.w * dinv};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) x[u][v] = fmaf(-c[u], r[v], x[u][v]);
      if (orow) {                    // row p -> scaled pivot row
#pragma unroll
        for (int v = 0; v < 8; ++v) x[lr][v] = r[v];
      }
      if (ocol) {                    // column p -> -col / piv; the pivot itself -> 1 / piv
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u][q] = (orow && u == lr) ? dinv : -c[u] * dinv;
      }
    }
  }
  // check the recorded pivots once, after the elimination
  gj_sync<NB>();
  if (threadIdx.x < kb && !(pv[threadIdx.x] > 0.f && isfinite(pv[threadIdx.x]))) atomicMin(bad, threadIdx.x + 1);
  gj_sync<NB>();
}

// rows/columns of a partial pivot tile beyond kb become the identity
__device__ __forceinline__ void pad_identity(float (&x)[4][8], int kb) {
  const int bi = threadIdx.x % 16, bj = threadIdx.x / 16;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v)
      if (4 * bi + u >= kb || 8 * bj + v >= kb) x[u][v] = (4 * bi + u == 8 * bj + v) ? 1.f : 0.f;
}

// Invert x (pivot tile kk) and write P^{-1} to Pinv (64 x 64) and into tile
// (kk, kk) of D.
// (D == nullptr: Pinv only.)
template <bool NB>
__device__ void pivot_store(float (&x)[4][8], int64_t n, int kk, int kb, float* Pinv, float* D, int* info,
                            float (*prow)[GJB], float (*pcol)[GJB], int* bad) {
  if (threadIdx.x == 0) *bad = GJB + 1;
  gj_sync<NB>();
  gj_invert_tile<NB>(x, kb, prow, pcol, bad);
  if (threadIdx.x == 0 && *bad <= GJB && info) atomicCAS(info, 0, kk * GJB + *bad);
  store_block(x, Pinv, GJB, 0, 0);
  if (D) store_block(x, D, n, int64_t(kk) * GJB, int64_t(kk) * GJB);
}

// Pivot of sweep k (tile (k, k) of A as it stands); P^{-1} also into D's tile.
template <typename T>
__global__ void __launch_bounds__(GJT) k_gj_pivot(const T* A, T* D, int64_t n, int k, T* Pinv, int* info,
                                                  const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ __align__(16) float prow[2][GJB], pcol[2][GJB];
  __shared__ int bad;
  const int kb = int((n - int64_t(k) * GJB) < GJB ? (n - int64_t(k) * GJB) : GJB);
  float x[4][8];
  load_block(A, n, int64_t(k) * GJB, int64_t(k) * GJB, x);
  pad_identity(x, kb);
  pivot_store<false>(x, n, k, kb, Pinv, D, info, prow, pcol, &bad);
}

// x += SGN L R with L = Lc (64 x 64, stored by columns: Lc[l][r] = L(r, l))
// and R = Rc (64 x 64, stored by columns: Rc[c][l] = R(l, c)), four inner
// steps per iteration: four float4 of L and eight float4 of R (two distinct
// addresses per warp, broadcast) for 128 multiply-adds.
template <int SGN>
__device__ __forceinline__ void tile_fma_cc(const float (*Lc)[GJP], const float (*Rc)[GJP], float (&x)[4][8]) {
  const int bi = threadIdx.x % 16, bj = threadIdx.x / 16;
#pragma unroll 2
  for (int l = 0; l < GJB; l += 4) {
    float a[4][4], b[8][4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const float4 t = *reinterpret_cast<const float4*>(&Lc[l + w][4 * bi]);
      a[w][0] = SGN * t.x;
      a[w][1] = SGN * t.y;
      a[w][2] = SGN * t.z;
      a[w][3] = SGN * t.w;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float4 t = *reinterpret_cast<const float4*>(&Rc[8 * bj + v][l]);
      b[v][0] = t.x;
      b[v][1] = t.y;
      b[v][2] = t.z;
      b[v][3] = t.w;
    }
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) x[u][v] = fmaf(a[w][u], b[v][w], x[u][v]);
  }
}

// S[c][r] = A(r0 + r, c0 + c) for r, c < 64 by cp.async, 16 bytes (four rows
// of one column) per copy, zero outside n x n.  Needs n % 4 == 0 (then every
// source address is 16-byte aligned: r0 and r are multiples of 4).  NT threads.
template <int NT>
__device__ __forceinline__ void copy_cols_async(const float* A, int64_t n, int64_t r0, int64_t c0, float (*S)[GJP],
                                                int t = int(threadIdx.x)) {
#pragma unroll
  for (int q = 0; q < GJB * GJB / 4 / NT; ++q) {
    const int e = t + q * NT;
    const int r = 4 * (e % 16), c = e / 16;
    const int64_t gr = r0 + r, gc = c0 + c;
    const bool in = gr < n && gc < n;
    cp_async16(&S[c][r], in ? A + gr + n * gc : A, in);
  }
}

// Pivot of sweep k + 1 during sweep k, from sweep k's input A and pivot
// inverse Pinv alone: X = A[k+1,k+1] - A[k+1,k] (P^{-1} A[k,k+1]), inverted;
// X^{-1} goes to Pinv_next and (D != nullptr) into D's tile (k+1, k+1).  The
// three operand tiles are fetched at once (ASYNC, n % 4 == 0: cp.async, 16
// bytes a copy; else scalar loads), all stored by columns, before the first
// product.  k_gj_pivot_next runs it on a side stream with D = A (the tile
// that sweep k + 1 writes into and that no kernel of sweep k reads), launched
// with kPivotReserve bytes of dynamic shared memory (unused: it keeps the
// tile CTAs of the concurrent sweep off this SM).
template <typename T, bool ASYNC>
__device__ __forceinline__ void pivot_next_body(const T* A, int64_t n, int k, const T* Pinv, T* Pinv_next, int* info,
                                                float (*Ls)[GJP], float (*Rc)[GJP], float (*L2s)[GJP],
                                                float (*prow)[GJB], float (*pcol)[GJB], int* bad, T* D) {
  const int k1 = k + 1;
  const int kb = int((n - int64_t(k1) * GJB) < GJB ? (n - int64_t(k1) * GJB) : GJB);
  const int64_t o = int64_t(k) * GJB, o1 = int64_t(k1) * GJB;
  const int bi = threadIdx.x % 16, bj = threadIdx.x / 16;
  if (ASYNC) {
    copy_cols_async<GJT>(Pinv, GJB, 0, 0, Ls);       // P^{-1}
    copy_cols_async<GJT>(A, n, o, o1, Rc);           // A[k, k+1]
    copy_cols_async<GJT>(A, n, o1, o, L2s);          // A[k+1, k]
    cp_async_commit();
  } else {
    load_cols<GJT>(Pinv, GJB, 0, 0, Ls, 1.f);
    load_cols<GJT>(A, n, o, o1, Rc, 1.f);
    load_cols<GJT>(A, n, o1, o, L2s, 1.f);
  }
  float x[4][8], t[4][8];
  load_block(A, n, o1, o1, x);                       // A[k+1, k+1]
  zero_block(t);
  if (ASYNC) cp_async_wait<0>();
  __syncthreads();
  tile_fma_cc<1>(Ls, Rc, t);                         // t = P^{-1} A[k, k+1]
  __syncthreads();
#pragma unroll
  for (int v = 0; v < 8; ++v)                        // Rc <- t, by columns
    *reinterpret_cast<float4*>(&Rc[8 * bj + v][4 * bi]) = make_float4(t[0][v], t[1][v], t[2][v], t[3][v]);
  __syncthreads();
  tile_fma_cc<-1>(L2s, Rc, x);                       // x = A[k+1,k+1] - A[k+1,k] t
  pad_identity(x, kb);
  pivot_store<false>(x, n, k1, kb, Pinv_next, D, info, prow, pcol, bad);
}

template <typename T, bool ASYNC>
__global__ void __launch_bounds__(GJT) k_gj_pivot_next(T* A, int64_t n, int k, const T* Pinv, T* Pinv_next,
                                                       int* info, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ __align__(16) float Ls[GJB][GJP], Rc[GJB][GJP], L2s[GJB][GJP];
  __shared__ __align__(16) float prow[2][GJB], pcol[2][GJB];
  __shared__ int bad;
  pivot_next_body<T, ASYNC>(A, n, k, Pinv, Pinv_next, info, Ls, Rc, L2s, prow, pcol, &bad, A);
}

// x += SGN L R over the inner indices l0 .. l0 + 31 only, thread (bi, bj)
// owning rows 4 bi .. + 3 and columns 8 bj .. + 7 (the layout of
// tile_fma_cc, for one 128-thread group of a larger CTA); L and R stored by
// columns.
template <int SGN>
__device__ __forceinline__ void tile_fma_cc_k32(const float (*Lc)[GJP], const float (*Rc)[GJP], float (&x)[4][8],
                                                int bi, int bj, int l0) {
#pragma unroll 2
  for (int l = l0; l < l0 + 32; l += 4) {
    float a[4][4], b[8][4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const float4 t = *reinterpret_cast<const float4*>(&Lc[l + w][4 * bi]);
      a[w][0] = SGN * t.x;
      a[w][1] = SGN * t.y;
      a[w][2] = SGN * t.z;
      a[w][3] = SGN * t.w;
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float4 t = *reinterpret_cast<const float4*>(&Rc[8 * bj + v][l]);
      b[v][0] = t.x;
      b[v][1] = t.y;
      b[v][2] = t.z;
      b[v][3] = t.w;
    }
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) x[u][v] = fmaf(a[w][u], b[v][w], x[u][v]);
  }
}

// Partial tile of group 1 into T (by columns) / added from T by group 0.
__device__ __forceinline__ void tile_put_cols(const float (&x)[4][8], float (*T)[GJP], int bi, int bj) {
#pragma unroll
  for (int v = 0; v < 8; ++v)
    *reinterpret_cast<float4*>(&T[8 * bj + v][4 * bi]) = make_float4(x[0][v], x[1][v], x[2][v], x[3][v]);
}
__device__ __forceinline__ void tile_add_cols(float (&x)[4][8], const float (*T)[GJP], int bi, int bj) {
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const float4 q = *reinterpret_cast<const float4*>(&T[8 * bj + v][4 * bi]);
    x[0][v] += q.x;
    x[1][v] += q.y;
    x[2][v] += q.z;
    x[3][v] += q.w;
  }
}

// The pivot of sweep k + 1 as pivot_next_body forms it (n % 4 == 0), inside
// a 256-thread CTA.  Each product is split over the inner index: warps 0-3
// take l < 32 and warps 4-7 l >= 32, both in the 4 x 8 layout of the
// inversion, and the second half is added through shared memory (two
// warps per scheduler; the 128-thread products took 3.6K and 4.0K cycles,
// 256 threads on 4 x 4 entries over the whole inner index 4.0K and 3.8K).
// Warps 0-3 then hold X in their registers, invert it (named barrier 1) and
// write X^{-1} to Pinv_next.  smem: at least 4 x 64 x GJP + 4 x 64 floats +
// one int, 16-byte aligned.
template <typename T>
__device__ __forceinline__ void pivot_next_wide(const T* A, int64_t n, int k, const T* Pinv, T* Pinv_next, int* info,
                                                unsigned char* smem) {
  float (*Ls)[GJP] = reinterpret_cast<float (*)[GJP]>(smem);
  float (*Rc)[GJP] = Ls + GJB;
  float (*L2s)[GJP] = Rc + GJB;
  float (*Ts)[GJP] = L2s + GJB;
  float (*prow)[GJB] = reinterpret_cast<float (*)[GJB]>(Ts + GJB);
  float (*pcol)[GJB] = prow + 2;
  int* bad = reinterpret_cast<int*>(pcol + 2);
  const int k1 = k + 1;
  const int kb = int((n - int64_t(k1) * GJB) < GJB ? (n - int64_t(k1) * GJB) : GJB);
  const int64_t o = int64_t(k) * GJB, o1 = int64_t(k1) * GJB;
  const int tid = threadIdx.x, grp = tid >> 7, bi = tid % 16, bj = (tid & 127) / 16;
  copy_cols_async<256>(Pinv, GJB, 0, 0, Ls);         // P^{-1}
  copy_cols_async<256>(A, n, o, o1, Rc);             // A[k, k+1]
  copy_cols_async<256>(A, n, o1, o, L2s);            // A[k+1, k]
  cp_async_commit();
  float x[4][8], t[4][8];
  if (grp == 0) load_block(A, n, o1, o1, x);         // A[k+1, k+1]
  else zero_block(x);
  zero_block(t);
  cp_async_wait<0>();
  __syncthreads();
  tile_fma_cc_k32<1>(Ls, Rc, t, bi, bj, 32 * grp);   // t = P^{-1} A[k, k+1], half the inner index
  if (grp == 1) tile_put_cols(t, Ts, bi, bj);
  __syncthreads();
  if (grp == 0) {
    tile_add_cols(t, Ts, bi, bj);
    tile_put_cols(t, Rc, bi, bj);                    // Rc <- t, by columns
  }
  __syncthreads();
  tile_fma_cc_k32<-1>(L2s, Rc, x, bi, bj, 32 * grp); // x = A[k+1,k+1] - A[k+1,k] t, half the inner index
  if (grp == 1) tile_put_cols(x, Ts, bi, bj);
  __syncthreads();
  if (grp == 0) {
    tile_add_cols(x, Ts, bi, bj);
    pad_identity(x, kb);
    pivot_store<true>(x, n, k1, kb, Pinv_next, nullptr, info, prow, pcol, bad);
  }
}

// One sweep of the tensor-core path in one launch (n % 4 == 0, k0 = 64 k).
// CTA 0 forms and inverts the pivot of sweep k + 1 from this sweep's input
// (pivot_next_wide).
// CTA 1 + ib + mt jb produces the output tile of rows i0 = 128 ib .. + 127
// and columns j0 = 128 jb .. + 127 in two rounds of tensor-core products:
//   (1) its slice of the row panel, transposed: for l < 64 and j in the tile,
//           Rt[j, l] = sum_m A[k0 + m, j] P^{-1}[l, m]
//       with A[k, k] taken as the identity, so that the columns of block k
//       get P^{-1} itself (M = 128 rows j, N = 64, K = 64, TMEM columns
//       128 .. 191); the CTAs whose rows hold block k store it as rows k of
//       B (B[k, j] = P^{-1} A[k, j], B[k, k] = P^{-1});
//   (2) the rank-64 update of the tile from Rt (TMEM columns 0 .. 127):
//           B[i, j] = A[i, j] - sum_l A[i, k0 + l] Rt[j, l]   (j outside block k)
//           B[i, j] = -sum_l A[i, k0 + l] Rt[j, l]             (j in block k)
//       stored for the rows i outside block k.
// Every float32 operand enters as three bfloat16 pieces and six piece
// products (float32-level products, float32 accumulation in TMEM).  This
// replaces the separate row-panel launch and the side-stream pivot launch of
// a sweep by one launch.
constexpr int kSwPPiece = GJB * GJB * 2;                             // one piece of P^{-1}: 8 KB
constexpr int kSwPc = 3 * kUtPiece;                                  // column-panel pieces (rows i)
constexpr int kSwRt = 3 * kUtPiece;                                  // A[k, J]^T pieces, then Rt pieces (rows j)
constexpr int kSwPp = 3 * kSwPPiece;                                 // P^{-1} pieces (rows l)
constexpr int kSwStageOff = kSwPc + kSwRt + kSwPp;                   // 120 KB
constexpr int kSwStage = (GJB * kUtM + kUtN * GJP + GJB * GJP) * 4;  // sa, sk, sp: 83 KB >= 128 x 128 x 4
constexpr int kSwSmem = kSwStageOff + kSwStage;                      // 203 KB
static_assert(kSwStage >= kUtM * kUtN * 4, "the output tile is staged where the operands were");
static_assert(kSwSmem + 1024 <= 227 * 1024, "one CTA per SM");

// Output tile t = ib + mt jb of sweep k (256 threads): operands, the two
// rounds of products and the stores.  bar: an initialised mbarrier whose next
// two phases have parities 0 and 1; tb: 256 allocated TMEM columns.  Returns
// false when a wait for the products ran out (the tile is then not written,
// *info = n + 1, the timeout counter grows, and the products last committed
// have been waited for once more, bounded).
template <typename T>
__device__ bool sweep_tile(const T* A, T* B, const T* Pk, int64_t n, int k, int t, unsigned char* sw_smem,
                           uint64_t* barp, uint32_t tb, int* info, int* tmo) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* apc = sw_smem;                                      // A[I, k] pieces, rows i
  unsigned char* rpc = sw_smem + kSwPc;                              // A[k, J]^T pieces, then Rt pieces, rows j
  unsigned char* ppc = sw_smem + kSwPc + kSwRt;                      // P^{-1} pieces, rows l
  float (*sa)[kUtM] = reinterpret_cast<float (*)[kUtM]>(sw_smem + kSwStageOff);   // [l][i]
  float (*sk)[GJP] = reinterpret_cast<float (*)[GJP]>(sw_smem + kSwStageOff + GJB * kUtM * 4);  // [j][m]
  float (*sp)[GJP] = sk + kUtN;                                      // [m][l]
  float (*si)[kUtM] = sa;                                            // [j][i], the output tile, at the end
  uint64_t& bar = *barp;
  const int mt = int((n + kUtM - 1) / kUtM);
  const int64_t i0 = int64_t(t % mt) * kUtM, j0 = int64_t(t / mt) * kUtN, k0 = int64_t(k) * GJB;
  // the operands of (1) first (A[k0 + m, j0 + j], not for j in block k, and
  // P^{-1}), then the column panel A[i0 + r, k0 + l], split while (1) runs
#pragma unroll
  for (int q = 0; q < kUtN * GJB / 4 / 256; ++q) {
    const int e = tid + 256 * q, j = e / 16, m = 4 * (e % 16);
    const int64_t jj = j0 + j;
    if (jj / GJB == k) continue;
    const bool in = jj < n && k0 + m < n;
    cp_async16(&sk[j][m], in ? A + (k0 + m) + n * jj : A, in);
  }
#pragma unroll
  for (int q = 0; q < GJB * GJB / 4 / 256; ++q) {
    const int e = tid + 256 * q, m = e / 16, l = 4 * (e % 16);
    cp_async16(&sp[m][l], Pk + l + GJB * m, true);
  }
  cp_async_commit();
#pragma unroll
  for (int q = 0; q < GJB * kUtM / 4 / 256; ++q) {
    const int e = tid + 256 * q, l = e / 32, r = 4 * (e % 32);
    const bool in = i0 + r < n && k0 + l < n;
    cp_async16(&sa[l][r], in ? A + (i0 + r) + n * (k0 + l) : A, in);
  }
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();
  const int row = tid & 127, l0 = 32 * (tid >> 7);
  float v[32];
  {
    const int64_t jj = j0 + row;
    if (jj / GJB == k) {
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = (int64_t(l0 + c) == jj - k0) ? 1.f : 0.f;
    } else {
#pragma unroll
      for (int c = 0; c < 32; c += 4) {
        const float4 x4 = *reinterpret_cast<const float4*>(&sk[row][l0 + c]);
        v[c] = x4.x;
        v[c + 1] = x4.y;
        v[c + 2] = x4.z;
        v[c + 3] = x4.w;
      }
    }
    ut_store_half(rpc, row, l0, v);
    if (tid < 128) {
      const int pr = tid & 63, p0 = 32 * (tid >> 6);
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = sp[p0 + c][pr];
      ut_store_half<kSwPPiece>(ppc, pr, p0, v);
    }
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  constexpr int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
  if (tid == 0) {                                 // (1) Rt in TMEM columns 128 .. 191
    const uint32_t id = tc::idesc_bf16(kUtN, GJB, false, false);
    const uint32_t sr_ = tc::smem_u32(rpc), sp_ = tc::smem_u32(ppc);
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int ks = 0; ks < GJB / 16; ++ks)
        tc::mma_bf16(tb + 128, tc::sdesc(sr_ + pa[c] * kUtPiece + ks * 256, 128, 1024),
                     tc::sdesc(sp_ + pb[c] * kSwPPiece + ks * 256, 128, 1024), id, (c | ks) ? 1u : 0u);
    tc::mma_commit(&bar);
  }
  __syncwarp();
  cp_async_wait<0>();
  __syncthreads();                                // the column panel has landed
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = sa[l0 + c][row];
  ut_store_half(apc, row, l0, v);
  int ph = 0;                                     // commits made so far - 1
  // after this barrier no thread reads the staging area any more
  bool ok = __syncthreads_and(tc::mbar_wait(&bar, 0u) ? 1 : 0) != 0;
  // the tile of A to subtract from, while the rest runs
#pragma unroll
  for (int q = 0; q < kUtN * kUtM / 4 / 256; ++q) {
    const int e = tid + 256 * q, c = e / 32, r = 4 * (e % 32);
    const bool in = i0 + r < n && j0 + c < n;
    cp_async16(&si[c][r], in ? A + (i0 + r) + n * (j0 + c) : A, in);
  }
  cp_async_commit();
  if (ok) {
    tc::tc_fence_after();
    // warp w: rows j = 32 (w % 4) + lane, l = 32 (w / 4) .. + 31
    const int qr = warp & 3, lw = 32 * (warp >> 2), j = 32 * qr + lane;
    tc::tmem_ld32(tb + (uint32_t(32 * qr) << 16) + 128u + uint32_t(lw), v);
    const int64_t jj = j0 + j;
    if (k0 >= i0 && k0 < i0 + kUtM && jj < n) {   // rows k of B
#pragma unroll
      for (int c = 0; c < 32; c += 4)
        if (k0 + lw + c < n)
          *reinterpret_cast<float4*>(B + (k0 + lw + c) + n * jj) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
    }
    ut_store_half(rpc, j, lw, v);                 // the products of (1) have read rpc
    tc::fence_async_smem();                       // (and the column-panel pieces written above)
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0) {                               // (2) the update in TMEM columns 0 .. 127
      const uint32_t id = tc::idesc_bf16(kUtM, kUtN, false, false);
      const uint32_t sa_ = tc::smem_u32(apc), sr_ = tc::smem_u32(rpc);
#pragma unroll
      for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int ks = 0; ks < GJB / 16; ++ks)
          tc::mma_bf16(tb, tc::sdesc(sa_ + pa[c] * kUtPiece + ks * 256, 128, 1024),
                       tc::sdesc(sr_ + pb[c] * kUtPiece + ks * 256, 128, 1024), id, (c | ks) ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    __syncwarp();
    ph = 1;
    cp_async_wait<0>();
    ok = __syncthreads_and(tc::mbar_wait(&bar, 1u) ? 1 : 0) != 0;
  }
  cp_async_wait<0>();
  if (ok) {
    // warp w: TMEM lanes (rows) 32 (w % 4) .., columns 64 (w / 4) .. + 63;
    // the result replaces the staged tile (lanes = rows: no bank is read
    // twice), then the CTA stores it along the columns, 16 bytes a thread
    // (storing each warp's 32 rows of a column from registers took 6.9K
    // cycles against 4.8K)
    tc::tc_fence_after();
    const int qr = warp & 3, cbase = 64 * (warp >> 2), r = 32 * qr + lane;
#pragma unroll 1
    for (int c0 = cbase; c0 < cbase + 64; c0 += 32) {
      float d[32];
      tc::tmem_ld32(tb + (uint32_t(32 * qr) << 16) + uint32_t(c0), d);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int64_t j = j0 + c0 + c;
        si[c0 + c][r] = ((j / GJB == k) ? 0.f : si[c0 + c][r]) - d[c];
      }
    }
  }
  __syncthreads();
  if (ok) {
#pragma unroll 4
    for (int q = 0; q < kUtN * kUtM / 4 / 256; ++q) {   // four rows per copy: a 64-row block never splits one
      const int e = tid + 256 * q, c = e / 32, rr = 4 * (e % 32);
      const int64_t i = i0 + rr, j = j0 + c;
      if (i < n && j < n && i / GJB != k)
        *reinterpret_cast<float4*>(B + i + n * j) = *reinterpret_cast<const float4*>(&si[c][rr]);
    }
  } else {
    if (tid == 0) {
      if (tmo) atomicAdd(tmo, 1);
      if (info) atomicCAS(info, 0, int(n + 1));
    }
    tc::mbar_wait(&bar, uint32_t(ph) & 1u);       // bounded drain of the products last committed
  }
  tc::tc_fence_before();
  __syncthreads();
  return ok;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gj_sweep_tc(const T* A, T* B, const T* Pk, T* Pn, int64_t n, int k,
                                                     const int* skip, int* info, int* tmo) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(1024) unsigned char sw_smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase_s;
  const int nt = int((n + GJB - 1) / GJB);
  if (blockIdx.x == 0) {                          // the pivot of sweep k + 1
    if (k + 1 < nt) pivot_next_wide<T>(A, n, k, Pk, Pn, info, sw_smem);
    return;
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&tbase_s, 256);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tb = tbase_s;
  sweep_tile<T>(A, B, Pk, n, k, int(blockIdx.x) - 1, sw_smem, &bar, tb, info, tmo);
  if (threadIdx.x < 32) tc::tmem_dealloc(tb, 256);
}

// The first pivot after the one-launch elimination of the leading identity
// block (k0 panels), formed from the matrix before that elimination:
//     X = A[k0, k0] - sum_{c < k0} A[k0, c] A[c, k0]
// (the identity block's own pivot is I), inverted, X^{-1} into Pinv.  It
// depends on the input alone, so it runs on the side stream while the
// identity elimination runs (n % 4 == 0).  256 threads: group g (warps
// 4g .. 4g + 3) sums the blocks c = g, g + 2, ... in the 4 x 8 layout of the
// inversion, each group with its own operand buffers and named barrier
// (2 + g); group 1's sum is added through shared memory and group 0 inverts.
constexpr int kPivIdentSmem = (5 * GJB * GJP + 4 * GJB) * 4 + 16;
template <typename T>
__global__ void __launch_bounds__(256) k_gj_pivot_ident(const T* A, int64_t n, int k0, T* Pinv, int* info,
                                                        const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char pi_smem[];
  float (*Ts)[GJP] = reinterpret_cast<float (*)[GJP]>(pi_smem);
  const int tid = threadIdx.x, grp = tid >> 7, lt = tid & 127, bi = lt % 16, bj = lt / 16;
  float (*Lc)[GJP] = Ts + GJB * (1 + 2 * grp);       // A[k0, c], by columns
  float (*Rc)[GJP] = Lc + GJB;                       // A[c, k0], by columns
  float (*prow)[GJB] = reinterpret_cast<float (*)[GJB]>(Ts + 5 * GJB);
  float (*pcol)[GJB] = prow + 2;
  int* bad = reinterpret_cast<int*>(pcol + 2);
  const int kb = int((n - int64_t(k0) * GJB) < GJB ? (n - int64_t(k0) * GJB) : GJB);
  const int64_t o = int64_t(k0) * GJB;
  float x[4][8];
  if (grp == 0) load_block(A, n, o, o, x);
  else zero_block(x);
  for (int c = grp; c < k0; c += 2) {
    const int64_t oc = int64_t(c) * GJB;
    copy_cols_async<128>(A, n, o, oc, Lc, lt);
    copy_cols_async<128>(A, n, oc, o, Rc, lt);
    cp_async_commit();
    cp_async_wait<0>();
    asm volatile("bar.sync %0, 128;\n" ::"r"(2 + grp) : "memory");
    tile_fma_cc_k32<-1>(Lc, Rc, x, bi, bj, 0);
    tile_fma_cc_k32<-1>(Lc, Rc, x, bi, bj, 32);
    asm volatile("bar.sync %0, 128;\n" ::"r"(2 + grp) : "memory");   // buffers free for the next block
  }
  if (grp == 1) tile_put_cols(x, Ts, bi, bj);
  __syncthreads();
  if (grp == 0) {
    tile_add_cols(x, Ts, bi, bj);
    pad_identity(x, kb);
    pivot_store<true>(x, n, k0, kb, Pinv, nullptr, info, prow, pcol, bad);
  }
}

// Invert the n x n SPD matrix A (full storage, column-major); B is the second
// buffer and pinv holds 2 GJB x GJB blocks.  *result receives the buffer with
// the inverse.  When the leading `ident` rows/columns of A are the identity,
// the first ident / GJB sweeps are replaced by one block elimination.  With
// side != null the pivot of sweep k + 1 is inverted on `side` while sweep k's
// row panel and update run on s (fork/join through ev_fork / ev_join,
// graph-capturable).  The tensor-core path (n % 4 == 0, n >= kUtMinN or
// tc_mode == 1) runs a sweep as one k_gj_sweep_tc launch while its 1 + mt^2
// CTAs fit on the GPU at once.  (All sweeps in one launch, separated by grid
// barriers on global sync words, measured slower: 253 against 240 us at
// n = 1200 from the first sweep.)
template <typename T>
int gj_invert(T* A, T* B, T* pinv, int64_t n, int64_t ident, int* info, const int* skip, cudaStream_t s,
              cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join, T** result, int tc_mode) {
  // the rank-64 updates on the tensor cores from n = kUtMinN (tc_mode < 0),
  // or as tc_mode says (0: SIMT, 1: tensor cores)
  const bool use_tc = n % 4 == 0 && (tc_mode < 0 ? (n >= kUtMinN) : (tc_mode != 0));
  // one launch per sweep (k_gj_sweep_tc) while its 1 + mt^2 CTAs fit on the
  // GPU at once; beyond that each of its CTAs recomputing its slice of the
  // row panel costs more than a row-panel launch (n = 2700, 485 CTAs: 1.16
  // against 1.11 ms per inverse), and the sweep runs as row panel +
  // k_gj_update2_tc with the pivot on the side stream
  const unsigned mt = unsigned((n + kUtM - 1) / kUtM);
  int nsm = 0, dev = 0;
  if (use_tc && (cudaGetDevice(&dev) != cudaSuccess ||
                 cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
    return CP_ECUDA;
  const bool fused = use_tc && 1 + int64_t(mt) * mt <= nsm;
  int* tmo = nullptr;
  if (use_tc) {
    if (tc_timeout_counter(&tmo) != CP_OK) return CP_ECUDA;
    if (cudaFuncSetAttribute(k_gj_update_tc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUtSmemAll) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_gj_sweep_tc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSwSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_gj_update2_tc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUtSmem) !=
            cudaSuccess)
      return CP_ECUDA;
  }
  if (side && (cudaFuncSetAttribute(k_gj_pivot_next<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kPivotReserve) != cudaSuccess ||
               cudaFuncSetAttribute(k_gj_pivot_next<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kPivotReserve) != cudaSuccess))
    return CP_ECUDA;
  const int nt = int((n + GJB - 1) / GJB);
  T* src = A;
  T* dst = B;
  int k0 = int(ident / GJB);
  if (k0 >= nt) k0 = nt - 1;
  // with one-launch sweeps the first pivot is formed from the input on the
  // side stream while the identity block is eliminated
  const bool pivot0_side = fused && side && k0 > 0;
  if (k0 > 0) {
    if (n % 4 == 0) {
      if (cudaFuncSetAttribute(k_gj_identity<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kIdentSmem) != cudaSuccess)
        return CP_ECUDA;
      if (pivot0_side) {
        if (cudaFuncSetAttribute(k_gj_pivot_ident<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kPivIdentSmem) != cudaSuccess ||
            cudaEventRecord(ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(side, ev_fork, 0) != cudaSuccess)
          return CP_ECUDA;
        k_gj_pivot_ident<T><<<1, 256, kPivIdentSmem, side>>>(src, n, k0, pinv + size_t(k0 & 1) * GJB * GJB, info,
                                                             skip);
        if (cudaEventRecord(ev_join, side) != cudaSuccess) return CP_ECUDA;
      }
      if (launch_pdl(k_gj_identity<T, true>, nt * nt * 2, GJTH, kIdentSmem, s, src, dst, n, k0, use_tc ? 1 : 0,
                     skip) != cudaSuccess)
        return CP_ECUDA;
      if (use_tc) {
        const int64_t base = int64_t(k0) * GJB;
        const unsigned t = unsigned((n - base + kUtM - 1) / kUtM);
        if (launch_pdl(k_gj_update_tc<T>, dim3(t, t), 256, kUtSmemAll, s, static_cast<const T*>(src), dst, n, base,
                       k0, skip, info, tmo) != cudaSuccess)
          return CP_ECUDA;
      }
    } else {
      if (launch_pdl(k_gj_identity<T, false>, nt * nt * 2, GJTH, (GJB * GJP + GJB * (GJH + 4)) * 4, s, src, dst, n,
                     k0, 0, skip) != cudaSuccess)
        return CP_ECUDA;
    }
    T* t = src;
    src = dst;
    dst = t;
  }
  if (pivot0_side) {
    if (cudaStreamWaitEvent(s, ev_join, 0) != cudaSuccess) return CP_ECUDA;
  } else if (launch_pdl(k_gj_pivot<T>, 1, GJT, 0, s, src, dst, n, k0, pinv + size_t(k0 & 1) * GJB * GJB, info,
                        skip) != cudaSuccess) {
    return CP_ECUDA;
  }
  for (int k = k0; k < nt; ++k) {
    T* pk = pinv + size_t(k & 1) * GJB * GJB;
    T* pn = pinv + size_t((k + 1) & 1) * GJB * GJB;
    if (nt > 1 && fused) {
      // one launch per sweep: the next pivot in CTA 0, the row panel and the update in the others
      if (launch_pdl(k_gj_sweep_tc<T>, 1 + mt * mt, 256, kSwSmem, s, static_cast<const T*>(src), dst,
                     static_cast<const T*>(pk), pn, n, k, skip, info, tmo) != cudaSuccess)
        return CP_ECUDA;
    } else if (nt > 1) {
      const bool next = (k + 1 < nt);
      if (next && side) {
        if (cudaEventRecord(ev_fork, s) != cudaSuccess) return CP_ECUDA;
        if (cudaStreamWaitEvent(side, ev_fork, 0) != cudaSuccess) return CP_ECUDA;
        if (n % 4 == 0) k_gj_pivot_next<T, true><<<1, GJT, kPivotReserve, side>>>(src, n, k, pk, pn, info, skip);
        else k_gj_pivot_next<T, false><<<1, GJT, kPivotReserve, side>>>(src, n, k, pk, pn, info, skip);
        if (cudaEventRecord(ev_join, side) != cudaSuccess) return CP_ECUDA;
      }
      if (use_tc) {
        if (launch_pdl(k_gj_rowpanel<T, true>, (nt - 1) * 2, GJTH, kTileSmem, s, src, dst, n, k, pk, skip) !=
                cudaSuccess ||
            launch_pdl(k_gj_update2_tc<T>, dim3(mt, mt), 256, kUtSmem, s, static_cast<const T*>(src), dst, n, k,
                       (next && side) ? 1 : 0, skip, info, tmo) != cudaSuccess)
          return CP_ECUDA;
      } else if (n % 4 == 0) {
        if (launch_pdl(k_gj_rowpanel<T, true>, (nt - 1) * 2, GJTH, kTileSmem, s, src, dst, n, k, pk, skip) !=
                cudaSuccess ||
            launch_pdl(k_gj_update<T, true>, (nt - 1) * nt * 2, GJTH, kTileSmem, s, src, dst, n, k, pk,
                       (next && side) ? 1 : 0, skip) != cudaSuccess)
          return CP_ECUDA;
      } else {
        if (launch_pdl(k_gj_rowpanel<T, false>, (nt - 1) * 2, GJTH, kTileSmem, s, src, dst, n, k, pk, skip) !=
                cudaSuccess ||
            launch_pdl(k_gj_update<T, false>, (nt - 1) * nt * 2, GJTH, kTileSmem, s, src, dst, n, k, pk,
                       (next && side) ? 1 : 0, skip) != cudaSuccess)
          return CP_ECUDA;
      }
      if (next && side) {
        if (cudaStreamWaitEvent(s, ev_join, 0) != cudaSuccess) return CP_ECUDA;
      } else if (next) {
        if (launch_pdl(k_gj_pivot<T>, 1, GJT, 0, s, dst, src, n, k + 1, pn, info, skip) != cudaSuccess)
          return CP_ECUDA;
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
                               cudaStream_t, cudaEvent_t, cudaEvent_t, float**, int);

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
  pdl_enter();
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
  CP_CUDA(launch_pdl(k_gemv_acc, g, GVT, 0, s, X, n, r, y, b2, r2, r2prev, done, tol2, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn

// One side stream and a fork/join event pair for every cp_spd_invert_f32
// call of the process, created on first use; calls are serialised by the
// mutex while they enqueue (the device work of consecutive calls on
// different streams is ordered by the events).
static std::mutex g_inv_mu;
static cudaStream_t g_inv_side = nullptr;
static cudaEvent_t g_inv_fork = nullptr, g_inv_join = nullptr;

extern "C" int cp_spd_invert_f32(int64_t n, int64_t ident, float* A, float* work, float* pinv, int* info,
                                 int* in_work, void* stream) {
  if (!A || !work || !pinv || !in_work || n < 1 || ident < 0 || ident > n) return CP_EINVAL;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(work) & 15)) return CP_EINVAL;
  std::lock_guard<std::mutex> lock(g_inv_mu);
  if (!g_inv_side) {
    if (cudaStreamCreateWithFlags(&g_inv_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g_inv_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g_inv_join, cudaEventDisableTiming) != cudaSuccess)
      return CP_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (info && cudaMemsetAsync(info, 0, sizeof(int), s) != cudaSuccess) return CP_ECUDA;
  float* res = nullptr;
  const int rc = cpdgn::gj_invert<float>(A, work, pinv, n, ident, info, nullptr, s, g_inv_side, g_inv_fork,
                                         g_inv_join, &res, -1);
  if (rc != CP_OK) return rc;
  *in_work = (res == work) ? 1 : 0;
  return CP_OK;
}
