// Float64 Cholesky factorisation of the N R^2 x N R^2 core system and the two
// triangular solves of the core solve (Theorem 1, Eq. inverse_f1a, in the
// symmetric positive definite form core = I + S^T K S).  Column-major, lower
// triangle; the upper triangle is never read and is left unspecified.
//
// GB300 runs float64 at 2 multiply-adds per clock per SM with ~40 cycles of
// latency, so the design spreads every panel's work over all SMs and keeps
// the number of launches small:
//
//  k_chol64 (one persistent launch, one CTA per SM, blocked right-looking
//  with 32-wide panels and a one-tile lookahead).  Per panel k:
//    phase A  every CTA solves its share of the panel's rows
//             X <- X L_kk^{-T} (one warp per row, lane = column) with the
//             stored factor L_kk of the diagonal tile;
//    phase B  the trailing update A_ij -= L_ik L_jk^T over 32 x 32 tiles of
//             the lower triangle: CTA 0 updates the next diagonal tile and
//             factors it (the whole CTA, see factor_tile), storing L_{k+1,k+1},
//             while the other tiles are dealt round-robin to the other CTAs;
//  separated by grid barriers (an arrival counter and a generation word in
//  the workspace, every wait bounded).  Finally each diagonal tile's inverse
//  L_cc^{-1} is written to `dinv` for the solves.
//
//  k_trsv64 (one launch per direction, dataflow).  CTA t takes block row
//  c = t (forward) or nb - 1 - t (backward) from an atomic ticket, so a CTA
//  only ever waits on block rows taken by CTAs that started before it; it
//  accumulates the off-diagonal products of the block rows already published
//  (each wait bounded), multiplies by L_cc^{-1} (or its transpose) and
//  publishes its block with a flag.
//
// A non-positive or non-finite pivot records its 1-based index in *info
// (first one wins) and the factorisation continues with the pivot replaced
// by 1, so no NaN is produced; a wait that runs out sets the abort word, adds
// one to the caller's timeout counter, makes every CTA return, and sets *info
// to n + 1 so that the result is never used as a factor.
#include "common.cuh"

namespace cpdgn {

constexpr int CB = 32;                           // panel / tile width
constexpr int CT = 256;                          // threads per CTA (8 warps)
constexpr uint64_t kWaitNs = 2000000000ull;      // every wait gives up after 2 s

__device__ __forceinline__ uint64_t chol_gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sync words of the factorisation and the solves, in the workspace.  Zeroed
// (cudaMemsetAsync) before every launch that uses them.
struct CholSync {
  unsigned count;        // grid barrier: CTAs arrived
  unsigned gen;          // grid barrier: generation
  int abort;             // set when a wait ran out
  int ticket;            // block-row ticket of a solve
  int flags[1];          // solve: block row published (nb entries)
};

size_t chol64_sync_bytes(int64_t n) { return sizeof(CholSync) + sizeof(int) * size_t((n + CB - 1) / CB); }
size_t chol64_dinv_bytes(int64_t n) { return sizeof(double) * CB * CB * size_t((n + CB - 1) / CB); }

__device__ void chol_fail(CholSync* sy, int* info, int64_t n, int* tmo) {
  if (atomicExch(&sy->abort, 1) == 0) {
    if (tmo) atomicAdd(tmo, 1);
  }
  if (info) atomicExch(info, int(n + 1));
}

// Grid-wide barrier of the G co-resident CTAs of k_chol64; false if aborted.
__device__ bool grid_barrier(CholSync* sy, unsigned G, unsigned& epoch, int* info, int64_t n, int* tmo) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned target = epoch + 1;
    int ok = 1;
    if (atomicAdd(&sy->count, 1u) == G - 1) {
      sy->count = 0;                 // nobody arrives again before gen moves
      __threadfence();
      atomicExch(&sy->gen, target);
    } else {
      const uint64_t t0 = chol_gtimer();
      for (;;) {
        if (int(*reinterpret_cast<volatile unsigned*>(&sy->gen) - target) >= 0) break;
        if (*reinterpret_cast<volatile int*>(&sy->abort)) { ok = 0; break; }
        if (chol_gtimer() - t0 > kWaitNs) {
          chol_fail(sy, info, n, tmo);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    epoch = target;
    s_ok = ok && !*reinterpret_cast<volatile int*>(&sy->abort);
  }
  __syncthreads();
  return s_ok != 0;
}

// 1 / d for d > 0 (finite) by Newton's iteration for the reciprocal,
// x <- x (2 - d x), written as x + x (1 - d x), from the hardware's
// approximate double reciprocal: two iterations take its ~2^-20 relative
// error below the rounding of a double, in four dependent multiply-adds.
__device__ __forceinline__ double recip64(double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  x = fma(x, fma(-d, x, 1.0), x);
  x = fma(x, fma(-d, x, 1.0), x);
  return x;
}

// Factor the kb x kb tile D (lower part) in place with the whole CTA.
// Column j of the elimination needs only the reciprocal of its pivot:
// D[i][k] -= D[i][j] D[k][j] / D[j][j] for j < k <= i, with column j itself
// left unscaled; the square roots L_jj = sqrt(d_j), L_ij = D[i][j] / sqrt(d_j)
// and rinv[j] = 1 / L_jj are formed at the end for all columns at once.
//
// On this part every float64 warp instruction holds the SM's float64 units
// for about 16 clocks, so the work of a column is packed into as few warps as
// possible: the packed lower-triangle entries are numbered column by column
// from the last column down (k = 31 first), so the entries still to update
// at column j (k > j) are a prefix of the numbering and the warps beyond it
// skip the column.  The reciprocal of the next pivot is formed once, by the
// thread that updates that pivot, and shared through shared memory.
// Thread t owns entries t, t + CT, t + 2 CT.  Returns the first bad pivot
// (1-based) or 0; every thread gets it.
__device__ int factor_tile(double (*D)[CB + 1], int kb, double* rinv) {
  constexpr int NE = CB * (CB + 1) / 2;           // 528 packed entries
  constexpr int PER = (NE + CT - 1) / CT;         // 3
  __shared__ double s_q[CB];
  __shared__ int s_fbad;
  int ei[PER], ek[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int e = int(threadIdx.x) + q * CT, i = -1, k = -1;
    if (e < NE) {                                  // column k holds 32 - k entries
      k = CB - 1;
      while (e >= CB - k) { e -= CB - k; --k; }
      i = k + e;
    }
    ei[q] = i;
    ek[q] = k;
  }
  // rows / columns beyond kb: identity, so the padded tile factors trivially
#pragma unroll
  for (int q = 0; q < PER; ++q)
    if (ei[q] >= kb) D[ei[q]][ek[q]] = (ei[q] == ek[q]) ? 1.0 : 0.0;
  if (threadIdx.x == 0) s_fbad = 0;
  __syncthreads();
  // reciprocal of pivot 0 (an invalid pivot is recorded and replaced by 1)
  if (threadIdx.x == 0) {
    double d = D[0][0];
    if (!(d > 0.0) || !isfinite(d)) {
      s_fbad = 1;
      d = 1.0;
    }
    s_q[0] = recip64(d);
  }
  __syncthreads();
  for (int j = 0; j < CB - 1; ++j) {
    const double qj = s_q[j];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int i = ei[q], k = ek[q];
      if (k > j) {
        const double v = fma(-D[i][j] * qj, D[k][j], D[i][k]);
        D[i][k] = v;
        if (i == j + 1 && k == j + 1) {            // the next pivot: its reciprocal now
          double d = v;
          if (!(d > 0.0) || !isfinite(d)) {
            if (s_fbad == 0) s_fbad = j + 2;
            d = 1.0;
          }
          s_q[j + 1] = recip64(d);
        }
      }
    }
    __syncthreads();
  }
  // square roots of the pivots, then the columns
  if (threadIdx.x < CB) {
    double d = D[threadIdx.x][threadIdx.x];
    if (!(d > 0.0) || !isfinite(d)) d = 1.0;
    rinv[threadIdx.x] = rsqrt(d);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = ei[q], k = ek[q];
    if (i >= 0) {
      const double v = D[i][k];
      D[i][k] = (i == k) ? ((v > 0.0 && isfinite(v)) ? v * rinv[k] : 1.0) : v * rinv[k];
    }
  }
  __syncthreads();
  const int bad = s_fbad;
  return (bad > 0 && bad <= kb) ? bad : 0;
}

// CTA 0 factors the diagonal tile kk of A (lower part, already fully
// updated) in shared memory and stores L_kk in its place, 1 / L_jj into the
// diagonal of dinv's tile kk and a bad pivot into *info.
__device__ void factor_store(double* A, int64_t n, int kk, double* dinv, int* info, double (*D)[CB + 1],
                             double* rinv) {
  const int64_t k0 = int64_t(kk) * CB;
  const int kb = int((n - k0) < CB ? (n - k0) : CB);
  for (int e = threadIdx.x; e < CB * CB; e += CT) {
    const int i = e % CB, j = e / CB;
    D[i][j] = (i < kb && j <= i) ? A[(k0 + i) + n * (k0 + j)] : 0.0;
  }
  __syncthreads();
  const int bad = factor_tile(D, kb, rinv);
  if (threadIdx.x == 0 && bad && info) atomicCAS(info, 0, int(k0) + bad);
  for (int e = threadIdx.x; e < kb * kb; e += CT) {
    const int i = e % kb, j = e / kb;
    if (j <= i) A[(k0 + i) + n * (k0 + j)] = D[i][j];
  }
  if (threadIdx.x < CB) dinv[int64_t(kk) * CB * CB + threadIdx.x * (CB + 1)] = rinv[threadIdx.x];
}

// Lookahead: the diagonal tile of panel k + 1 is the first tile of panel k's
// trailing update; CTA 0 updates it, factors it and stores L_{k+1,k+1} while
// the other CTAs update the rest of the trailing matrix, so the diagonal
// factorisation (about 17 us) leaves the critical path whenever the rest of
// the update takes longer.  Panel k's rows below the diagonal are then solved
// by every CTA from the stored L_kk.
__global__ void __launch_bounds__(CT) k_chol64(double* A, int64_t n, double* dinv, int* info, CholSync* sy,
                                               int* tmo, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double D[CB][CB + 1];
  __shared__ double rinv[CB];
  __shared__ double Pi[CB][CB + 1], Pj[CB][CB + 1];
  const unsigned G = gridDim.x;
  const int cta = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = int((n + CB - 1) / CB);
  unsigned epoch = 0;
  if (cta == 0) factor_store(A, n, 0, dinv, info, D, rinv);
  if (!grid_barrier(sy, G, epoch, info, n, tmo)) return;
  for (int k = 0; k < nb; ++k) {
    const int64_t k0 = int64_t(k) * CB;
    const int kb = int((n - k0) < CB ? (n - k0) : CB);
    // ---- phase A: panel solve X <- X L_kk^{-T} with the stored L_kk ----
    if (k0 + kb < n) {
      for (int e = tid; e < CB * CB; e += CT) {
        const int i = e % CB, j = e / CB;
        D[i][j] = (i < kb && j <= i) ? A[(k0 + i) + n * (k0 + j)] : 0.0;
      }
      if (tid < CB) rinv[tid] = tid < kb ? dinv[int64_t(k) * CB * CB + tid * (CB + 1)] : 0.0;
      __syncthreads();
      for (int64_t r = k0 + kb + int64_t(cta) * 8 + warp; r < n; r += int64_t(G) * 8) {
        double x = lane < kb ? A[r + n * (k0 + lane)] : 0.0;
#pragma unroll 8
        for (int j = 0; j < kb; ++j) {
          const double xj = __shfl_sync(0xffffffffu, x, j) * rinv[j];
          if (lane == j) x = xj;
          else if (lane > j) x = fma(-xj, D[lane][j], x);
        }
        if (lane < kb) A[r + n * (k0 + lane)] = x;
      }
    }
    if (k + 1 == nb) break;
    if (!grid_barrier(sy, G, epoch, info, n, tmo)) return;
    // ---- phase B: trailing update of the lower triangle ----
    // tile e = 0 is (k + 1, k + 1): CTA 0 alone, then its factorisation;
    // tiles e >= 1 go to CTAs 1 .. G - 1 (to CTA 0 as well when G == 1)
    const int t = nb - k - 1;
    const int64_t T = int64_t(t) * (t + 1) / 2;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t e0 = (G == 1) ? 0 : (cta == 0 ? 0 : cta);
    const int64_t es = (G == 1) ? 1 : (cta == 0 ? T : int64_t(G) - 1);
    for (int64_t e = e0; e < T; e += es) {
      int ti = int((sqrt(8.0 * double(e) + 1.0) - 1.0) * 0.5);
      while (int64_t(ti + 1) * (ti + 2) / 2 <= e) ++ti;
      while (int64_t(ti) * (ti + 1) / 2 > e) --ti;
      const int tj = int(e - int64_t(ti) * (ti + 1) / 2);
      const int64_t r0 = int64_t(k + 1 + ti) * CB, c0 = int64_t(k + 1 + tj) * CB;
      for (int q = tid; q < CB * CB; q += CT) {
        const int i = q % CB, l = q / CB;
        Pi[i][l] = (r0 + i < n) ? A[(r0 + i) + n * (k0 + l)] : 0.0;
        Pj[i][l] = (c0 + i < n) ? A[(c0 + i) + n * (k0 + l)] : 0.0;
      }
      __syncthreads();
      double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll 8
      for (int l = 0; l < CB; ++l) {
        const double a0 = Pi[tx][l], a1 = Pi[tx + 16][l], b0 = Pj[ty][l], b1 = Pj[ty + 16][l];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int64_t r = r0 + tx + 16 * u, c = c0 + ty + 16 * v;
          if (r < n && c < n && r >= c) A[r + n * c] -= acc[u][v];
        }
      __syncthreads();
      if (e == 0) factor_store(A, n, k + 1, dinv, info, D, rinv);   // CTA 0: L_{k+1,k+1}
    }
    if (!grid_barrier(sy, G, epoch, info, n, tmo)) return;
  }
  // every L_kk and 1 / L_jj was stored, and every read of them in a panel
  // solve finished, before the last barrier of the loop
  // ---- inverses of the diagonal tiles: warps 0-2 of each CTA, one tile each ----
  if (warp < 3) {
    double (*Lt)[CB + 1] = warp == 0 ? D : (warp == 1 ? Pi : Pj);
    for (int c = cta * 3 + warp; c < nb; c += int(G) * 3) {
      const int64_t c0 = int64_t(c) * CB;
      const int cb = int((n - c0) < CB ? (n - c0) : CB);
      for (int q = lane; q < CB * CB; q += 32) {
        const int i = q % CB, l = q / CB;
        Lt[i][l] = (i < cb && l < cb && l <= i) ? A[(c0 + i) + n * (c0 + l)] : (i == l ? 1.0 : 0.0);
      }
      __syncwarp();
      double* Xc = dinv + int64_t(c) * CB * CB;
      const double ri = (lane < cb) ? Xc[lane * (CB + 1)] : 1.0;     // 1 / L_ii, lane i
      __syncwarp();
      // lane j: column j of L^{-1} by forward substitution, x_i = 0 for i < j
      double x[CB];
#pragma unroll
      for (int i = 0; i < CB; ++i) {
        const double rii = __shfl_sync(0xffffffffu, ri, i);
        if (i < lane) {
          x[i] = 0.0;
        } else if (i == lane) {
          x[i] = rii;
        } else {
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
          for (int l = 0; l < i; l += 4) {
            s0 = fma(Lt[i][l], x[l], s0);
            if (l + 1 < i) s1 = fma(Lt[i][l + 1], x[l + 1], s1);
            if (l + 2 < i) s2 = fma(Lt[i][l + 2], x[l + 2], s2);
            if (l + 3 < i) s3 = fma(Lt[i][l + 3], x[l + 3], s3);
          }
          x[i] = -((s0 + s1) + (s2 + s3)) * rii;
        }
      }
#pragma unroll
      for (int i = 0; i < CB; ++i) Xc[i + CB * lane] = x[i];
      __syncwarp();
    }
  }
}

// Forward (L z = b) or backward (L^T y = b) solve with the factor and the
// diagonal-tile inverses of k_chol64.  One CTA per block row (ticket order).
__global__ void __launch_bounds__(CT) k_trsv64(const double* L, const double* dinv, int64_t n, const double* b,
                                               double* x, int backward, CholSync* sy, int* info, int* tmo,
                                               const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ int s_c;
  __shared__ double part[8][CB];
  __shared__ double rr[CB];
  __shared__ double Xs[CB][CB + 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = int((n + CB - 1) / CB);
  if (tid == 0) s_c = atomicAdd(&sy->ticket, 1);
  __syncthreads();
  const int t = s_c;
  if (t >= nb) return;
  const int c = backward ? nb - 1 - t : t;
  const int64_t c0 = int64_t(c) * CB;
  const int cb = int((n - c0) < CB ? (n - c0) : CB);
  // the diagonal tile's inverse and the right-hand side do not depend on
  // any other block: fetch them before the first wait
  {
    const double* Xc = dinv + int64_t(c) * CB * CB;
    for (int e = tid; e < CB * CB; e += CT) Xs[e % CB][e / CB] = Xc[e];
  }
  const double bl = (tid < cb) ? b[c0 + tid] : 0.0;
  double acc = 0.0;                // forward: row c0 + lane; backward: outputs 4 warp .. 4 warp + 3
  double accb[4] = {0.0, 0.0, 0.0, 0.0};
  bool ok = true;
  const int j_lo = backward ? c + 1 : 0, j_hi = backward ? nb : c;
  for (int jj = j_lo; jj < j_hi && ok; ++jj) {
    const int j = backward ? (nb - 1 - (jj - j_lo)) : jj;     // wait in publication order
    const int64_t j0 = int64_t(j) * CB;
    const int jb = int((n - j0) < CB ? (n - j0) : CB);
    // this thread's entries of the off-diagonal tile, loaded before the wait
    double lv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int l = 4 * warp + q;
      if (!backward) lv[q] = (l < jb && lane < cb) ? L[(c0 + lane) + n * (j0 + l)] : 0.0;
      else lv[q] = (l < cb && lane < jb) ? L[(j0 + lane) + n * (c0 + l)] : 0.0;
    }
    if (lane == 0) {
      const uint64_t t0 = chol_gtimer();
      for (int it = 0;; ++it) {
        if (*reinterpret_cast<volatile int*>(&sy->flags[j])) break;
        if (*reinterpret_cast<volatile int*>(&sy->abort)) { ok = false; break; }
        if ((it & 63) == 63 && chol_gtimer() - t0 > kWaitNs) {
          chol_fail(sy, info, n, tmo);
          ok = false;
          break;
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (!ok) break;
    __threadfence();
    if (!backward) {
      // acc(row c0 + lane) += sum over this warp's 4 columns l of L[c0 + lane, j0 + l] x[j0 + l]
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * warp + q;
        if (l < jb) acc = fma(lv[q], __ldcg(x + j0 + l), acc);
      }
    } else {
      // output i = 4 warp + q: sum over rows l (= lane) of L[j0 + l, c0 + i] x[j0 + l]
      const double xl = lane < jb ? __ldcg(x + j0 + lane) : 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) accb[q] = fma(lv[q], xl, accb[q]);
    }
  }
  if (!backward) {
    part[warp][lane] = acc;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = accb[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) part[0][4 * warp + q] = v;
    }
  }
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(&sy->abort)) return;
  if (tid < CB) {
    double sum = 0.0;
    if (!backward) {
      for (int w = 0; w < 8; ++w) sum += part[w][tid];
    } else {
      sum = part[0][tid];
    }
    rr[tid] = tid < cb ? bl - sum : 0.0;
  }
  __syncthreads();
  if (tid < CB) {
    double s0 = 0.0, s1 = 0.0;
    if (!backward) {
#pragma unroll 8
      for (int l = 0; l < CB; l += 2) {
        s0 = fma(Xs[tid][l], rr[l], s0);
        s1 = fma(Xs[tid][l + 1], rr[l + 1], s1);
      }
    } else {
#pragma unroll 8
      for (int l = 0; l < CB; l += 2) {
        s0 = fma(Xs[l][tid], rr[l], s0);
        s1 = fma(Xs[l + 1][tid], rr[l + 1], s1);
      }
    }
    if (tid < cb) x[c0 + tid] = s0 + s1;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) atomicExch(&sy->flags[c], 1);
}

static int chol64_grid() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
      sms = kSMs;
  }
  return sms;
}

// Factor A = L L^T in place (lower triangle), L_cc^{-1} into dinv.
// sync: chol64_sync_bytes(n) bytes of workspace; tmo: device timeout counter.
int chol64_factor(double* A, int64_t n, double* dinv, int* info, void* sync, int* tmo, const int* skip,
                  cudaStream_t s) {
  if (n < 1) return CP_EINVAL;
  CholSync* sy = static_cast<CholSync*>(sync);
  if (cudaMemsetAsync(sy, 0, sizeof(CholSync), s) != cudaSuccess) return CP_ECUDA;
  const int nb = int((n + CB - 1) / CB);
  int G = chol64_grid();
  // enough CTAs for the widest phase, at most one per SM (they must all be
  // resident at once for the grid barrier)
  int64_t want = int64_t(nb) * (nb - 1) / 2;
  const int64_t rows = (n + 7) / 8;
  if (rows > want) want = rows;
  if (want < 1) want = 1;
  if (G > want) G = int(want);
  CP_CUDA(launch_pdl(k_chol64, G, CT, 0, s, A, n, dinv, info, sy, tmo, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

// y = (L L^T)^{-1} b with the factor of chol64_factor; z: n doubles of scratch.
int chol64_solve(const double* L, const double* dinv, int64_t n, const double* b, double* z, double* y,
                 void* sync, int* info, int* tmo, const int* skip, cudaStream_t s) {
  CholSync* sy = static_cast<CholSync*>(sync);
  const int nb = int((n + CB - 1) / CB);
  if (cudaMemsetAsync(sy, 0, chol64_sync_bytes(n), s) != cudaSuccess) return CP_ECUDA;
  CP_CUDA(launch_pdl(k_trsv64, nb, CT, 0, s, L, dinv, n, b, z, 0, sy, info, tmo, skip));
  if (cudaMemsetAsync(sy, 0, chol64_sync_bytes(n), s) != cudaSuccess) return CP_ECUDA;
  CP_CUDA(launch_pdl(k_trsv64, nb, CT, 0, s, L, dinv, n, z, y, 1, sy, info, tmo, skip));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn
