// All-mode MTTKRP and direct residual in one pass over the tensor.
//
//   M_n = Y_(n) (A^(N) (.) ... A^(n+1) (.) A^(n-1) (.) ... A^(1))     (Algorithm 1 step 6)
//   ||E||^2 = sum (Y - Y_hat)^2                                        (Sec. 4.6, e_t)
//
// Y is streamed once as mode-1 fibres (columns of Y_(1), contiguous in
// memory).  For fibre f with multi-index (i_2..i_N):
//   kr_f[r]   = prod_{k>=2} A^(k)[i_k, r]          (row f of KR_1)
//   t_f[r]    = sum_i Y[i, f] A^(1)[i, r]           (row f of Y_(1)^T A^(1))
//   M_1      += y_f kr_f^T
//   M_n[i_n] += t_f * prod_{k>=2, k!=n} A^(k)[i_k]   (n >= 2: reuse of t_f, the
//                                                    partial Khatri-Rao product)
//   e         = y_f - A^(1) kr_f,  ||E||^2 += e^T e
// so each tensor element costs 3R multiply-adds whatever N is.  With `grad`
// set, e = y - y_hat is formed first and takes the place of y in M_1 and t_f,
// so the pass gives the gradient blocks G_n = E_(n) KR_n = M_n - A^(n) Gamma^(n)
// (Sec. 4.6, g = J^T vec(E)) with rounding relative to E rather than to Y.
// A CTA owns a
// contiguous range of fibres and keeps its partial M_1 (and M_n, n >= 2, when
// they fit) in shared memory; partials are added to the float64 outputs at
// the end.  TA is the arithmetic type: float64 for float64 tensors, float32
// for float32 and bfloat16 tensors (with float64 accumulation of ||E||^2 per
// tile and of the cross-CTA sums).
#include <type_traits>

#include "common.cuh"

namespace cpdgn {

struct MttkrpParams {
  Dims d;
  const void* Y;
  const double* a;
  double* m;             // zeroed R*T output (may be null: fit only)
  double* resid2;        // zeroed scalar (may be null)
  const int* skip;       // device flag: nonzero -> return at once (may be null)
  int64_t fib_per_cta;
  int TF;                // fibres per tile
  int mn_in_smem;        // 1: partial M_n (n >= 2) in shared memory
  int I1p;               // padded leading dimension of the tile
  int grad;              // 1: accumulate e = y - y_hat instead of y (gradient blocks)
};

constexpr int kMtThreads = 256;

template <typename TY, typename TA, int RMAX>
__global__ void __launch_bounds__(kMtThreads) k_mttkrp(MttkrpParams p) {
  pdl_enter();
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int R = d.R;
  const int N = d.N;
  const int I1 = int(d.I[0]);
  const int TF = p.TF;
  const int tid = threadIdx.x;
  const bool want_m = p.m != nullptr;
  const bool want_e = p.resid2 != nullptr;

  // shared-memory carve-up (all TA unless noted)
  TA* A1s = reinterpret_cast<TA*>(smem_raw);                 // I1 x R, row-major [i][r]
  TA* M1s = A1s + size_t(I1) * R;                            // I1 x R
  TA* Yt = M1s + size_t(I1) * R;                             // TF x I1p  [f][i]
  TA* krs = Yt + size_t(TF) * p.I1p;                         // TF x R
  TA* ts = krs + size_t(TF) * R;                             // TF x R
  TA* loos = ts + size_t(TF) * R;                            // (N-1) x TF x R
  TA* Mns = loos + size_t(N - 1) * TF * R;                   // sum_{n>=2} I_n x R (optional)
  int64_t mn_elems = p.mn_in_smem ? (d.T - d.I[0]) * R : 0;
  int* fidx = reinterpret_cast<int*>(Mns + mn_elems);        // TF x CP_MAX_N
  double* red = reinterpret_cast<double*>(fidx + TF * CP_MAX_N + 2);  // kMtThreads (8-aligned below)
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 15) & ~uintptr_t(15));

  const double* a = p.a;
  for (int e = tid; e < I1 * R; e += kMtThreads) {
    int i = e / R, r = e % R;
    A1s[e] = TA(a[i + int64_t(r) * I1]);
    M1s[e] = TA(0);
  }
  for (int64_t e = tid; e < mn_elems; e += kMtThreads) Mns[e] = TA(0);
  // prefix offsets of modes >= 2 inside Mns
  int64_t mn_off[CP_MAX_N];
  {
    int64_t o = 0;
    for (int n = 1; n < N; ++n) { mn_off[n] = o; o += d.I[n] * R; }
  }
  __syncthreads();

  const int64_t f_begin = int64_t(blockIdx.x) * p.fib_per_cta;
  int64_t f_end = f_begin + p.fib_per_cta;
  if (f_end > d.nfib) f_end = d.nfib;
  double e2_total = 0.0;
  const TY* Y = reinterpret_cast<const TY*>(p.Y);

  for (int64_t f0 = f_begin; f0 < f_end; f0 += TF) {
    const int nf = int((f_end - f0) < TF ? (f_end - f0) : TF);
    // P0: tile of nf fibres, contiguous in memory
    {
      const int64_t base = f0 * I1;
      const int tot = nf * I1;
      int f = 0, i = tid;
      while (i >= I1 && f < nf) { i -= I1; ++f; }
      for (int e = tid; e < tot; e += kMtThreads) {
        Yt[f * p.I1p + i] = TA(load_y(Y, base + e));
        i += kMtThreads;
        while (i >= I1) { i -= I1; ++f; }
      }
    }
    // P1: fibre indices, Khatri-Rao rows and leave-one-out products
    for (int e = tid; e < nf * R; e += kMtThreads) {
      const int f = e / R, r = e % R;
      int64_t rem = f0 + f;
      TA v[CP_MAX_N];
      int idx[CP_MAX_N];
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k) {
        if (k < N) {
          idx[k] = int(rem % d.I[k]);
          rem /= d.I[k];
          v[k] = TA(a[d.aoff[k] + idx[k] + int64_t(r) * d.I[k]]);
        }
      }
      TA kr = TA(1);
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k)
        if (k < N) kr *= v[k];
      krs[f * R + r] = kr;
#pragma unroll
      for (int n = 1; n < CP_MAX_N; ++n) {
        if (n < N) {
          TA lo = TA(1);
#pragma unroll
          for (int k = 1; k < CP_MAX_N; ++k)
            if (k < N && k != n) lo *= v[k];
          loos[(size_t(n - 1) * TF + f) * R + r] = lo;
        }
      }
      if (r == 0) {
#pragma unroll
        for (int k = 1; k < CP_MAX_N; ++k)
          if (k < N) fidx[f * CP_MAX_N + k] = idx[k];
      }
    }
    __syncthreads();
    // P3: M_1 rows and the residual; one row per thread.  With p.grad the
    // tile entry is replaced by e = y - y_hat, which P2 and M_1 then use.
    for (int i = tid; i < I1; i += kMtThreads) {
      TA arow[RMAX], acc[RMAX];
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        arow[r] = (r < R) ? A1s[i * R + r] : TA(0);
        acc[r] = TA(0);
      }
      TA e2 = TA(0);
      for (int f = 0; f < nf; ++f) {
        const TA y = Yt[f * p.I1p + i];
        const TA* kf = krs + f * R;
        TA yh = TA(0);
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) yh = fma(arow[r], kf[r], yh);
        const TA e = y - yh;
        e2 = fma(e, e, e2);
        const TA src = p.grad ? e : y;
        if (p.grad) Yt[f * p.I1p + i] = e;
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) acc[r] = fma(src, kf[r], acc[r]);
      }
      e2_total += double(e2);
      if (want_m) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) M1s[i * R + r] += acc[r];
      }
    }
    __syncthreads();
    // P2: t_f = y_f^T A^(1) (or e_f^T A^(1)); needed only for M_n, n >= 2
    if (want_m) {
      for (int e = tid; e < nf * R; e += kMtThreads) {
        const int f = e / R, r = e % R;
        const TA* yf = Yt + f * p.I1p;
        TA s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        int i = 0;
        for (; i + 3 < I1; i += 4) {
          s0 = fma(yf[i], A1s[i * R + r], s0);
          s1 = fma(yf[i + 1], A1s[(i + 1) * R + r], s1);
          s2 = fma(yf[i + 2], A1s[(i + 2) * R + r], s2);
          s3 = fma(yf[i + 3], A1s[(i + 3) * R + r], s3);
        }
        for (; i < I1; ++i) s0 = fma(yf[i], A1s[i * R + r], s0);
        ts[f * R + r] = (s0 + s1) + (s2 + s3);
      }
    }
    // P4: M_n, n >= 2, from t_f and the leave-one-out products
    if (want_m) {
      for (int e = tid; e < nf * R; e += kMtThreads) {
        const int f = e / R, r = e % R;
        const TA t = ts[f * R + r];
#pragma unroll
        for (int n = 1; n < CP_MAX_N; ++n) {
          if (n < N) {
            const TA c = t * loos[(size_t(n - 1) * TF + f) * R + r];
            const int in = fidx[f * CP_MAX_N + n];
            if (p.mn_in_smem)
              atomicAdd(&Mns[mn_off[n] + int64_t(in) * R + r], c);
            else
              atomicAdd(&p.m[d.aoff[n] + in + int64_t(r) * d.I[n]], double(c));
          }
        }
      }
    }
    __syncthreads();
  }

  // flush partials
  if (want_m) {
    for (int e = tid; e < I1 * R; e += kMtThreads) {
      int i = e % I1, r = e / I1;   // consecutive threads -> consecutive rows (coalesced)
      atomicAdd(&p.m[i + int64_t(r) * I1], double(M1s[i * R + r]));
    }
    if (p.mn_in_smem) {
      for (int n = 1; n < N; ++n) {
        const int In = int(d.I[n]);
        for (int e = tid; e < In * R; e += kMtThreads) {
          int i = e % In, r = e / In;
          atomicAdd(&p.m[d.aoff[n] + i + int64_t(r) * In], double(Mns[mn_off[n] + int64_t(i) * R + r]));
        }
      }
    }
  }
  if (want_e) {
    double s = block_sum<kMtThreads>(e2_total, red);
    if (tid == 0) atomicAdd(p.resid2, s);
  }
}

// ---------------------------------------------------------------------------
// k_mttkrp_tiled: the production pass (I_1 <= 256 * RPT).
//
// Per tile of TF fibres (double-buffered in shared memory with cp.async):
//   phase B: thread = row i (RPT rows), all fibres of the tile:
//            M_1[i] += y[i,f] kr_f,  e = y[i,f] - A1[i] . kr_f,  e2 += e^2
//            (per fibre: R/4 broadcast 16-byte loads of kr_f feed 2R FMAs)
//   phase A: t_f = A1^T y_f as 4 x 4 register blocks of (f, r) with the
//            I_1 sum split into segments, then the segments summed
//   phase D: M_n[i_n(f)] += t_f * loo_f(n) for n >= 2: mode 2 directly
//            (fibres of a tile have distinct i_2 when TF <= I_2), modes >= 3
//            by one thread per (n, r) scanning the tile's fibres in order.
// ---------------------------------------------------------------------------
constexpr int kT2 = 256;          // threads
constexpr int kSeg = 8;           // segments of the I_1 sum in phase A

struct Tiled {
  Dims d;
  const void* Y;
  const double* a;
  double* m;
  double* resid2;
  const int* skip;
  int64_t fib_per_cta;
  int TF, ldy, Rp;                // fibres per tile, tile leading dim, R padded to 4
  int64_t mn_elems;               // sum_{n>=2} I_n R
  int grad;                       // 1: accumulate e = y - y_hat instead of y
};

template <typename TY>
__device__ __forceinline__ void cp_async_elem(TY* dst, const TY* src);
template <>
__device__ __forceinline__ void cp_async_elem<float>(float* dst, const float* src) {
  unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
template <>
__device__ __forceinline__ void cp_async_elem<double>(double* dst, const double* src) {
  unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ double to_f(double x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// Copy nf fibres starting at fibre f0 into the tile buffer (row f at f * ldy);
// bfloat16 tensors are widened to the float32 tile type TT on the way.
template <typename TY, typename TT>
__device__ void tile_copy(const TY* Y, int64_t f0, int nf, int I1, int ldy, TT* dst) {
  const int tot = nf * I1;
  const int64_t base = f0 * I1;
  int f = 0, i = threadIdx.x;
  while (i >= I1 && f < nf) { i -= I1; ++f; }
  for (int e = threadIdx.x; e < tot; e += kT2) {
    if constexpr (sizeof(TY) == 2) {
      dst[f * ldy + i] = __bfloat162float(Y[base + e]);
    } else {
      cp_async_elem<TY>(dst + f * ldy + i, Y + base + e);
    }
    i += kT2;
    while (i >= I1) { i -= I1; ++f; }
  }
}

template <typename TY, typename TT, typename TA, int RMAX, int RPT>
__global__ void __launch_bounds__(kT2) k_mttkrp_tiled(Tiled p) {
  pdl_enter();
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int R = d.R, N = d.N, Rp = p.Rp;
  const int I1 = int(d.I[0]);
  const int TF = p.TF, ldy = p.ldy;
  const int tid = threadIdx.x;
  const bool want_m = p.m != nullptr;

  TA* A1s = reinterpret_cast<TA*>(smem_raw);                         // I1 x Rp row-major
  TA* krs = A1s + size_t(I1) * Rp;                                    // TF x Rp
  TA* ts = krs + size_t(TF) * Rp;                                     // kSeg x TF x Rp partials
  TA* loos = ts + size_t(kSeg) * TF * Rp;                             // (N-1) x TF x Rp
  TA* Mns = loos + size_t(N - 1) * TF * Rp;                           // mn_elems
  TT* Yt0 = reinterpret_cast<TT*>(Mns + p.mn_elems);                  // 2 x TF x ldy
  TT* Yt1 = Yt0 + size_t(TF) * ldy;
  int* fidx = reinterpret_cast<int*>(Yt1 + size_t(TF) * ldy + 8);     // TF x CP_MAX_N
  double* red = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(fidx + TF * CP_MAX_N) + 15) & ~uintptr_t(15));

  const double* a = p.a;
  for (int e = tid; e < I1 * Rp; e += kT2) {
    const int i = e / Rp, r = e % Rp;
    A1s[e] = (r < R) ? TA(a[i + int64_t(r) * I1]) : TA(0);
  }
  for (int64_t e = tid; e < p.mn_elems; e += kT2) Mns[e] = TA(0);
  int64_t mn_off[CP_MAX_N];
  {
    int64_t o = 0;
    for (int n = 1; n < N; ++n) { mn_off[n] = o; o += d.I[n] * R; }
  }
  const int64_t f_begin = int64_t(blockIdx.x) * p.fib_per_cta;
  const int64_t f_end = (f_begin + p.fib_per_cta < d.nfib) ? f_begin + p.fib_per_cta : d.nfib;
  const TY* Y = reinterpret_cast<const TY*>(p.Y);

  TA acc[RPT][RMAX];
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int r = 0; r < RMAX; ++r) acc[q][r] = TA(0);
  double e2_total = 0.0;

  if (f_begin < f_end) {
    const int nf0 = int((f_end - f_begin) < TF ? (f_end - f_begin) : TF);
    tile_copy<TY, TT>(Y, f_begin, nf0, I1, ldy, Yt0);
  }
  cp_async_commit();
  int buf = 0;
  for (int64_t f0 = f_begin; f0 < f_end; f0 += TF) {
    const int nf = int((f_end - f0) < TF ? (f_end - f0) : TF);
    TT* Ycur = buf ? Yt1 : Yt0;
    TT* Ynext = buf ? Yt0 : Yt1;
    // prefetch the next tile
    const int64_t f1 = f0 + TF;
    if (f1 < f_end) {
      const int nf1 = int((f_end - f1) < TF ? (f_end - f1) : TF);
      tile_copy<TY, TT>(Y, f1, nf1, I1, ldy, Ynext);
    }
    cp_async_commit();
    // fibre multi-indices (i_2..i_N) of this tile
    for (int f = tid; f < nf; f += kT2) {
      int64_t rem = f0 + f;
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k) {
        if (k < N) {
          fidx[f * CP_MAX_N + k] = int(rem % d.I[k]);
          rem /= d.I[k];
        }
      }
    }
    __syncthreads();
    // Khatri-Rao rows and leave-one-out products
    for (int e = tid; e < nf * Rp; e += kT2) {
      const int f = e / Rp, r = e % Rp;
      TA v[CP_MAX_N];
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k)
        if (k < N) v[k] = (r < R) ? TA(a[d.aoff[k] + fidx[f * CP_MAX_N + k] + int64_t(r) * d.I[k]]) : TA(0);
      TA kr = TA(1);
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k)
        if (k < N) kr *= v[k];
      krs[f * Rp + r] = (r < R) ? kr : TA(0);
      if (want_m) {
#pragma unroll
        for (int n = 1; n < CP_MAX_N; ++n) {
          if (n < N) {
            TA lo = TA(1);
#pragma unroll
            for (int k = 1; k < CP_MAX_N; ++k)
              if (k < N && k != n) lo *= v[k];
            loos[(size_t(n - 1) * TF + f) * Rp + r] = lo;
          }
        }
      }
    }
    cp_async_wait<1>();
    __syncthreads();
    // phase B: rows
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int i = tid + q * kT2;
      if (i < I1) {
        TA arow[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) arow[r] = (r < Rp) ? A1s[i * Rp + r] : TA(0);
        TA e2 = TA(0);
        for (int f = 0; f < nf; ++f) {
          const TA y = TA(to_f(Ycur[f * ldy + i]));
          const TA* kf = krs + f * Rp;
          TA yh0 = TA(0), yh1 = TA(0);
#pragma unroll
          for (int r = 0; r < RMAX; r += 2) {
            if (r < Rp) {     // Rp is a multiple of 4: pairs are whole
              yh0 = fma(arow[r], kf[r], yh0);
              yh1 = fma(arow[r + 1], kf[r + 1], yh1);
            }
          }
          const TA e = y - (yh0 + yh1);
          e2 = fma(e, e, e2);
          const TA src = p.grad ? e : y;
          if (p.grad) Ycur[f * ldy + i] = TT(e);
#pragma unroll
          for (int r = 0; r < RMAX; r += 2) {
            if (r < Rp) {
              acc[q][r] = fma(src, kf[r], acc[q][r]);
              acc[q][r + 1] = fma(src, kf[r + 1], acc[q][r + 1]);
            }
          }
        }
        e2_total += double(e2);
      }
    }
    if (p.grad) __syncthreads();       // phase A reads rows of other threads
    // phase A: t_f partials over kSeg segments of rows, 4 x 4 blocks
    if (want_m) {
      const int nfb = (nf + 3) / 4, nrb = Rp / 4;
      const int seg_len = (I1 + kSeg - 1) / kSeg;
      for (int task = tid; task < nfb * nrb * kSeg; task += kT2) {
        const int rb = task % nrb, fb = (task / nrb) % nfb, sg = task / (nrb * nfb);
        const int ib = sg * seg_len, ie = (ib + seg_len < I1) ? ib + seg_len : I1;
        TA c[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) c[u][v] = TA(0);
        const int fr = fb * 4;
        for (int i = ib; i < ie; ++i) {
          TA yv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) yv[u] = (fr + u < nf) ? TA(to_f(Ycur[(fr + u) * ldy + i])) : TA(0);
          const TA* ar = A1s + i * Rp + rb * 4;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const TA av = ar[v];
#pragma unroll
            for (int u = 0; u < 4; ++u) c[u][v] = fma(yv[u], av, c[u][v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) ts[(size_t(sg) * TF + fr + u) * Rp + rb * 4 + v] = c[u][v];
      }
    }
    __syncthreads();
    if (want_m) {
      // sum the segments: ts[0] <- sum_sg ts[sg]
      for (int e = tid; e < nf * Rp; e += kT2) {
        TA s = ts[e];
#pragma unroll
        for (int sg = 1; sg < kSeg; ++sg) s += ts[size_t(sg) * TF * Rp + e];
        ts[e] = s;
      }
      __syncthreads();
      // phase D, mode 2: distinct i_2 inside the tile when TF <= I_2
      const bool direct2 = TF <= d.I[1];
      if (direct2) {
        for (int e = tid; e < nf * R; e += kT2) {
          const int f = e / R, r = e % R;
          const int i2 = fidx[f * CP_MAX_N + 1];
          Mns[mn_off[1] + int64_t(i2) * R + r] += ts[f * Rp + r] * loos[(size_t(0) * TF + f) * Rp + r];
        }
      }
      // modes >= 3 (and mode 2 otherwise): one thread per (n, r), fibres in order
      const int n_lo = direct2 ? 2 : 1;
      for (int task = tid; task < (N - n_lo) * R; task += kT2) {
        const int n = n_lo + task / R, r = task % R;
        int cur = fidx[0 * CP_MAX_N + n];
        TA s = TA(0);
        for (int f = 0; f < nf; ++f) {
          const int in = fidx[f * CP_MAX_N + n];
          if (in != cur) {
            Mns[mn_off[n] + int64_t(cur) * R + r] += s;
            s = TA(0);
            cur = in;
          }
          s = fma(ts[f * Rp + r], loos[(size_t(n - 1) * TF + f) * Rp + r], s);
        }
        Mns[mn_off[n] + int64_t(cur) * R + r] += s;
      }
    }
    __syncthreads();
    buf ^= 1;
  }
  cp_async_wait<0>();
  // flush
  if (want_m) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int i = tid + q * kT2;
      if (i < I1) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) atomicAdd(&p.m[i + int64_t(r) * I1], double(acc[q][r]));
      }
    }
    for (int n = 1; n < N; ++n) {
      const int In = int(d.I[n]);
      for (int e = tid; e < In * R; e += kT2) {
        const int i = e % In, r = e / In;
        atomicAdd(&p.m[d.aoff[n] + i + int64_t(r) * In], double(Mns[mn_off[n] + int64_t(i) * R + r]));
      }
    }
  }
  if (p.resid2) {
    const double sum = block_sum<kT2>(e2_total, red);
    if (tid == 0) atomicAdd(p.resid2, sum);
  }
}

// ---------------------------------------------------------------------------
// k_mttkrp3: the production pass.  Per tile of TF fibres (double-buffered in
// shared memory with cp.async), three register-tiled products that every
// thread shares, each inner step fed by 16-byte shared-memory loads:
//   B: M_1[i, r]  += sum_f y[i, f] kr_f[r]          4 rows x 4 r per thread,
//                                                    accumulators live in
//                                                    registers across tiles
//   C: yh[i, f]    = sum_r A1[i, r] kr_f[r],  e2 += (y - yh)^2
//                                                    4 rows x 4 fibres
//   A: t_f[r]      = sum_i y[i, f] A1[i, r]          8 fibres x 4 r over
//                                                    kSeg row segments
// then t is summed over segments and M_n[i_n(f)] += t_f * loo_f(n), n >= 2:
// mode 2 into a shared-memory partial (tile fibres have distinct i_2 when
// TF <= I_2), modes >= 3 by one thread per (n, r) that sums the tile's fibres
// per i_n run and adds the run to the float64 output.
// ---------------------------------------------------------------------------
constexpr int kT3 = 256;
constexpr int kSeg3 = 16;

struct P3 {
  Dims d;
  const void* Y;
  const double* a;
  double* m;
  double* resid2;
  const int* skip;
  int64_t fib_per_cta;
  int TF, ldy, Rp, ldi, nrb, npairB, FS;
  int mn2_smem;           // 1: mode-2 partial in shared memory
  int grad;               // 1: accumulate e = y - y_hat instead of y
  int fast;               // 1: factor rows of modes 2..N and the partials of M_2..M_N in shared memory
  int fib32;              // 1: fibre numbers fit 32 bits
  int afoff[CP_MAX_N];    // fast: offset (floats) of mode k's rows (I_k x Rp) in the factor area
  int mhoff[CP_MAX_N];    // fast: offset (floats) of mode n's partial (I_n x R) in the partial area
  int af_size, mh_size;   // fast: floats of the two areas
};

// bfloat16 tiles are fetched 16 bytes (8 values) at a time into registers at
// the top of a tile and written to the other tile buffer as float32 at its
// end, so the loads of tile t + 1 overlap the products of tile t.  A tile of
// at most kPref3 * kT3 * 8 values takes this path.
constexpr int kPref3 = 2;

template <typename TY>
__device__ __forceinline__ void tile_copy3(const TY* Y, int64_t f0, int nf, int I1, int ldy, float* dst);
template <>
__device__ __forceinline__ void tile_copy3<float>(const float* Y, int64_t f0, int nf, int I1, int ldy,
                                                  float* dst) {
  const int tot = nf * I1;
  const int64_t base = f0 * I1;
  int f = 0, i = threadIdx.x;
  while (i >= I1 && f < nf) { i -= I1; ++f; }
  for (int e = threadIdx.x; e < tot; e += kT3) {
    cp_async_elem<float>(dst + f * ldy + i, Y + base + e);
    i += kT3;
    while (i >= I1) { i -= I1; ++f; }
  }
}
template <>
__device__ __forceinline__ void tile_copy3<__nv_bfloat16>(const __nv_bfloat16* Y, int64_t f0, int nf, int I1,
                                                          int ldy, float* dst) {
  const int tot = nf * I1;
  const int64_t base = f0 * I1;
  int f = 0, i = threadIdx.x;
  while (i >= I1 && f < nf) { i -= I1; ++f; }
  for (int e = threadIdx.x; e < tot; e += kT3) {
    dst[f * ldy + i] = __bfloat162float(Y[base + e]);
    i += kT3;
    while (i >= I1) { i -= I1; ++f; }
  }
}

__device__ __forceinline__ void bf16_fetch3(const __nv_bfloat16* Y, int64_t f0, int nf, int I1,
                                            uint4 (&v)[kPref3]) {
  const int nvec = (nf * I1) / 8;
  const uint4* src = reinterpret_cast<const uint4*>(Y + f0 * I1);
#pragma unroll
  for (int q = 0; q < kPref3; ++q) {
    const int e8 = int(threadIdx.x) + q * kT3;
    if (e8 < nvec) v[q] = src[e8];
  }
}

__device__ __forceinline__ void bf16_store3(const __nv_bfloat16* Y, int64_t f0, int nf, int I1, int ldy,
                                            const uint4 (&v)[kPref3], float* dst) {
  const int tot = nf * I1, nvec = tot / 8;
#pragma unroll
  for (int q = 0; q < kPref3; ++q) {
    const int e8 = int(threadIdx.x) + q * kT3;
    if (e8 < nvec) {
      int e = 8 * e8, f = e / I1, i = e - f * I1;
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v[q]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 x = __bfloat1622float2(h[j]);
        dst[f * ldy + i] = x.x;
        if (++i == I1) { i = 0; ++f; }
        dst[f * ldy + i] = x.y;
        if (++i == I1) { i = 0; ++f; }
      }
    }
  }
  for (int e = 8 * nvec + int(threadIdx.x); e < tot; e += kT3) {   // the last values of a ragged tile
    const int f = e / I1;
    dst[f * ldy + e - f * I1] = __bfloat162float(Y[f0 * I1 + e]);
  }
}

template <typename TY, int PB>
__global__ void __launch_bounds__(kT3) k_mttkrp3(P3 p) {
  pdl_enter();
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Dims& d = p.d;
  const int R = d.R, N = d.N, Rp = p.Rp;
  const int I1 = int(d.I[0]);
  const int TF = p.TF, ldy = p.ldy, ldi = p.ldi;
  const int tid = threadIdx.x;
  const bool want_m = p.m != nullptr;

  float* A1s = reinterpret_cast<float*>(smem_raw);             // ldi x Rp   [i][r]
  float* A1t = A1s + size_t(ldi) * Rp;                          // Rp x ldi   [r][i]
  float* krs = A1t + size_t(Rp) * ldi;                          // TF x Rp    [f][r]
  float* krt = krs + size_t(TF) * Rp;                           // Rp x TF    [r][f]
  float* ts = krt + size_t(Rp) * TF;                            // kSeg3 x TF x Rp
  float* loos = ts + size_t(p.fast ? 1 : kSeg3) * TF * Rp;       // (N-1) x TF x Rp
  float* Mn2 = loos + size_t(N - 1) * TF * Rp;                  // I_2 x R (if mn2_smem)
  const int64_t mn2 = p.mn2_smem ? d.I[1] * R : 0;
  float* Af = Mn2 + ((mn2 + 3) & ~int64_t(3));                  // fast: rows of A^(2..N), [i][r]
  // fast: partials of M_2..M_N, [i][r] (one writer per entry and tile, in a
  // fixed order, so the sums do not depend on thread timing)
  float* Mnh = Af + ((p.af_size + 3) & ~3);
  float* Yt0 = Mnh + ((p.mh_size + 3) & ~3);                    // 2 x TF x ldy
  float* Yt1 = Yt0 + size_t(TF) * ldy;
  int* fidx = reinterpret_cast<int*>(Yt1 + size_t(TF) * ldy);   // TF x CP_MAX_N
  double* red = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(fidx + TF * CP_MAX_N) + 15) & ~uintptr_t(15));

  const double* a = p.a;
  for (int e = tid; e < ldi * Rp; e += kT3) {
    const int i = e / Rp, r = e % Rp;
    const float v = (i < I1 && r < R) ? float(a[i + int64_t(r) * I1]) : 0.f;
    A1s[e] = v;
    A1t[r * ldi + i] = v;
  }
  for (int64_t e = tid; e < mn2; e += kT3) Mn2[e] = 0.f;
  if (p.fast) {
    for (int e = tid; e < 2 * TF * ldy; e += kT3) Yt0[e] = 0.f;   // the padding of each row stays 0
    for (int k = 1; k < N; ++k) {
      const int Ik = int(d.I[k]);
      for (int e = tid; e < Ik * Rp; e += kT3) {
        const int i = e / Rp, r = e % Rp;
        Af[p.afoff[k] + e] = (r < R) ? float(a[d.aoff[k] + i + int64_t(r) * Ik]) : 0.f;
      }
    }
    for (int e = tid; e < p.mh_size; e += kT3) Mnh[e] = 0.f;
  }

  const int64_t f_begin = int64_t(blockIdx.x) * p.fib_per_cta;
  const int64_t f_end = (f_begin + p.fib_per_cta < d.nfib) ? f_begin + p.fib_per_cta : d.nfib;
  const TY* Y = reinterpret_cast<const TY*>(p.Y);

  // product B ownership: pair q = tid + k * kT3 (k < PB) -> (row block, r block),
  // with FS threads splitting the fibres of one pair when pairs are few
  const int nrbB = p.nrb, ncb = Rp / 4, FS = p.FS;
  float accB[PB][4][4];
#pragma unroll
  for (int k = 0; k < PB; ++k)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) accB[k][u][v] = 0.f;
  double e2_total = 0.0;

  // bfloat16 with the fast layout: register prefetch (see bf16_fetch3)
  constexpr bool kBf = sizeof(TY) == 2;
  const bool pref = kBf && p.fast;
  uint4 pv[kPref3];
  if (f_begin < f_end) {
    const int nf0 = int((f_end - f_begin) < TF ? (f_end - f_begin) : TF);
    if (pref) {
      if constexpr (kBf) {
        bf16_fetch3(reinterpret_cast<const __nv_bfloat16*>(Y), f_begin, nf0, I1, pv);
        bf16_store3(reinterpret_cast<const __nv_bfloat16*>(Y), f_begin, nf0, I1, ldy, pv, Yt0);
      }
    } else {
      tile_copy3<TY>(Y, f_begin, nf0, I1, ldy, Yt0);
    }
  }
  cp_async_commit();
  int buf = 0;
  for (int64_t f0 = f_begin; f0 < f_end; f0 += TF) {
    const int nf = int((f_end - f0) < TF ? (f_end - f0) : TF);
    float* Yc = buf ? Yt1 : Yt0;
    float* Yn = buf ? Yt0 : Yt1;
    const int64_t f1 = f0 + TF;
    const int nf1 = f1 < f_end ? int((f_end - f1) < TF ? (f_end - f1) : TF) : 0;
    if (pref) {
      if constexpr (kBf) {
        if (nf1 > 0) bf16_fetch3(reinterpret_cast<const __nv_bfloat16*>(Y), f1, nf1, I1, pv);
      }
    } else if (nf1 > 0) {
      tile_copy3<TY>(Y, f1, nf1, I1, ldy, Yn);
    }
    cp_async_commit();
    for (int f = tid; f < TF; f += kT3) {
      if (p.fib32) {
        uint32_t rem = uint32_t(f0 + (f < nf ? f : 0));
#pragma unroll
        for (int k = 1; k < CP_MAX_N; ++k)
          if (k < N) {
            const uint32_t Ik = uint32_t(d.I[k]);
            const uint32_t qt = rem / Ik;
            fidx[f * CP_MAX_N + k] = int(rem - qt * Ik);
            rem = qt;
          }
      } else {
        int64_t rem = f0 + (f < nf ? f : 0);
#pragma unroll
        for (int k = 1; k < CP_MAX_N; ++k)
          if (k < N) {
            fidx[f * CP_MAX_N + k] = int(rem % d.I[k]);
            rem /= d.I[k];
          }
      }
    }
    __syncthreads();
    for (int e = tid; e < TF * Rp; e += kT3) {
      const int f = e / Rp, r = e % Rp;
      const bool ok = (f < nf) && (r < R);
      float v[CP_MAX_N];
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k)
        if (k < N)
          v[k] = !ok ? 0.f
                     : (p.fast ? Af[p.afoff[k] + fidx[f * CP_MAX_N + k] * Rp + r]
                               : float(a[d.aoff[k] + fidx[f * CP_MAX_N + k] + int64_t(r) * d.I[k]]));
      float kr = 1.f;
#pragma unroll
      for (int k = 1; k < CP_MAX_N; ++k)
        if (k < N) kr *= v[k];
      kr = ok ? kr : 0.f;
      krs[f * Rp + r] = kr;
      krt[r * TF + f] = kr;
      if (want_m) {
#pragma unroll
        for (int n = 1; n < CP_MAX_N; ++n)
          if (n < N) {
            float lo = 1.f;
#pragma unroll
            for (int k = 1; k < CP_MAX_N; ++k)
              if (k < N && k != n) lo *= v[k];
            loos[(size_t(n - 1) * TF + f) * Rp + r] = ok ? lo : 0.f;
          }
      }
    }
    cp_async_wait<1>();
    __syncthreads();

    // ---- product C: residual (with p.grad the tile becomes E = Y - Y_hat,
    // which products B and A then use) ----
    {
      const int nfb = TF / 4;
      float e2 = 0.f;
      for (int q = tid; q < nrbB * nfb; q += kT3) {
        const int rb = q % nrbB, fb = q / nrbB;
        float c[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) c[u][v] = 0.f;
        for (int r = 0; r < Rp; ++r) {
          const float4 a4 = *reinterpret_cast<const float4*>(A1t + r * ldi + rb * 4);
          const float4 k4 = *reinterpret_cast<const float4*>(krt + r * TF + fb * 4);
          const float av[4] = {a4.x, a4.y, a4.z, a4.w};
          const float kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) c[u][v] = fmaf(av[u], kv[v], c[u][v]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int f = fb * 4 + v;
          if (f < nf) {
            const float4 y4 = *reinterpret_cast<const float4*>(Yc + f * ldy + rb * 4);
            const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
            float ev[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float e = (rb * 4 + u < I1) ? yv[u] - c[u][v] : 0.f;
              ev[u] = e;
              e2 = fmaf(e, e, e2);
            }
            if (p.grad)
              *reinterpret_cast<float4*>(Yc + f * ldy + rb * 4) = make_float4(ev[0], ev[1], ev[2], ev[3]);
          }
        }
      }
      e2_total += double(e2);
    }
    if (p.grad) __syncthreads();
    // ---- product B: M_1 += Y_tile KR_tile ----
    if (want_m) {
#pragma unroll
      for (int k = 0; k < PB; ++k) {
        const int q = (tid / FS) + k * (kT3 / FS);
        const int fs = tid % FS;
        if (q < p.npairB) {
          const int rb = q % nrbB, cb = q / nrbB;
          for (int f = fs; f < nf; f += FS) {
            const float4 y4 = *reinterpret_cast<const float4*>(Yc + f * ldy + rb * 4);
            const float4 k4 = *reinterpret_cast<const float4*>(krs + f * Rp + cb * 4);
            const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
            const float kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) accB[k][u][v] = fmaf(yv[u], kv[v], accB[k][u][v]);
          }
        }
      }
    }
    // ---- product A, fast layout: thread = (fibre f, 4 ranks), the whole row
    // range, y read 16 bytes at a time (rows ldy = 4 mod 32 floats apart, so
    // the 32 fibres of a warp hit every bank once per 8 lanes) ----
    if (want_m && p.fast) {
      const int nrq = Rp / 4;
      for (int task = tid; task < TF * nrq; task += kT3) {
        const int f = task % TF, rq = task / TF;
        float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
        const float* yr = Yc + f * ldy;
        for (int i = 0; i < ldi; i += 4) {
          const float4 y4 = *reinterpret_cast<const float4*>(yr + i);
          const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 a4 = *reinterpret_cast<const float4*>(A1s + (i + u) * Rp + rq * 4);
            c0 = fmaf(yv[u], a4.x, c0);
            c1 = fmaf(yv[u], a4.y, c1);
            c2 = fmaf(yv[u], a4.z, c2);
            c3 = fmaf(yv[u], a4.w, c3);
          }
        }
        *reinterpret_cast<float4*>(ts + f * Rp + rq * 4) = make_float4(c0, c1, c2, c3);
      }
    }
    // ---- product A: t partials ----
    if (want_m && !p.fast) {
      const int nfb8 = TF / 8, seg = (I1 + kSeg3 - 1) / kSeg3;
      for (int task = tid; task < nfb8 * ncb * kSeg3; task += kT3) {
        const int cb = task % ncb, fb = (task / ncb) % nfb8, sg = task / (ncb * nfb8);
        const int ib = sg * seg, ie = (ib + seg < I1) ? ib + seg : I1;
        float c[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) c[u][v] = 0.f;
        const float* yb = Yc + fb * 8 * ldy;
        for (int i = ib; i < ie; ++i) {
          const float4 a4 = *reinterpret_cast<const float4*>(A1s + i * Rp + cb * 4);
          const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float yv = yb[u * ldy + i];
#pragma unroll
            for (int v = 0; v < 4; ++v) c[u][v] = fmaf(yv, av[v], c[u][v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          *reinterpret_cast<float4*>(ts + (size_t(sg) * TF + fb * 8 + u) * Rp + cb * 4) =
              make_float4(c[u][0], c[u][1], c[u][2], c[u][3]);
      }
    }
    __syncthreads();
    if (want_m) {
      for (int e = tid; !p.fast && e < TF * Rp; e += kT3) {
        float sum = ts[e];
#pragma unroll
        for (int sg = 1; sg < kSeg3; ++sg) sum += ts[size_t(sg) * TF * Rp + e];
        ts[e] = sum;
      }
      __syncthreads();
      if (p.fast) {
        // modes 2..N without atomics, one writer per partial entry, so the
        // sums do not depend on thread timing.  The tile holds TF <= I_2
        // consecutive fibres, so (i) their i_2 are distinct: mode 2 is one
        // add per (fibre, rank); (ii) i_2 wraps at most once inside it, so
        // for n >= 3 the tile is two runs [0, sw) and [sw, nf) of constant
        // i_n, each summed by a warp.
        for (int e = tid; e < nf * R; e += kT3) {
          const int f = e / R, r = e % R;
          Mnh[p.mhoff[1] + fidx[f * CP_MAX_N + 1] * R + r] += ts[f * Rp + r] * loos[f * Rp + r];
        }
        if (N > 2) {
          // warp n - 2: lane = (rank, half of the tile's fibres), so the loads
          // of a fibre's ranks are contiguous; the halves meet by a shuffle
          const int i20 = fidx[1];
          const int sw = (int(d.I[1]) - i20 < nf) ? int(d.I[1]) - i20 : nf;   // first fibre of the second run
          const int warp = tid >> 5, lane = tid & 31;
          const int nh = Rp <= 16 ? 2 : 1, r = lane % (32 / nh), h = lane / (32 / nh);
          const int fh = (nf + nh - 1) / nh, fa = h * fh, fe = (fa + fh < nf) ? fa + fh : nf;
          for (int n = 2 + warp; n < N; n += kT3 / 32) {
            const float* lo = loos + size_t(n - 1) * TF * Rp;
            float s0 = 0.f, s1 = 0.f;
            if (r < Rp) {
              for (int f = fa; f < fe; ++f) {
                const float v = ts[f * Rp + r] * lo[f * Rp + r];
                if (f < sw) s0 += v;
                else s1 += v;
              }
            }
            if (nh == 2) {
              s0 += __shfl_xor_sync(0xffffffffu, s0, 16);
              s1 += __shfl_xor_sync(0xffffffffu, s1, 16);
            }
            if (h == 0 && r < R) {
              Mnh[p.mhoff[n] + fidx[n] * R + r] += s0;
              if (sw < nf) Mnh[p.mhoff[n] + fidx[sw * CP_MAX_N + n] * R + r] += s1;
            }
          }
        }
      }
      // mode 2
      if (!p.fast && p.mn2_smem) {
        if (TF <= d.I[1]) {
          for (int e = tid; e < nf * R; e += kT3) {
            const int f = e / R, r = e % R;
            Mn2[int64_t(fidx[f * CP_MAX_N + 1]) * R + r] += ts[f * Rp + r] * loos[f * Rp + r];
          }
        } else {
          for (int e = tid; e < nf * R; e += kT3) {
            const int f = e / R, r = e % R;
            atomicAdd(&Mn2[int64_t(fidx[f * CP_MAX_N + 1]) * R + r], ts[f * Rp + r] * loos[f * Rp + r]);
          }
        }
      }
      // modes >= 3 (and mode 2 without the shared partial): per (n, r), runs of equal i_n
      const int n_lo = p.mn2_smem ? 2 : 1;
      for (int task = tid; !p.fast && task < (N - n_lo) * R; task += kT3) {
        const int n = n_lo + task / R, r = task % R;
        int cur = fidx[n];
        float sacc = 0.f;
        for (int f = 0; f < nf; ++f) {
          const int in = fidx[f * CP_MAX_N + n];
          if (in != cur) {
            atomicAdd(&p.m[d.aoff[n] + cur + int64_t(r) * d.I[n]], double(sacc));
            sacc = 0.f;
            cur = in;
          }
          sacc = fmaf(ts[f * Rp + r], loos[(size_t(n - 1) * TF + f) * Rp + r], sacc);
        }
        atomicAdd(&p.m[d.aoff[n] + cur + int64_t(r) * d.I[n]], double(sacc));
      }
    }
    if (pref) {
      if constexpr (kBf) {
        if (nf1 > 0) bf16_store3(reinterpret_cast<const __nv_bfloat16*>(Y), f1, nf1, I1, ldy, pv, Yn);
      }
    }
    __syncthreads();
    buf ^= 1;
  }
  cp_async_wait<0>();
  __syncthreads();
  if (want_m) {
#pragma unroll
    for (int k = 0; k < PB; ++k) {
      const int q = (tid / FS) + k * (kT3 / FS);
      if (q < p.npairB) {
        const int rb = q % nrbB, cb = q / nrbB;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = rb * 4 + u, r = cb * 4 + v;
            if (i < I1 && r < R) atomicAdd(&p.m[i + int64_t(r) * I1], double(accB[k][u][v]));
          }
      }
    }
    if (p.fast) {
      for (int n = 1; n < N; ++n) {
        const int In = int(d.I[n]);
        for (int e = tid; e < In * R; e += kT3) {
          const int i = e % In, r = e / In;
          atomicAdd(&p.m[d.aoff[n] + i + int64_t(r) * In], double(Mnh[p.mhoff[n] + i * R + r]));
        }
      }
    } else if (p.mn2_smem) {
      const int I2 = int(d.I[1]);
      for (int e = tid; e < I2 * R; e += kT3) {
        const int i = e % I2, r = e / I2;
        atomicAdd(&p.m[d.aoff[1] + i + int64_t(r) * I2], double(Mn2[int64_t(i) * R + r]));
      }
    }
  }
  if (p.resid2) {
    const double sum = block_sum<kT3>(e2_total, red);
    if (tid == 0) atomicAdd(p.resid2, sum);
  }
}

static size_t smem3(const Dims& d, int TF, int ldy, int Rp, int ldi, int mn2_smem, int af_size = 0,
                    int mh_size = 0) {
  const bool fast = af_size > 0;
  size_t f = size_t(ldi) * Rp * 2 + size_t(TF) * Rp * 2 + size_t(fast ? 1 : kSeg3) * TF * Rp +
             size_t(d.N - 1) * TF * Rp;
  if (mn2_smem) f += (size_t(d.I[1]) * d.R + 3) & ~size_t(3);
  f += ((size_t(af_size) + 3) & ~size_t(3)) + ((size_t(mh_size) + 3) & ~size_t(3));
  f += 2 * size_t(TF) * ldy;
  return f * 4 + size_t(TF) * CP_MAX_N * 4 + 16 + kT3 * 8 + 16;
}

template <typename TY, int PB>
static int launch3_t(const P3& p, int grid, size_t smem, cudaStream_t s) {
  auto kern = k_mttkrp3<TY, PB>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return CP_ECUDA;
  CP_CUDA(launch_pdl(kern, grid, kT3, smem, s, p));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

// Returns CP_OK and launches, or CP_EINVAL when the shape does not fit this
// kernel (the caller then uses the generic pass).
int launch_mttkrp3(const Dims& d, const void* Y, const double* a, double* m, double* resid2, const int* skip,
                   cudaStream_t s, int grad) {
  if (d.y_dtype == CP_F64) return CP_EINVAL;
  const int I1 = int(d.I[0]);
  const int Rp = (d.R + 3) / 4 * 4;
  const int nrb = (I1 + 3) / 4;
  const int npairB = nrb * (Rp / 4);
  int PB = (npairB + kT3 - 1) / kT3;
  if (PB > 4) return CP_EINVAL;
  if (PB == 3) PB = 4;
  int FS = 1;
  if (PB == 1) {
    while (FS < 8 && npairB * FS * 2 <= kT3) FS *= 2;
  }
  const int ldi = nrb * 4;
  int TF = int(16384 / (size_t(I1) * 4));
  if (TF > 64) TF = 64;
  TF &= ~7;
  if (TF < 8) TF = 8;
  // leading dimension: a multiple of 4 floats (16-byte rows), 4 mod 32 words
  int ldy = (I1 + 3) / 4 * 4;
  while (ldy % 32 != 4) ldy += 4;
  const size_t max_smem = 200 * 1024;
  // the fast layout: factor rows of modes 2..N (float, I_k x Rp) and the
  // partials of M_2..M_N (I_n x R) in shared memory; bfloat16 tiles then go
  // through the register prefetch, which holds at most kPref3 * kT3 * 8 values
  int af_size = 0, mh_size = 0;
  int afoff[CP_MAX_N] = {0}, mhoff[CP_MAX_N] = {0};
  for (int k = 1; k < d.N; ++k) {
    afoff[k] = af_size;
    mhoff[k] = mh_size;
    af_size += int(d.I[k]) * Rp;
    mh_size += int(d.I[k]) * d.R;
  }
  // the fast layout also needs tiles of at most I_2 fibres (see the mode sums)
  int fast = (af_size + mh_size <= 24576 && d.I[1] >= 8) ? 1 : 0;
  const int TF_all = TF;
  if (fast && TF > d.I[1]) TF = int(d.I[1]) & ~7;
  if (fast && d.y_dtype == CP_BF16 && int64_t(TF) * I1 > int64_t(kPref3) * kT3 * 8) fast = 0;
  if (fast && d.y_dtype == CP_BF16 && (reinterpret_cast<uintptr_t>(Y) & 15) != 0) fast = 0;   // 16-byte loads
  if (!fast) TF = TF_all;
  int mn2_smem = fast ? 0 : 1;
  size_t smem = fast ? smem3(d, TF, ldy, Rp, ldi, 0, af_size, mh_size) : smem3(d, TF, ldy, Rp, ldi, 1);
  if (fast && smem > max_smem) {
    fast = 0;
    mn2_smem = 1;
    TF = TF_all;
    smem = smem3(d, TF, ldy, Rp, ldi, 1);
  }
  if (!fast && (smem > max_smem || d.I[1] * d.R > 16384)) {
    mn2_smem = 0;
    smem = smem3(d, TF, ldy, Rp, ldi, 0);
  }
  while (smem > max_smem && TF > 8) {
    TF = (TF / 2) & ~7;
    if (TF < 8) TF = 8;
    smem = fast ? smem3(d, TF, ldy, Rp, ldi, 0, af_size, mh_size) : smem3(d, TF, ldy, Rp, ldi, mn2_smem);
  }
  if (smem > max_smem) return CP_EINVAL;
  int per_sm = int((228 * 1024) / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 3) per_sm = 3;
  const int64_t ntiles = (d.nfib + TF - 1) / TF;
  int64_t grid = int64_t(kSMs) * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  const int64_t tiles_per = (ntiles + grid - 1) / grid;
  P3 p;
  p.d = d;
  p.Y = Y;
  p.a = a;
  p.m = m;
  p.resid2 = resid2;
  p.skip = skip;
  p.fib_per_cta = tiles_per * TF;
  p.TF = TF;
  p.ldy = ldy;
  p.Rp = Rp;
  p.ldi = ldi;
  p.nrb = nrb;
  p.npairB = npairB;
  p.FS = FS;
  p.mn2_smem = mn2_smem;
  p.grad = grad;
  p.fast = fast;
  p.fib32 = (d.nfib + TF < int64_t(0xFFFFFFFFll)) ? 1 : 0;
  for (int k = 0; k < CP_MAX_N; ++k) {
    p.afoff[k] = fast ? afoff[k] : 0;
    p.mhoff[k] = fast ? mhoff[k] : 0;
  }
  p.af_size = fast ? af_size : 0;
  p.mh_size = fast ? mh_size : 0;
  grid = (d.nfib + p.fib_per_cta - 1) / p.fib_per_cta;
  if (d.y_dtype == CP_F32) {
    switch (PB) {
      case 1: return launch3_t<float, 1>(p, int(grid), smem, s);
      case 2: return launch3_t<float, 2>(p, int(grid), smem, s);
      default: return launch3_t<float, 4>(p, int(grid), smem, s);
    }
  }
  switch (PB) {
    case 1: return launch3_t<__nv_bfloat16, 1>(p, int(grid), smem, s);
    case 2: return launch3_t<__nv_bfloat16, 2>(p, int(grid), smem, s);
    default: return launch3_t<__nv_bfloat16, 4>(p, int(grid), smem, s);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int rmax_for(int R) {
  if (R <= 4) return 4;
  if (R <= 8) return 8;
  if (R <= 16) return 16;
  if (R <= 24) return 24;
  return 32;
}

template <typename TY, typename TA, int RMAX>
static int launch_t(const MttkrpParams& p, int grid, size_t smem, cudaStream_t s) {
  auto kern = k_mttkrp<TY, TA, RMAX>;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
      return CP_ECUDA;
  }
  CP_CUDA(launch_pdl(kern, grid, kMtThreads, smem, s, p));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

template <typename TY, typename TA>
static int launch_r(const MttkrpParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (rmax_for(p.d.R)) {
    case 4: return launch_t<TY, TA, 4>(p, grid, smem, s);
    case 8: return launch_t<TY, TA, 8>(p, grid, smem, s);
    case 16: return launch_t<TY, TA, 16>(p, grid, smem, s);
    case 24: return launch_t<TY, TA, 24>(p, grid, smem, s);
    default: return launch_t<TY, TA, 32>(p, grid, smem, s);
  }
}

static size_t mttkrp_smem(const Dims& d, int TF, int I1p, int mn_in_smem, size_t ta) {
  size_t e = size_t(d.I[0]) * d.R * 2 + size_t(TF) * I1p + size_t(TF) * d.R * (2 + (d.N - 1));
  if (mn_in_smem) e += size_t(d.T - d.I[0]) * d.R;
  size_t bytes = e * ta + size_t(TF) * CP_MAX_N * sizeof(int) + 2 * sizeof(int) + 16 +
                 kMtThreads * sizeof(double) + 16;
  return bytes;
}

template <typename TY, typename TA, int RMAX, int RPT>
static int launch_tiled_t(const Tiled& p, int grid, size_t smem, cudaStream_t s) {
  using TT = typename std::conditional<sizeof(TY) == 2, float, TY>::type;
  auto kern = k_mttkrp_tiled<TY, TT, TA, RMAX, RPT>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return CP_ECUDA;
  CP_CUDA(launch_pdl(kern, grid, kT2, smem, s, p));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

template <typename TY, typename TA, int RPT>
static int launch_tiled_r(const Tiled& p, int grid, size_t smem, cudaStream_t s) {
  switch (rmax_for(p.d.R)) {
    case 4: return launch_tiled_t<TY, TA, 4, RPT>(p, grid, smem, s);
    case 8: return launch_tiled_t<TY, TA, 8, RPT>(p, grid, smem, s);
    case 16: return launch_tiled_t<TY, TA, 16, RPT>(p, grid, smem, s);
    case 24: return launch_tiled_t<TY, TA, 24, RPT>(p, grid, smem, s);
    default: return launch_tiled_t<TY, TA, 32, RPT>(p, grid, smem, s);
  }
}

template <typename TY, typename TA>
static int launch_tiled_q(const Tiled& p, int grid, size_t smem, cudaStream_t s) {
  const int I1 = int(p.d.I[0]);
  if (I1 <= kT2) return launch_tiled_r<TY, TA, 1>(p, grid, smem, s);
  if (I1 <= 2 * kT2) return launch_tiled_r<TY, TA, 2>(p, grid, smem, s);
  return launch_tiled_r<TY, TA, 3>(p, grid, smem, s);
}

static size_t tiled_smem(const Dims& d, int TF, int ldy, int Rp, size_t ta, size_t ty) {
  const size_t mn = size_t(d.T - d.I[0]) * d.R;
  size_t e = size_t(d.I[0]) * Rp + size_t(TF) * Rp * (1 + kSeg + (d.N - 1)) + mn;
  return e * ta + 2 * size_t(TF) * ldy * ty + 8 * 8 + size_t(TF) * CP_MAX_N * sizeof(int) + 16 +
         kT2 * sizeof(double) + 16;
}

// Enqueue one pass (m and resid2 must already be zeroed).
int launch_mttkrp_tc(const Dims& d, const void* Y, const double* a, double* m, double* resid2, const int* skip,
                     cudaStream_t s, int grad);

// grad = 1: the pass gives the gradient blocks E_(n) KR_n instead of M_n
// (not for the two-plane bfloat16 tensor, whose pass reads Y's planes as
// tensor-core operands directly: CP_EINVAL there).
int launch_mttkrp(const Dims& d, const void* Y, const double* a, double* m, double* resid2,
                  const int* skip, cudaStream_t s, int grad) {
  if (grad && d.y_dtype == CP_BF16X2) return CP_EINVAL;
  if (launch_mttkrp_tc(d, Y, a, m, resid2, skip, s, grad) == CP_OK) return CP_OK;
  if (launch_mttkrp3(d, Y, a, m, resid2, skip, s, grad) == CP_OK) return CP_OK;
  const size_t ta = (d.y_dtype == CP_F64) ? sizeof(double) : sizeof(float);
  // shared-memory tile element: bfloat16 tensors are widened to float32
  const size_t ty = (d.y_dtype == CP_F64) ? 8 : 4;
  const int I1 = int(d.I[0]);
  const size_t max_smem = 220 * 1024;
  if (I1 <= 3 * kT2) {
    const int Rp = (d.R + 3) / 4 * 4;
    // fibres per tile: about 16 KB of tensor per buffer, 4..64, and <= I_2 when possible
    int TF = int(16384 / (size_t(I1) * ty));
    if (TF > 64) TF = 64;
    if (TF < 4) TF = 4;
    TF &= ~3;                                    // phase A works on blocks of 4 fibres
    // leading dimension: odd in 4-byte words (conflict-free strided reads)
    int ldy = I1;
    if (ldy % 2 == 0) ldy += 1;                // odd: fibre rows fall in distinct banks
    size_t smem = tiled_smem(d, TF, ldy, Rp, ta, ty);
    while (smem > max_smem && TF > 4) {
      TF = (TF / 2) & ~3;
      if (TF < 4) TF = 4;
      smem = tiled_smem(d, TF, ldy, Rp, ta, ty);
    }
    if (smem <= max_smem) {
      int per_sm = int((228 * 1024) / (smem + 1024));
      if (per_sm < 1) per_sm = 1;
      if (per_sm > 4) per_sm = 4;
      const int64_t ntiles = (d.nfib + TF - 1) / TF;
      int64_t grid = int64_t(kSMs) * per_sm;
      if (grid > ntiles) grid = ntiles;
      if (grid < 1) grid = 1;
      const int64_t tiles_per = (ntiles + grid - 1) / grid;
      Tiled p;
      p.d = d;
      p.Y = Y;
      p.a = a;
      p.m = m;
      p.resid2 = resid2;
      p.skip = skip;
      p.fib_per_cta = tiles_per * TF;
      p.TF = TF;
      p.ldy = ldy;
      p.Rp = Rp;
      p.mn_elems = int64_t(d.T - d.I[0]) * d.R;
      p.grad = grad;
      grid = (d.nfib + p.fib_per_cta - 1) / p.fib_per_cta;
      switch (d.y_dtype) {
        case CP_F64: return launch_tiled_q<double, double>(p, int(grid), smem, s);
        case CP_F32: return launch_tiled_q<float, float>(p, int(grid), smem, s);
        default: return launch_tiled_q<__nv_bfloat16, float>(p, int(grid), smem, s);
      }
    }
  }
  // general fallback: one CTA tile of whole fibres (any I_1 that fits)
  int TF = kMtThreads / d.R;
  if (TF > 32) TF = 32;
  if (TF < 1) TF = 1;
  const int I1p = I1 + 1;
  int mn_in_smem = 1;
  size_t smem = mttkrp_smem(d, TF, I1p, 1, ta);
  if (smem > max_smem) {
    mn_in_smem = 0;
    smem = mttkrp_smem(d, TF, I1p, 0, ta);
  }
  while (smem > max_smem && TF > 1) {
    TF /= 2;
    smem = mttkrp_smem(d, TF, I1p, 0, ta);
  }
  if (smem > max_smem) return CP_EINVAL;
  int per_sm = int((228 * 1024) / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  int64_t ntiles = (d.nfib + TF - 1) / TF;
  int64_t grid = int64_t(kSMs) * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  int64_t tiles_per = (ntiles + grid - 1) / grid;
  MttkrpParams p;
  p.d = d;
  p.Y = Y;
  p.a = a;
  p.m = m;
  p.resid2 = resid2;
  p.skip = skip;
  p.fib_per_cta = tiles_per * TF;
  p.TF = TF;
  p.mn_in_smem = mn_in_smem;
  p.I1p = I1p;
  p.grad = grad;
  grid = (d.nfib + p.fib_per_cta - 1) / p.fib_per_cta;
  switch (d.y_dtype) {
    case CP_F64: return launch_r<double, double>(p, int(grid), smem, s);
    case CP_F32: return launch_r<float, float>(p, int(grid), smem, s);
    default: return launch_r<__nv_bfloat16, float>(p, int(grid), smem, s);
  }
}

}  // namespace cpdgn

using namespace cpdgn;

extern "C" int cp_mttkrp_all(const cp_shape* shape, const void* Y, const double* a, double* m,
                             double* resid2, void* ws, size_t ws_bytes, void* stream) {
  (void)ws;
  (void)ws_bytes;
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!Y || !a || !m) return CP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CP_CUDA(cudaMemsetAsync(m, 0, size_t(d.T) * d.R * sizeof(double), s));
  if (resid2) CP_CUDA(cudaMemsetAsync(resid2, 0, sizeof(double), s));
  return launch_mttkrp(d, Y, a, m, resid2, nullptr, s, 0);
}

namespace cpdgn {
__global__ void k_rel_err(const double* resid2, double y_norm2, double* rel) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) *rel = sqrt(*resid2 / y_norm2);
}
}  // namespace cpdgn

extern "C" int cp_fit(const cp_shape* shape, const void* Y, const double* a, double y_norm2,
                      double* resid2, double* rel_err, void* ws, size_t ws_bytes, void* stream) {
  (void)ws;
  (void)ws_bytes;
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!Y || !a || !resid2) return CP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CP_CUDA(cudaMemsetAsync(resid2, 0, sizeof(double), s));
  CP_TRY(launch_mttkrp(d, Y, a, nullptr, resid2, nullptr, s, 0));
  if (rel_err && y_norm2 > 0) {
    CP_CUDA(launch_pdl(k_rel_err, 1, 32, 0, s, resid2, y_norm2, rel_err));
    if (cudaGetLastError() != cudaSuccess) return CP_ECUDA;
  }
  return CP_OK;
}
