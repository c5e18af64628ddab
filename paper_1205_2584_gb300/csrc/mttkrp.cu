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
// so each tensor element costs 3R multiply-adds whatever N is.  A CTA owns a
// contiguous range of fibres and keeps its partial M_1 (and M_n, n >= 2, when
// they fit) in shared memory; partials are added to the float64 outputs at
// the end.  TA is the arithmetic type: float64 for float64 tensors, float32
// for float32 and bfloat16 tensors (with float64 accumulation of ||E||^2 per
// tile and of the cross-CTA sums).
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
};

constexpr int kMtThreads = 256;

template <typename TY, typename TA, int RMAX>
__global__ void __launch_bounds__(kMtThreads) k_mttkrp(MttkrpParams p) {
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
    // P2: t_f = y_f^T A^(1)  (needed only for M_n, n >= 2)
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
    // P3: M_1 rows and the residual; one row per thread
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
        for (int r = 0; r < RMAX; ++r) {
          if (r < R) {
            const TA k = kf[r];
            acc[r] = fma(y, k, acc[r]);
            yh = fma(arow[r], k, yh);
          }
        }
        const TA e = y - yh;
        e2 = fma(e, e, e2);
      }
      e2_total += double(e2);
      if (want_m) {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) M1s[i * R + r] += acc[r];
      }
    }
    __syncthreads();
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
  kern<<<grid, kMtThreads, smem, s>>>(p);
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

// Enqueue one pass (m and resid2 must already be zeroed).
int launch_mttkrp(const Dims& d, const void* Y, const double* a, double* m, double* resid2,
                  const int* skip, cudaStream_t s) {
  const size_t ta = (d.y_dtype == CP_F64) ? sizeof(double) : sizeof(float);
  int TF = kMtThreads / d.R;
  if (TF > 32) TF = 32;
  if (TF < 1) TF = 1;
  const int I1 = int(d.I[0]);
  const int I1p = I1 + ((ta == 4) ? 1 : 1);
  const size_t max_smem = 220 * 1024;
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
  if (smem > max_smem) return CP_EINVAL;   // I_1 * R too large for one CTA's tile
  // CTAs resident per SM given the shared-memory footprint
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
  return launch_mttkrp(d, Y, a, m, resid2, nullptr, s);
}

namespace cpdgn {
__global__ void k_rel_err(const double* resid2, double y_norm2, double* rel) {
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
  CP_TRY(launch_mttkrp(d, Y, a, nullptr, resid2, nullptr, s));
  if (rel_err && y_norm2 > 0) {
    k_rel_err<<<1, 32, 0, s>>>(resid2, y_norm2, rel_err);
    if (cudaGetLastError() != cudaSuccess) return CP_ECUDA;
  }
  return CP_OK;
}
