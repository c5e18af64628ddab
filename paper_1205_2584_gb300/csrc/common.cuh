// Shared definitions of the cpdgn CUDA library: validated problem geometry,
// workspace layout and small device helpers.  Every kernel of the library is
// hand-written CUDA for sm_103a; nothing here calls a library compute routine.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/cpdgn.h"

namespace cpdgn {

constexpr int kSMs = 152;            // GB300: 2 dies x 76 SMs (grid sizing hint only)

// Geometry derived from a cp_shape, passed to kernels by value.
struct Dims {
  int N, R, RR;                      // RR = R * R
  int y_dtype;
  int64_t I[CP_MAX_N];
  int64_t row0[CP_MAX_N + 1];        // first row of mode n in the stacked T x R layout
  int64_t aoff[CP_MAX_N];            // offset of A^(n) in a: R * row0[n]
  int64_t T;                         // sum I_n
  int64_t J;                         // prod I_n
  int64_t nfib;                      // J / I_1 (mode-1 fibres)
  int64_t ncore;                     // N R^2
  int mg;                            // 1: a state's pass writes the gradient blocks
                                     // G_n = E_(n) KR_n (E = Y - Y_hat) instead of
                                     // M_n = Y_(n) KR_n (set by cp_state_create)
};

inline int make_dims(const cp_shape* s, Dims* d) {
  if (!s || !d) return CP_EINVAL;
  if (s->N < 2 || s->N > CP_MAX_N || s->R < 1 || s->R > CP_MAX_R) return CP_EINVAL;
  if (s->y_dtype != CP_F64 && s->y_dtype != CP_F32 && s->y_dtype != CP_BF16 && s->y_dtype != CP_BF16X2)
    return CP_EINVAL;
  // the two-plane form exists only for the tensor-core pass (3-way, I_1 % 8 == 0)
  if (s->y_dtype == CP_BF16X2 && (s->N != 3 || s->I[0] % 8 != 0)) return CP_EINVAL;
  d->N = s->N;
  d->R = s->R;
  d->RR = s->R * s->R;
  d->y_dtype = s->y_dtype;
  d->T = 0;
  d->J = 1;
  for (int n = 0; n < CP_MAX_N; ++n) d->I[n] = 0;
  for (int n = 0; n < s->N; ++n) {
    if (s->I[n] < 1 || s->I[n] > (int64_t(1) << 40)) return CP_EINVAL;
    d->I[n] = s->I[n];
    d->row0[n] = d->T;
    d->aoff[n] = d->T * s->R;
    d->T += s->I[n];
    if (d->J > (int64_t(1) << 62) / s->I[n]) return CP_EINVAL;
    d->J *= s->I[n];
  }
  for (int n = s->N; n < CP_MAX_N; ++n) { d->row0[n] = d->T; d->aoff[n] = d->T * s->R; }
  d->row0[CP_MAX_N] = d->T;
  d->nfib = d->J / d->I[0];
  d->ncore = int64_t(s->N) * d->RR;
  d->mg = 0;
  return CP_OK;
}

// ---------------------------------------------------------------------------
// Workspace layout.  Byte offsets of 256-aligned segments.  The "scratch"
// part serves the stand-alone calls; a cp_state places its own buffers
// first and the scratch part after them.
// ---------------------------------------------------------------------------
struct Layout {
  size_t off[40];
  size_t total;
};

enum Seg {
  // scratch
  S_C = 0,        // N R^2     C^(n)
  S_GNM,          // N^2 R^2   Gamma^(n,m)
  S_GALL,         // R^2
  S_P,            // N R^2     A^(n)T M_n
  S_LC,           // N R^2     chol(C^(n))
  S_U,            // N R^2     L_G^{-T}
  S_GT,           // N R^2     Gt_mu^(n)
  S_W,            // N R^2     w
  S_KW,           // N R^2     K w
  S_B,            // N R^2     S^T K w
  S_Y,            // N R^2     core^{-1} b
  S_Z,            // N R^2     temporaries of the matrix-free operator
  S_RES,          // N R^2     refinement residual
  S_D,            // N R^2     refinement correction
  S_F,            // N R^2     f
  S_WP,           // N(N-1)/2 R^3   W_(n,m) of the core build
  S_CORE32,       // 2 (N R^2)^2 float  (mixed mode: core and its Gauss-Jordan partner)
  S_GPART,        // partial sums of the Gram kernel
  S_PINV,         // 2 x 64 x 64 float: pivot inverses of the Gauss-Jordan sweeps
  S_PART,         // partial sums of the update kernel
  S_SCAL,         // small scalars and flags (doubles)
  S_INFO,         // ints
  S_DINV,         // ceil(N R^2 / 32) x 32 x 32 double: inverses of the Cholesky factor's diagonal tiles
  S_SYNC,         // grid-barrier and dataflow words of the float64 Cholesky and solves
  // state
  S_STATUS,       // cp_status
  S_M,            // R T  MTTKRP at the current factors
  S_MT,           // R T  MTTKRP at the trial factors
  S_AT,           // R T  trial factors
  S_DELTA,        // R T  last step
  S_SCALE,        // N R  normalisation scales
  S_MU,           // 1 double (copy of mu for the stand-alone calls)
  S_CORE64,       // (N R^2)^2 double (float64 core mode)
  S_NSEG
};

// Rows per CTA of the update kernel and the number of its CTAs.
constexpr int kUpdRows = 8;
inline int64_t update_ctas(const Dims& d) {
  int64_t c = 0;
  for (int n = 0; n < d.N; ++n) c += (d.I[n] + kUpdRows - 1) / kUpdRows;
  return c;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline void make_layout(const Dims& d, int core_mode, int with_state, Layout* L) {
  size_t sz[S_NSEG];
  for (int i = 0; i < S_NSEG; ++i) sz[i] = 0;
  const size_t dbl = sizeof(double);
  const size_t nr2 = size_t(d.ncore);
  sz[S_C] = d.N * d.RR * dbl;
  sz[S_GNM] = size_t(d.N) * d.N * d.RR * dbl;
  sz[S_GALL] = d.RR * dbl;
  sz[S_P] = sz[S_LC] = sz[S_U] = sz[S_GT] = d.N * d.RR * dbl;
  sz[S_W] = sz[S_KW] = sz[S_B] = sz[S_Y] = sz[S_Z] = sz[S_RES] = sz[S_D] = sz[S_F] = nr2 * dbl;
  sz[S_WP] = size_t(d.N) * (d.N - 1) / 2 * d.RR * d.R * dbl;
  sz[S_CORE32] = (core_mode == CP_CORE_MIXED) ? 2 * nr2 * nr2 * sizeof(float) : 0;
  {
    size_t ch = 0;
    for (int n = 0; n < d.N; ++n) ch += size_t((d.I[n] + 7) / 8);
    sz[S_GPART] = ch * size_t(d.R * (d.R + 1) / 2 + d.RR) * dbl;   // kGramRows = 8
  }
  sz[S_PINV] = 2 * 64 * 64 * sizeof(float);
  sz[S_PART] = size_t(update_ctas(d)) * (1 + d.R) * dbl;
  sz[S_SCAL] = 64 * dbl;
  sz[S_INFO] = 64 * sizeof(int);
  {
    const size_t nbk = size_t((d.ncore + 31) / 32);
    sz[S_DINV] = nbk * 32 * 32 * dbl;
    sz[S_SYNC] = 64 + nbk * sizeof(int);
  }
  if (with_state) {
    sz[S_STATUS] = sizeof(cp_status);
    sz[S_M] = sz[S_MT] = sz[S_AT] = sz[S_DELTA] = size_t(d.T) * d.R * dbl;
    sz[S_SCALE] = size_t(d.N) * d.R * dbl;
    sz[S_MU] = dbl;
    sz[S_CORE64] = (core_mode == CP_CORE_F64) ? nr2 * nr2 * dbl : 0;
  }
  size_t o = 0;
  for (int i = 0; i < S_NSEG; ++i) {
    L->off[i] = o;
    o += align256(sz[i]);
  }
  L->total = o;
}

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T to_acc(double x) { return T(x); }

__device__ __forceinline__ double load_y(const double* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float load_y(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float load_y(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(p[i]);
}

// Fixed-order block reduction of one double per thread (deterministic).
template <int NT>
__device__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Programmatic dependent launch.  The step's kernels are launched with the
// programmatic-serialisation attribute (launch_pdl), so a kernel's CTAs may be
// scheduled while its predecessor on the stream still runs.  Every such
// kernel begins with pdl_enter(): each CTA first waits (griddepcontrol.wait)
// until the predecessor has completed and its writes are visible, before it
// reads anything (the skip flag included) or exits, so each kernel completes
// after its predecessor and the ordering stays transitive; it then lets its
// own successor be scheduled.  A successor is scheduled only once every CTA
// of the kernel has started, so a grid whose CTAs wait on one another (all
// resident at once) is never crowded out by it.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace cpdgn

#define CP_TRY(expr)                   \
  do {                                 \
    int _rc = (expr);                  \
    if (_rc != CP_OK) return _rc;      \
  } while (0)

#define CP_CUDA(expr)                                  \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return CP_ECUDA;            \
  } while (0)

#define CP_LAUNCHED()                                  \
  do {                                                 \
    if (cudaPeekAtLastError() != cudaSuccess) return CP_ECUDA; \
  } while (0)
