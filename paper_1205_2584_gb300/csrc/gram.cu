// Gramians and the products A^(n)T M_n of one damped step, float64.
//
//   C^(n) = A^(n)T A^(n),  Gamma^(n,m) = Hadamard_{k != n,m} C^(k),
//   Gamma = Hadamard_k C^(k)                          (Theorem 1, Eq. Gamma_a)
//   P^(n) = A^(n)T M_n                                (for w, Appendix D)
//
// GB300 executes float64 at 2 FMA/clock/SM, so the T x R^2 products are split
// over CTAs of kGramRows rows each (k_gram_partial) and summed in a fixed
// order by k_gram_reduce: deterministic, and no SM does more than
// kGramRows * (R(R+1)/2 + R^2) multiply-adds.
#include "common.cuh"

namespace cpdgn {

constexpr int kGramRows = 8;
constexpr int kGramThreads = 256;

inline int64_t gram_chunks(const Dims& d) {
  int64_t c = 0;
  for (int n = 0; n < d.N; ++n) c += (d.I[n] + kGramRows - 1) / kGramRows;
  return c;
}
// entries per chunk: upper triangle of C, then P (R^2) when wanted
__host__ __device__ inline int gram_entries(int R, bool withP) { return R * (R + 1) / 2 + (withP ? R * R : 0); }

__global__ void __launch_bounds__(kGramThreads) k_gram_partial(Dims d, const double* a, const double* m,
                                                               double* part, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  __shared__ double As[kGramRows][CP_MAX_R + 1];
  __shared__ double Ms[kGramRows][CP_MAX_R + 1];
  const int R = d.R;
  int b = blockIdx.x, n = 0;
  for (; n < d.N; ++n) {
    const int nb = int((d.I[n] + kGramRows - 1) / kGramRows);
    if (b < nb) break;
    b -= nb;
  }
  const int64_t In = d.I[n];
  const int64_t i0 = int64_t(b) * kGramRows;
  const int rows = int((In - i0) < kGramRows ? (In - i0) : kGramRows);
  const bool withP = m != nullptr;
  for (int e = threadIdx.x; e < kGramRows * R; e += kGramThreads) {
    const int i = e % kGramRows, r = e / kGramRows;
    const bool ok = i < rows;
    As[i][r] = ok ? a[d.aoff[n] + i0 + i + In * r] : 0.0;
    if (withP) Ms[i][r] = ok ? m[d.aoff[n] + i0 + i + In * r] : 0.0;
  }
  __syncthreads();
  const int nC = R * (R + 1) / 2;
  const int E = gram_entries(R, withP);
  double* out = part + int64_t(blockIdx.x) * E;
  for (int e = threadIdx.x; e < E; e += kGramThreads) {
    int r, s;
    const double (*Bs)[CP_MAX_R + 1];
    if (e < nC) {   // upper triangle, column by column: s = col, r <= s
      s = int((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while ((s + 1) * (s + 2) / 2 <= e) ++s;
      while (s * (s + 1) / 2 > e) --s;
      r = e - s * (s + 1) / 2;
      Bs = As;
    } else {
      const int q = e - nC;
      r = q % R;
      s = q / R;
      Bs = Ms;
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kGramRows; ++i) acc = fma(As[i][r], Bs[i][s], acc);
    out[e] = acc;
  }
}

// C^(n) (mirrored) and P^(n) from the partials, summed in chunk order.
__global__ void k_gram_reduce(Dims d, const double* part, bool withP, double* C, double* P,
                              const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR;
  const int nC = R * (R + 1) / 2;
  const int E = gram_entries(R, withP);
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(d.N) * E) return;
  const int n = int(idx / E), e = int(idx % E);
  int64_t c0 = 0;
  for (int k = 0; k < n; ++k) c0 += (d.I[k] + kGramRows - 1) / kGramRows;
  const int64_t c1 = c0 + (d.I[n] + kGramRows - 1) / kGramRows;
  double s = 0.0;
#pragma unroll 8
  for (int64_t c = c0; c < c1; ++c) s += part[c * E + e];
  if (e < nC) {
    int col = int((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((col + 1) * (col + 2) / 2 <= e) ++col;
    while (col * (col + 1) / 2 > e) --col;
    const int row = e - col * (col + 1) / 2;
    C[int64_t(n) * RR + row + R * col] = s;
    C[int64_t(n) * RR + col + R * row] = s;
  } else {
    P[int64_t(n) * RR + (e - nC)] = s;
  }
}

// Gamma^(n,m) for all n, m and Gamma (one thread per entry).
__global__ void k_gram_hadamard(Dims d, const double* C, double* Gnm, double* Gall, const int* skip) {
  pdl_enter();
  if (skip && *skip) return;
  const int RR = d.RR, N = d.N;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nG = int64_t(N) * N * RR;
  if (idx < nG) {
    const int e = int(idx % RR);
    const int nm = int(idx / RR);
    const int n = nm / N, mm = nm % N;
    double v = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != n && k != mm) v *= C[int64_t(k) * RR + e];
    if (Gnm) Gnm[idx] = v;
  } else if (idx < nG + RR) {
    const int e = int(idx - nG);
    double v = 1.0;
    for (int k = 0; k < N; ++k) v *= C[int64_t(k) * RR + e];
    if (Gall) Gall[e] = v;
  }
}

size_t gram_part_bytes(const Dims& d) {
  return size_t(gram_chunks(d)) * gram_entries(d.R, true) * sizeof(double);
}

// C, P (if m) and, if Gnm / Gall are given, the Hadamard products.
int launch_gram(const Dims& d, const double* a, const double* m, double* part, double* C, double* P,
                double* Gnm, double* Gall, const int* skip, cudaStream_t s) {
  const int64_t nch = gram_chunks(d);
  CP_CUDA(launch_pdl(k_gram_partial, unsigned(nch), kGramThreads, 0, s, d, a, m, part, skip));
  const int64_t ne = int64_t(d.N) * gram_entries(d.R, m != nullptr);
  CP_CUDA(launch_pdl(k_gram_reduce, unsigned((ne + 127) / 128), 128, 0, s, d, part, m != nullptr, C, P, skip));
  if (Gnm || Gall) {
    const int64_t nH = int64_t(d.N) * d.N * d.RR + d.RR;
    CP_CUDA(launch_pdl(k_gram_hadamard, unsigned((nH + 127) / 128), 128, 0, s, d, C, Gnm, Gall, skip));
  }
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn

using namespace cpdgn;

extern "C" int cp_gram(const cp_shape* shape, const double* a, double* C, double* Gamma_nm,
                       double* Gamma_all, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !C || !ws) return CP_EINVAL;
  if (ws_bytes < gram_part_bytes(d)) return CP_ENOMEM;
  return launch_gram(d, a, nullptr, static_cast<double*>(ws), C, nullptr, Gamma_nm, Gamma_all, nullptr,
                     static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// cp_gram_noalloc: cp_gram with its partial sums in a fixed device array.
//
// Some callers cannot allocate device memory: code running inside a host
// framework that owns the whole device memory pool and forbids any further
// allocation, or a plugin that is handed only its inputs and outputs.  This
// entry point needs neither a workspace argument nor any allocation: the
// partial sums of the row-block reduction live in the file-scope array
// below, which every GPU that loads the library keeps until the process
// exits.  All calls share it, so calls that overlap on the GPU (different
// streams, no ordering between them) race and give wrong results; calls on
// one stream, or otherwise ordered, are fine.  Nothing in it has to start at
// zero: every call writes each partial it later reads.
// ---------------------------------------------------------------------------
namespace cpdgn {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 18;   // 2 MiB of float64 partials
static __device__ __align__(256) double g_gram_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
static double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_gram_scratch on the current device, looked up once per
// device (cudaGetSymbolAddress with that device current) and cached.  The
// cache is keyed by device ordinal: after cudaDeviceReset (which unloads the
// module) the cached address is stale, so a process that resets a device
// must not call cp_gram_noalloc on it again.
static int noalloc_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CP_ECUDA;
  double* p = __atomic_load_n(&g_scratch_ptr[dev], __ATOMIC_ACQUIRE);
  if (!p) {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_gram_scratch) != cudaSuccess || !q) return CP_ECUDA;
    p = static_cast<double*>(q);
    __atomic_store_n(&g_scratch_ptr[dev], p, __ATOMIC_RELEASE);
  }
  *out = p;
  return CP_OK;
}

}  // namespace cpdgn

extern "C" int cp_gram_noalloc(const cp_shape* shape, const double* a, double* C, double* Gamma_nm,
                               double* Gamma_all, void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !C) return CP_EINVAL;
  // this call never forms P = A^T M, so its partials need R(R+1)/2 doubles per chunk
  if (size_t(gram_chunks(d)) * gram_entries(d.R, false) > kNoallocScratchDoubles) return CP_ENOMEM;
  double* scratch = nullptr;
  CP_TRY(noalloc_scratch(&scratch));
  return launch_gram(d, a, nullptr, scratch, C, nullptr, Gamma_nm, Gamma_all, nullptr,
                     static_cast<cudaStream_t>(stream));
}
