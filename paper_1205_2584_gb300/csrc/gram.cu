// Gramians and the per-mode R x R quantities of one damped step.
//
//   C^(n) = A^(n)T A^(n),  Gamma^(n,m) = Hadamard_{k != n,m} C^(k),
//   Gamma = Hadamard_k C^(k)                          (Theorem 1, Eq. Gamma_a)
//   P^(n) = A^(n)T M_n                                (for w, Appendix D)
//
// Float64 throughout.  GB300 runs float64 at 2 FMA/clock/SM, so every
// product here is spread over one thread per output entry and over as many
// CTAs as there are entries, instead of one CTA per mode.
#include "common.cuh"

namespace cpdgn {

// One thread per entry of C^(n) (and of P^(n) when m != null).
__global__ void k_gram_cp(Dims d, const double* a, const double* m, double* C, double* P,
                          const int* skip) {
  if (skip && *skip) return;
  const int RR = d.RR, R = d.R;
  const int64_t nC = int64_t(d.N) * RR;
  const int64_t tot = m ? 2 * nC : nC;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= tot) return;
  const bool isP = idx >= nC;
  if (isP) idx -= nC;
  const int n = int(idx / RR);
  const int e = int(idx % RR);
  const int r = e % R, s = e / R;
  const int64_t I = d.I[n];
  const double* A = a + d.aoff[n];
  const double* B = isP ? (m + d.aoff[n]) : A;
  const double* x = A + int64_t(r) * I;
  const double* y = B + int64_t(s) * I;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int64_t i = 0;
  for (; i + 3 < I; i += 4) {
    s0 = fma(x[i], y[i], s0);
    s1 = fma(x[i + 1], y[i + 1], s1);
    s2 = fma(x[i + 2], y[i + 2], s2);
    s3 = fma(x[i + 3], y[i + 3], s3);
  }
  for (; i < I; ++i) s0 = fma(x[i], y[i], s0);
  (isP ? P : C)[int64_t(n) * RR + e] = (s0 + s1) + (s2 + s3);
}

// Gamma^(n,m) for all n, m and Gamma (one thread per entry).
__global__ void k_gram_hadamard(Dims d, const double* C, double* Gnm, double* Gall,
                                const int* skip) {
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

int launch_gram(const Dims& d, const double* a, const double* m, double* C, double* P,
                double* Gnm, double* Gall, const int* skip, cudaStream_t s) {
  const int64_t nC = int64_t(d.N) * d.RR * (m ? 2 : 1);
  k_gram_cp<<<unsigned((nC + 63) / 64), 64, 0, s>>>(d, a, m, C, P, skip);
  const int64_t nH = int64_t(d.N) * d.N * d.RR + d.RR;
  k_gram_hadamard<<<unsigned((nH + 127) / 128), 128, 0, s>>>(d, C, Gnm, Gall, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn

using namespace cpdgn;

extern "C" int cp_gram(const cp_shape* shape, const double* a, double* C, double* Gamma_nm,
                       double* Gamma_all, void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!a || !C) return CP_EINVAL;
  return launch_gram(d, a, nullptr, C, nullptr, Gamma_nm, Gamma_all, nullptr,
                     static_cast<cudaStream_t>(stream));
}
