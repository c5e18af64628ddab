// Warp-level float64 helpers on small R x R column-major matrices in shared
// memory (R <= 32; lane = row), shared by the per-mode kernels and the
// batched kernel.
#pragma once
#include "common.cuh"

namespace cpdgn {

// In-place lower Cholesky of the R x R matrix G (column-major, ld R) by one
// warp (lane = row); rinv[k] receives 1 / L[k,k].  Float64 divides and square
// roots are slow on this part (2 float64 lanes per clock per SM), so each step
// takes one of each and the column is scaled by a multiply.  Returns false on
// a non-positive or non-finite pivot.
__device__ __forceinline__ bool warp_chol(double* G, double* rinv, int R) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < R; ++k) {
    __syncwarp();
    const double piv = G[k + R * k];
    if (!(piv > 0.0) || !isfinite(piv)) ok = false;
    const double dk = sqrt(piv);
    const double ik = 1.0 / dk;
    double lik = 0.0;
    if (lane > k && lane < R) lik = G[lane + R * k] * ik;
    __syncwarp();
    if (lane == k) {
      G[k + R * k] = dk;
      rinv[k] = ik;
    }
    if (lane > k && lane < R) G[lane + R * k] = lik;
    __syncwarp();
    if (lane > k && lane < R)
      for (int l = k + 1; l <= lane; ++l) G[lane + R * l] = fma(-lik, G[l + R * k], G[lane + R * l]);
  }
  __syncwarp();
  return ok;
}

// The same factorisation by a whole CTA.  The pivot chain is latency-bound:
// on this part a dependent float64 square root costs about 560 cycles and a
// divide about 360, a reciprocal square root about 320.  So one thread takes
// rsqrt of each pivot (L[k,k] = piv * rsqrt(piv), 1 / L[k,k] = rsqrt(piv),
// each within a few ulp of the square root and its reciprocal) while the
// others wait at a barrier, and the column scale and the trailing update are
// spread over all threads.  ok_s is a shared-memory flag; the return value is
// uniform over the CTA.
__device__ __forceinline__ bool cta_chol(double* G, double* rinv, int R, int* ok_s) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *ok_s = 1;
  for (int k = 0; k < R; ++k) {
    __syncthreads();
    if (tid == 0) {
      const double piv = G[k + R * k];
      if (!(piv > 0.0) || !isfinite(piv)) *ok_s = 0;
      const double ik = rsqrt(piv);
      G[k + R * k] = piv * ik;
      rinv[k] = ik;
    }
    __syncthreads();
    const double ik = rinv[k];
    const int m = R - k - 1;
    for (int i = tid; i < m; i += nt) G[k + 1 + i + R * k] *= ik;
    __syncthreads();
    for (int q = tid; q < m * m; q += nt) {
      const int i = k + 1 + q % m, l = k + 1 + q / m;
      if (l <= i) G[i + R * l] = fma(-G[i + R * k], G[l + R * k], G[i + R * l]);
    }
  }
  __syncthreads();
  return *ok_s != 0;
}

// z <- L^{-1} z, one warp; rinv = 1 / diag(L).
__device__ __forceinline__ void warp_fwd(const double* L, const double* rinv, double* z, int R) {
  const int lane = threadIdx.x & 31;
  for (int p = 0; p < R; ++p) {
    __syncwarp();
    const double zp = z[p] * rinv[p];
    __syncwarp();
    if (lane == p) z[p] = zp;
    if (lane > p && lane < R) z[lane] = fma(-L[lane + R * p], zp, z[lane]);
  }
  __syncwarp();
}

// z <- L^{-T} z, one warp.
__device__ __forceinline__ void warp_bwd(const double* L, const double* rinv, double* z, int R) {
  const int lane = threadIdx.x & 31;
  for (int p = R - 1; p >= 0; --p) {
    __syncwarp();
    const double zp = z[p] * rinv[p];
    __syncwarp();
    if (lane == p) z[p] = zp;
    if (lane < p) z[lane] = fma(-L[p + R * lane], zp, z[lane]);
  }
  __syncwarp();
}

}  // namespace cpdgn
