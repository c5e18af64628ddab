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

// 1 / d for d > 0 (finite) by Newton's iteration for the reciprocal,
// x <- x (2 - d x), written as x + x (1 - d x), from the hardware's
// approximate double reciprocal: two iterations take its error below the
// rounding of a double, in four dependent multiply-adds.
__device__ __forceinline__ double small_recip(double d) {
  double x;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
  x = fma(x, fma(-d, x, 1.0), x);
  x = fma(x, fma(-d, x, 1.0), x);
  return x;
}

// The same factorisation by a whole CTA (R <= 32, at least R threads).  The
// pivot chain is latency-bound: on this part a dependent float64 square root
// costs about 560 cycles, a reciprocal square root about 320.  So the
// elimination keeps each column unscaled, D[i][l] -= D[i][k] D[l][k] / d_k for
// k < l <= i, which needs only the reciprocal of each pivot: the thread that
// updates the next pivot forms it at once (small_recip), and one barrier per
// column separates the steps.  Lane = row i, the warps share the columns l.
// At the end L[i][k] = D[i][k] / sqrt(d_k) for all entries at once, with
// rinv[k] = 1 / sqrt(d_k).  A non-positive or non-finite pivot clears *ok_s
// and is replaced by 1, so no NaN spreads; the return value is uniform over
// the CTA.
__device__ __forceinline__ bool cta_chol(double* G, double* rinv, int R, int* ok_s) {
  __shared__ double q[CP_MAX_R];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  __syncthreads();
  if (tid == 0) {
    *ok_s = 1;
    double d = G[0];
    if (!(d > 0.0) || !isfinite(d)) {
      *ok_s = 0;
      d = 1.0;
      G[0] = 1.0;
    }
    q[0] = small_recip(d);
  }
  __syncthreads();
  for (int k = 0; k + 1 < R; ++k) {
    const int i = k + 1 + lane;
    if (i < R) {
      const double gik = G[i + R * k] * q[k];
      for (int l = k + 1 + w; l <= i; l += nw) {
        const double v = fma(-gik, G[l + R * k], G[i + R * l]);
        if (l == k + 1 && i == k + 1) {              // the next pivot: its reciprocal now
          double d = v;
          if (!(d > 0.0) || !isfinite(d)) {
            *ok_s = 0;
            d = 1.0;
          }
          G[i + R * l] = d;
          q[k + 1] = small_recip(d);
        } else {
          G[i + R * l] = v;
        }
      }
    }
    __syncthreads();
  }
  if (tid < R) rinv[tid] = rsqrt(G[tid + R * tid]);
  __syncthreads();
  for (int e = tid; e < R * R; e += nt) {
    const int i = e % R, k = e / R;
    if (i >= k) G[e] *= rinv[k];                     // L[k][k] = d_k / sqrt(d_k)
  }
  __syncthreads();
  return *ok_s != 0;
}

// z <- L^{-1} z and z <- L^{-T} z by one warp with z in registers (lane = row,
// R <= 32): each step broadcasts one entry by a shuffle, so the chain per row
// is a shuffle, a multiply and a multiply-add.  rl = rinv[lane] (1 / L[lane,lane]).
__device__ __forceinline__ double warp_fwd_reg(const double* L, double rl, double z, int R) {
  const int lane = threadIdx.x & 31;
  for (int p = 0; p < R; ++p) {
    const double zp = __shfl_sync(0xffffffffu, z, p) * __shfl_sync(0xffffffffu, rl, p);
    if (lane == p) z = zp;
    else if (lane > p && lane < R) z = fma(-L[lane + R * p], zp, z);
  }
  return z;
}
__device__ __forceinline__ double warp_bwd_reg(const double* L, double rl, double z, int R) {
  const int lane = threadIdx.x & 31;
  for (int p = R - 1; p >= 0; --p) {
    const double zp = __shfl_sync(0xffffffffu, z, p) * __shfl_sync(0xffffffffu, rl, p);
    if (lane == p) z = zp;
    else if (lane < p) z = fma(-L[p + R * lane], zp, z);
  }
  return z;
}

}  // namespace cpdgn
