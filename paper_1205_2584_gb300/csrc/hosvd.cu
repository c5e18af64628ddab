// HOSVD initialisation of the factors (Algorithm 1 step 1; Sec. 4.6: the
// factors are initialised with the mode-n singular vectors of the data
// tensor, after which a few ALS sweeps are run).
//
//   A^(n) = the R leading left singular vectors of the unfolding Y_(n)
//         = the R leading eigenvectors of S_n = Y_(n) Y_(n)^T,
//
// in descending order, each column's sign fixed so that its entry of largest
// magnitude is positive (singular vectors are defined up to sign).
//
// Per mode, on the device:
//   k_ugram       S_n = Y_(n) Y_(n)^T, float64 accumulation: with P the
//                 product of the dimensions before n and Q those after it,
//                 S_n = sum_q Y_q^T Y_q over the P x I_n blocks Y_q of vec(Y);
//                 32 x 32 output tiles (upper triangle) x chunks of the sum,
//                 added with float64 atomics;
//   subspace iteration with m = R + min(R, 32) columns (at most I_n):
//   k_symm_mm     Z = S Q;
//   k_gram_tn     G = Z^T Z;   k_chol_inv   L = chol(G), L^{-1} (one CTA);
//   k_mm_rt       Q = Z L^{-T}  (Cholesky QR, applied twice per iteration);
//   k_gram_tn     T = Q^T S Q (Rayleigh-Ritz);  k_jacobi   T = V diag V^T
//                 (cyclic Jacobi with the parallel round-robin ordering, one
//                 CTA);  k_select   A^(n) = Q V(:, leading R), sign fixed.
// Every kernel is plain float64 SIMT code; no library routine is called.
#include "common.cuh"

namespace cpdgn {

constexpr int kHT = 256;          // threads of the tiled kernels
constexpr int kHM = 64;           // largest subspace (columns of Q)

__device__ __forceinline__ double hload(const void* Y, int dt, int64_t J, int64_t i) {
  switch (dt) {
    case CP_F64: return static_cast<const double*>(Y)[i];
    case CP_F32: return static_cast<const float*>(Y)[i];
    case CP_BF16X2:
      return double(__bfloat162float(static_cast<const __nv_bfloat16*>(Y)[i])) +
             double(__bfloat162float(static_cast<const __nv_bfloat16*>(Y)[J + i]));
    default: return __bfloat162float(static_cast<const __nv_bfloat16*>(Y)[i]);
  }
}

// S (In x In column-major, zeroed by the caller) += sum over the K range of
// this CTA.  blockIdx.x: tile pair (ti <= tj) of the upper triangle;
// blockIdx.y: chunk of K = P * Q.  Element (k, i) of the unfolding block
// structure: k = p + P q, address p + P i + P In q.
__global__ void __launch_bounds__(kHT) k_ugram(const void* Y, int dt, int64_t J, int64_t P, int In, int64_t K,
                                              int64_t kchunk, double* S) {
  __shared__ double Xi[64][33], Xj[64][33];
  const int nt = (In + 31) / 32;
  int b = blockIdx.x, ti = 0;
  while (b >= nt - ti) { b -= nt - ti; ++ti; }
  const int tj = ti + b;
  const int64_t k_begin = int64_t(blockIdx.y) * kchunk;
  const int64_t k_end = (k_begin + kchunk < K) ? k_begin + kchunk : K;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t kb = k_begin; kb < k_end; kb += 64) {
    for (int idx = tid; idx < 64 * 32; idx += kHT) {
      int kk, ii;
      if (P == 1) { ii = idx & 31; kk = idx >> 5; }
      else { kk = idx & 63; ii = idx >> 6; }
      const int64_t k = kb + kk;
      double vi = 0.0, vj = 0.0;
      if (k < k_end) {
        const int64_t p = k % P, q = k / P;
        const int i1 = ti * 32 + ii, i2 = tj * 32 + ii;
        if (i1 < In) vi = hload(Y, dt, J, p + P * i1 + P * In * q);
        if (i2 < In) vj = hload(Y, dt, J, p + P * i2 + P * In * q);
      }
      Xi[kk][ii] = vi;
      Xj[kk][ii] = vj;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 64; ++kk) {
      const double a0 = Xi[kk][tx], a1 = Xi[kk][tx + 16], b0 = Xj[kk][ty], b1 = Xj[kk][ty + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = ti * 32 + tx + 16 * u, j = tj * 32 + ty + 16 * v;
      if (i < In && j < In) {
        atomicAdd(&S[i + int64_t(In) * j], acc[u][v]);
        if (ti != tj) atomicAdd(&S[j + int64_t(In) * i], acc[u][v]);
      }
    }
}

// Deterministic start block: Q[i + I c] in [-1, 1) from a counter hash.
__global__ void k_randq(double* Q, int I, int m, unsigned seed) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < I * m; e += gridDim.x * blockDim.x) {
    uint32_t h = uint32_t(e) * 0x9E3779B1u ^ (seed * 0x85EBCA77u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    Q[e] = double(h) * (2.0 / 4294967296.0) - 1.0;
  }
}

// Z = S Q (S: I x I symmetric, Q: I x m); thread = output (i, c).
__global__ void k_symm_mm(const double* S, const double* Q, double* Z, int I, int m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I * m) return;
  const int i = e % I, c = e / I;
  const double* q = Q + int64_t(I) * c;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = 0;
  for (; k + 3 < I; k += 4) {
    s0 = fma(S[i + int64_t(I) * k], q[k], s0);
    s1 = fma(S[i + int64_t(I) * (k + 1)], q[k + 1], s1);
    s2 = fma(S[i + int64_t(I) * (k + 2)], q[k + 2], s2);
    s3 = fma(S[i + int64_t(I) * (k + 3)], q[k + 3], s3);
  }
  for (; k < I; ++k) s0 = fma(S[i + int64_t(I) * k], q[k], s0);
  Z[e] = (s0 + s1) + (s2 + s3);
}

// G = X^T Y (m x m) for I x m matrices X, Y; thread = output (r, c); G
// column-major.
__global__ void k_gram_tn(const double* X, const double* Y, double* G, int I, int m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int r = e % m, c = e / m;
  const double* x = X + int64_t(I) * r;
  const double* y = Y + int64_t(I) * c;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = 0;
  for (; k + 3 < I; k += 4) {
    s0 = fma(x[k], y[k], s0);
    s1 = fma(x[k + 1], y[k + 1], s1);
    s2 = fma(x[k + 2], y[k + 2], s2);
    s3 = fma(x[k + 3], y[k + 3], s3);
  }
  for (; k < I; ++k) s0 = fma(x[k], y[k], s0);
  G[e] = (s0 + s1) + (s2 + s3);
}

// One CTA: L = chol(G) (m x m), Linv = L^{-1} (lower, column-major).  A
// non-positive pivot (a rank-deficient block) is replaced by a tiny
// positive one so that the iteration continues; it is counted in *flag.
__global__ void __launch_bounds__(kHT) k_chol_inv(const double* G, double* Linv, int m, int* flag) {
  __shared__ double L[kHM][kHM + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += kHT) L[e % m][e / m] = G[e];
  double scale = 0.0;
  __syncthreads();
  for (int i = 0; i < m; ++i) scale = fmax(scale, L[i][i]);
  for (int j = 0; j < m; ++j) {
    __syncthreads();
    if (tid == 0) {
      double d = L[j][j];
      if (!(d > 1e-30 * scale) || !isfinite(d)) {
        atomicAdd(flag, 1);
        d = (scale > 0.0 ? scale : 1.0) * 1e-30;
      }
      L[j][j] = sqrt(d);
    }
    __syncthreads();
    const double ljj = L[j][j];
    for (int i = j + 1 + tid; i < m; i += kHT) L[i][j] /= ljj;
    __syncthreads();
    const int t = m - j - 1;
    for (int e = tid; e < t * t; e += kHT) {
      const int i = j + 1 + e % t, k = j + 1 + e / t;
      if (k <= i) L[i][k] = fma(-L[i][j], L[k][j], L[i][k]);
    }
  }
  __syncthreads();
  // Linv = L^{-1}: thread c < m solves L x = e_c by forward substitution,
  // writing column c of Linv (column-major) as it goes
  if (tid < m) {
    const int c = tid;
    double* x = Linv + int64_t(m) * c;
    for (int i = 0; i < m; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s = fma(-L[i][k], x[k], s);
      x[i] = (i < c) ? 0.0 : s / L[i][i];
    }
  }
}

// Q = Z Linv^T (Q[i, c] = sum_{l <= c} Z[i, l] Linv[c, l]); thread = (i, c).
__global__ void k_mm_rt(const double* Z, const double* Linv, double* Q, int I, int m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I * m) return;
  const int i = e % I, c = e / I;
  double s = 0.0;
  for (int l = 0; l <= c; ++l) s = fma(Z[i + int64_t(I) * l], Linv[c + m * l], s);
  Q[e] = s;
}

// One CTA: eigenvalues / vectors of the symmetric m x m matrix T by cyclic
// Jacobi sweeps in the round-robin (tournament) ordering: each round rotates
// m/2 disjoint index pairs at once.  Stops when the off-diagonal Frobenius
// norm falls below 1e-15 of the total, or after 40 sweeps.  V (m x m,
// column-major, eigenvectors in columns), w (eigenvalues).
constexpr int kJacobiSmem = 2 * kHM * (kHM + 1) * int(sizeof(double));
__global__ void __launch_bounds__(kHT) k_jacobi(const double* Tin, double* V, double* w, int m) {
  extern __shared__ double jsm[];
  double (*T)[kHM + 1] = reinterpret_cast<double (*)[kHM + 1]>(jsm);
  double (*Vs)[kHM + 1] = reinterpret_cast<double (*)[kHM + 1]>(jsm + kHM * (kHM + 1));
  __shared__ double cs[kHM / 2], sn[kHM / 2];
  __shared__ int pp[kHM / 2], qq[kHM / 2];
  __shared__ double red[kHT];
  __shared__ int done;
  const int tid = threadIdx.x;
  const int mm = m + (m & 1);                      // even number of players (a dummy when m is odd)
  for (int e = tid; e < m * m; e += kHT) {
    T[e % m][e / m] = Tin[e];
    Vs[e % m][e / m] = (e % m == e / m) ? 1.0 : 0.0;
  }
  if (tid == 0) done = 0;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence test
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < m * m; e += kHT) {
      const int i = e % m, j = e / m;
      const double v = T[i][j] * T[i][j];
      tot += v;
      if (i != j) off += v;
    }
    red[tid] = off;
    __syncthreads();
    for (int s = kHT / 2; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    const double offs = red[0];
    __syncthreads();
    red[tid] = tot;
    __syncthreads();
    for (int s = kHT / 2; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    if (tid == 0) done = !(offs > 1e-30 * red[0]);
    __syncthreads();
    if (done) break;
    for (int round = 0; round < mm - 1; ++round) {
      // pairs of this round: player 0 fixed, the others rotate
      if (tid < mm / 2) {
        const int a = (tid == 0) ? 0 : 1 + (tid - 1 + round) % (mm - 1);
        const int b = 1 + (mm - 2 - tid + round) % (mm - 1);
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < m && T[p][q] != 0.0) {
          const double tau = (T[q][q] - T[p][p]) / (2.0 * T[p][q]);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = rsqrt(1.0 + t * t);
          s = t * c;
        }
        if (q >= m) { p = 0; q = 0; c = 1.0; s = 0.0; }
        pp[tid] = p;
        qq[tid] = q;
        cs[tid] = c;
        sn[tid] = s;
      }
      __syncthreads();
      // rows p, q of T  (T <- J^T T)
      for (int e = tid; e < (mm / 2) * m; e += kHT) {
        const int k = e / m, j = e % m;
        const int p = pp[k], q = qq[k];
        if (p == q) continue;
        const double c = cs[k], s = sn[k];
        const double tp = T[p][j], tq = T[q][j];
        T[p][j] = c * tp - s * tq;
        T[q][j] = s * tp + c * tq;
      }
      __syncthreads();
      // columns p, q of T and of V  (T <- T J, V <- V J)
      for (int e = tid; e < (mm / 2) * m; e += kHT) {
        const int k = e / m, i = e % m;
        const int p = pp[k], q = qq[k];
        if (p == q) continue;
        const double c = cs[k], s = sn[k];
        const double tp = T[i][p], tq = T[i][q];
        T[i][p] = c * tp - s * tq;
        T[i][q] = s * tp + c * tq;
        const double vp = Vs[i][p], vq = Vs[i][q];
        Vs[i][p] = c * vp - s * vq;
        Vs[i][q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < m * m; e += kHT) V[e] = Vs[e % m][e / m];
  if (tid < m) w[tid] = T[tid][tid];
}

// A^(n)[:, r] = Q V[:, order[r]], order = eigenvalues descending; sign fixed
// so that the entry of largest magnitude is positive (the first one on ties).
// One CTA per output column r.
__global__ void __launch_bounds__(kHT) k_select(const double* Q, const double* V, const double* w, int I, int m,
                                                double* An, int R) {
  __shared__ double col[kHM];
  __shared__ double bv[kHT];
  __shared__ int bi[kHT];
  __shared__ int src;
  const int r = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) {
    // the r-th largest eigenvalue (selection by rank; ties broken by index)
    int s = 0;
    for (int c = 0; c < m; ++c) {
      int rank = 0;
      for (int d = 0; d < m; ++d)
        if (w[d] > w[c] || (w[d] == w[c] && d < c)) ++rank;
      if (rank == r) s = c;
    }
    src = s;
  }
  __syncthreads();
  if (tid < m) col[tid] = V[tid + m * src];
  __syncthreads();
  double best = -1.0;
  int besti = I;
  for (int i = tid; i < I; i += kHT) {
    double s = 0.0;
    for (int l = 0; l < m; ++l) s = fma(Q[i + int64_t(I) * l], col[l], s);
    An[i + int64_t(I) * r] = s;
    if (fabs(s) > best) { best = fabs(s); besti = i; }
  }
  bv[tid] = best;
  bi[tid] = besti;
  __syncthreads();
  for (int s = kHT / 2; s > 0; s >>= 1) {
    if (tid < s && (bv[tid + s] > bv[tid] || (bv[tid + s] == bv[tid] && bi[tid + s] < bi[tid]))) {
      bv[tid] = bv[tid + s];
      bi[tid] = bi[tid + s];
    }
    __syncthreads();
  }
  const bool flip = An[bi[0] + int64_t(I) * r] < 0.0;
  __syncthreads();
  if (flip)
    for (int i = tid; i < I; i += kHT) An[i + int64_t(I) * r] = -An[i + int64_t(I) * r];
}

static int hosvd_m(int In, int R) {
  int m = R + (R < 32 ? R : 32);
  if (m > kHM) m = kHM;
  if (m > In) m = In;
  return m;
}

static size_t hosvd_bytes(const Dims& d) {
  int64_t imax = 0;
  for (int n = 0; n < d.N; ++n) imax = d.I[n] > imax ? d.I[n] : imax;
  const size_t S = size_t(imax) * size_t(imax);
  const size_t QZ = 2 * size_t(imax) * kHM;
  const size_t small = 4 * size_t(kHM) * kHM + kHM;
  return (S + QZ + small) * sizeof(double) + 256;
}

}  // namespace cpdgn

using namespace cpdgn;

extern "C" int cp_hosvd_workspace_bytes(const cp_shape* shape, size_t* bytes) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!bytes) return CP_EINVAL;
  *bytes = hosvd_bytes(d);
  return CP_OK;
}

extern "C" int cp_hosvd(const cp_shape* shape, const void* Y, double* a, int iters, void* ws, size_t ws_bytes,
                        void* stream) {
  Dims d;
  CP_TRY(make_dims(shape, &d));
  if (!Y || !a || !ws || iters < 1 || iters > 1000) return CP_EINVAL;
  for (int n = 0; n < d.N; ++n)
    if (d.R > d.I[n] || d.I[n] > (int64_t(1) << 20)) return CP_EINVAL;
  if (ws_bytes < hosvd_bytes(d)) return CP_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t imax = 0;
  for (int n = 0; n < d.N; ++n) imax = d.I[n] > imax ? d.I[n] : imax;
  double* S = static_cast<double*>(ws);
  double* Q = S + imax * imax;
  double* Z = Q + imax * kHM;
  double* G = Z + imax * kHM;
  double* Li = G + kHM * kHM;
  double* V = Li + kHM * kHM;
  double* T = V + kHM * kHM;
  double* wv = T + kHM * kHM;
  int* flag = reinterpret_cast<int*>(wv + kHM);
  CP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  CP_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacobiSmem));
  int64_t P = 1;
  for (int n = 0; n < d.N; ++n) {
    const int In = int(d.I[n]);
    const int64_t Qo = d.J / (P * In);
    const int64_t K = P * Qo;
    const int m = hosvd_m(In, d.R);
    // S_n = Y_(n) Y_(n)^T
    CP_CUDA(cudaMemsetAsync(S, 0, size_t(In) * In * sizeof(double), s));
    const int nt = (In + 31) / 32;
    const int pairs = nt * (nt + 1) / 2;
    int64_t splits = (2 * int64_t(kSMs) + pairs - 1) / pairs;
    int64_t kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + 63) / 64 * 64;
    splits = (K + kchunk - 1) / kchunk;
    if (splits > 65535) return CP_EINVAL;
    k_ugram<<<dim3(unsigned(pairs), unsigned(splits)), kHT, 0, s>>>(Y, d.y_dtype, d.J, P, In, K, kchunk, S);
    // subspace iteration with Cholesky QR
    const int gq = (In * m + 255) / 256, gg = (m * m + 255) / 256;
    k_randq<<<gq, 256, 0, s>>>(Q, In, m, 0x5eedu + unsigned(n));
    for (int it = 0; it <= iters; ++it) {
      if (it > 0) k_symm_mm<<<gq, 256, 0, s>>>(S, Q, Z, In, m);
      else CP_CUDA(cudaMemcpyAsync(Z, Q, size_t(In) * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
      for (int pass = 0; pass < 2; ++pass) {
        const double* src = pass == 0 ? Z : Q;
        k_gram_tn<<<gg, 256, 0, s>>>(src, src, G, In, m);
        k_chol_inv<<<1, kHT, 0, s>>>(G, Li, m, flag);
        k_mm_rt<<<gq, 256, 0, s>>>(src, Li, pass == 0 ? Q : Z, In, m);
        if (pass == 1) CP_CUDA(cudaMemcpyAsync(Q, Z, size_t(In) * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
      }
    }
    // Rayleigh-Ritz
    k_symm_mm<<<gq, 256, 0, s>>>(S, Q, Z, In, m);
    k_gram_tn<<<gg, 256, 0, s>>>(Q, Z, T, In, m);
    k_jacobi<<<1, kHT, kJacobiSmem, s>>>(T, V, wv, m);
    k_select<<<d.R, kHT, 0, s>>>(Q, V, wv, In, m, a + d.aoff[n], d.R);
    P *= In;
  }
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
