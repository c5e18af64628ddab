// Damped per-mode inverses, w, and the symmetric positive definite core system.
//
// Theorem 3 writes (H + mu I)^{-1} = Gt - L_mu B_mu L_mu^T with
// B_mu = K (I + Psi_mu K)^{-1} (Eq. inverse_f1a).  With Psi_mu = S S^T,
// S = blkdiag(S_n), S_n = U_n kron L_n, where Gamma^(n) + mu I = L_G L_G^T,
// U_n = L_G^{-T} (U_n U_n^T = Gt^(n)) and C^(n) = L_n L_n^T, the push-through
// identity gives
//     B_mu w = K w - K S (I + S^T K S)^{-1} S^T K w,
// and core = I + S^T K S is symmetric positive definite whenever H + mu I is
// and every A^(n) has full column rank (x^T core x = v^T (H + mu I) v for
// v = Gt Z Psi^{-1} S x).  This replaces the paper's non-symmetric Phi_1 and
// the indefinite Phi_2 of Sec. 4.4 by a matrix Cholesky can factor.
//
// Block (n, m), n != m, of S^T K S, entry (i + R j, k + R l):
//     sum_a L_n[a,i] U_m[a,l] W_nm[a, (k,j)],
//     W_nm[a, (k,j)] = sum_b Gamma^(n,m)[a,b] L_m[b,k] U_n[b,j],
// which costs O(R^5) per block instead of the O(R^6) of the dense product.
//
// The matrix-free operators below apply S, S^T and K in O(N R^3) and
// O(N^2 R^2) float64 operations (Kronecker identity (U kron L) vec X =
// vec(L X U^T); K^(n,m) vec X = vec((Gamma^(n,m) * X)^T)).
#include "common.cuh"

namespace cpdgn {

// --- warp-level helpers on an R x R column-major matrix in shared memory ---

// In-place lower Cholesky of the R x R matrix G (column-major, ld R) by one
// warp (lane = row).  Returns false on a non-positive or non-finite pivot.
__device__ bool warp_chol(double* G, int R) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < R; ++k) {
    double piv = G[k + R * k];
    if (!(piv > 0.0) || !isfinite(piv)) ok = false;
    const double dk = sqrt(piv);
    __syncwarp();
    if (lane == k) G[k + R * k] = dk;
    if (lane > k && lane < R) G[lane + R * k] /= dk;
    __syncwarp();
    if (lane > k && lane < R) {
      const double lik = G[lane + R * k];
      for (int l = k + 1; l <= lane; ++l) G[lane + R * l] -= lik * G[l + R * k];
    }
    __syncwarp();
  }
  return ok;
}

// z <- L^{-1} z (forward substitution, L lower in G), one warp.
__device__ void warp_fwd(const double* L, double* z, int R) {
  const int lane = threadIdx.x & 31;
  for (int p = 0; p < R; ++p) {
    __syncwarp();
    const double zp = z[p] / L[p + R * p];
    __syncwarp();
    if (lane == p) z[p] = zp;
    if (lane > p && lane < R) z[lane] -= L[lane + R * p] * zp;
  }
  __syncwarp();
}

// z <- L^{-T} z (back substitution with L^T), one warp.
__device__ void warp_bwd(const double* L, double* z, int R) {
  const int lane = threadIdx.x & 31;
  for (int p = R - 1; p >= 0; --p) {
    __syncwarp();
    const double zp = z[p] / L[p + R * p];
    __syncwarp();
    if (lane == p) z[p] = zp;
    if (lane < p) z[lane] -= L[p + R * lane] * zp;
  }
  __syncwarp();
}

// CTA (n, j), one warp: column j of Gt^(n), U_n, L_n (chol C^(n)) and w_n.
//   Gt[:, j] = L_G^{-T} L_G^{-1} e_j;  U[:, j] = L_G^{-T} e_j
//   w_n[:, j] = P^(n) Gt[:, j] - C^(n) (Gamma^(n) Gt[:, j])     (Appendix D)
__global__ void __launch_bounds__(32) k_mode_prep(Dims d, const double* C, const double* Gnm,
                                                  const double* P, const double* mu, double* Gt,
                                                  double* U, double* LC, double* w, int* info,
                                                  const int* skip) {
  if (skip && *skip) return;
  __shared__ double G[CP_MAX_R * CP_MAX_R];
  __shared__ double Lc[CP_MAX_R * CP_MAX_R];
  __shared__ double z[CP_MAX_R], u[CP_MAX_R], v[CP_MAX_R];
  const int R = d.R, RR = d.RR, N = d.N;
  const int n = blockIdx.x / R, j = blockIdx.x % R;
  const int lane = threadIdx.x;
  const double* Gam = Gnm + (int64_t(n) * N + n) * RR;
  const double* Cn = C + int64_t(n) * RR;
  const double muv = *mu;
  for (int e = lane; e < RR; e += 32) {
    G[e] = Gam[e] + ((e % R) == (e / R) ? muv : 0.0);
    Lc[e] = Cn[e];
  }
  __syncwarp();
  const bool okG = warp_chol(G, R);
  const bool okC = warp_chol(Lc, R);
  if (lane == 0 && j == 0 && info && (!okG || !okC)) atomicCAS(info, 0, n + 1);
  if (lane < R) {
    z[lane] = (lane == j) ? 1.0 : 0.0;
    u[lane] = (lane == j) ? 1.0 : 0.0;
  }
  __syncwarp();
  warp_fwd(G, z, R);
  warp_bwd(G, z, R);   // z = Gt e_j
  warp_bwd(G, u, R);   // u = L_G^{-T} e_j
  if (lane < R) {
    double s = 0.0;
    for (int c = 0; c < R; ++c) s = fma(Gam[lane + R * c], z[c], s);
    v[lane] = s;
  }
  __syncwarp();
  if (lane < R) {
    const int64_t o = int64_t(n) * RR + lane + int64_t(R) * j;
    double s = 0.0;
    const double* Pn = P + int64_t(n) * RR;
    for (int c = 0; c < R; ++c) s = fma(Pn[lane + R * c], z[c], s);
    double t = 0.0;
    for (int c = 0; c < R; ++c) t = fma(Cn[lane + R * c], v[c], t);
    Gt[o] = z[lane];
    U[o] = u[lane];
    LC[o] = (lane >= j) ? Lc[lane + R * j] : 0.0;
    if (w) w[o] = s - t;
  }
}

int launch_mode_prep(const Dims& d, const double* C, const double* Gnm, const double* P,
                     const double* mu, double* Gt, double* U, double* LC, double* w, int* info,
                     const int* skip, cudaStream_t s) {
  k_mode_prep<<<d.N * d.R, 32, 0, s>>>(d, C, Gnm, P, mu, Gt, U, LC, w, info, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

// ---------------------------------------------------------------------------
// core = I + S^T K S, lower triangle
// ---------------------------------------------------------------------------

// pair p -> (n, m) with n > m, enumerated row by row: (1,0), (2,0), (2,1), ...
__device__ __forceinline__ void pair_of(int p, int* n, int* m) {
  int nn = 1;
  while ((nn * (nn + 1)) / 2 <= p) ++nn;
  *n = nn;
  *m = p - (nn * (nn - 1)) / 2;
}

// W_nm[a + R (k + R j)] = sum_b Gamma^(n,m)[a,b] L_m[b,k] U_n[b,j]; one thread per entry.
__global__ void k_core_w(Dims d, const double* Gnm, const double* LC, const double* U, double* Wp,
                         const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR, N = d.N;
  const int64_t R3 = int64_t(RR) * R;
  const int64_t npairs = int64_t(N) * (N - 1) / 2;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= npairs * R3) return;
  const int p = int(idx / R3);
  const int e = int(idx % R3);
  const int a = e % R, k = (e / R) % R, j = e / RR;
  int n, m;
  pair_of(p, &n, &m);
  const double* G = Gnm + (int64_t(n) * N + m) * RR;
  const double* Lm = LC + int64_t(m) * RR;
  const double* Un = U + int64_t(n) * RR;
  double s = 0.0;
  // L_m[b,k] = 0 for b < k and U_n[b,j] = 0 for b > j
  for (int b = k; b <= j; ++b) s = fma(G[a + R * b], Lm[b + R * k] * Un[b + R * j], s);
  Wp[idx] = s;
}

// One CTA per column of a lower block (n > m) or of a diagonal block;
// R^2 threads, thread = row i + R j inside the block.
template <typename T>
__global__ void k_core_fill(Dims d, const double* LC, const double* U, const double* Wp, T* core,
                            int64_t ld, const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR, N = d.N;
  const int npairs = N * (N - 1) / 2;
  const int blk = blockIdx.x / RR;       // 0..npairs-1: lower pairs; npairs..: diagonal blocks
  const int kap = blockIdx.x % RR;       // column inside the block: k + R l
  const int rho = threadIdx.x;           // row inside the block: i + R j
  if (blk >= npairs) {
    const int n = blk - npairs;
    if (rho < RR && rho >= kap)
      core[(int64_t(n) * RR + rho) + ld * (int64_t(n) * RR + kap)] = T(rho == kap ? 1 : 0);
    return;
  }
  int n, m;
  pair_of(blk, &n, &m);
  __shared__ T Ln[CP_MAX_R * CP_MAX_R];
  __shared__ T Uml[CP_MAX_R];
  __shared__ T Wk[CP_MAX_R * CP_MAX_R];   // W_nm[a, (k, j)] for this k, all a, j
  const int k = kap % R, l = kap / R;
  const double* W = Wp + int64_t(blk) * RR * R;
  for (int e = rho; e < RR; e += blockDim.x) {
    Ln[e] = T(LC[int64_t(n) * RR + e]);
    const int a = e % R, j = e / R;
    Wk[e] = T(W[a + R * (k + R * j)]);
  }
  if (rho < R) Uml[rho] = T(U[int64_t(m) * RR + rho + R * l]);
  __syncthreads();
  if (rho >= RR) return;
  const int i = rho % R, j = rho / R;
  T s = T(0);
  // L_n[a,i] = 0 for a < i and U_m[a,l] = 0 for a > l
  for (int a = i; a <= l; ++a) s = fma(Ln[a + R * i] * Uml[a], Wk[a + R * j], s);
  core[(int64_t(n) * RR + rho) + ld * (int64_t(m) * RR + kap)] = s;
}

template <typename T>
int launch_core_fill(const Dims& d, const double* LC, const double* U, const double* Wp, T* core,
                     const int* skip, cudaStream_t s) {
  const int npairs = d.N * (d.N - 1) / 2;
  int threads = ((d.RR + 31) / 32) * 32;
  k_core_fill<T><<<(npairs + d.N) * d.RR, threads, 0, s>>>(d, LC, U, Wp, core, d.ncore, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
template int launch_core_fill<double>(const Dims&, const double*, const double*, const double*,
                                      double*, const int*, cudaStream_t);
template int launch_core_fill<float>(const Dims&, const double*, const double*, const double*,
                                     float*, const int*, cudaStream_t);

int launch_core_w(const Dims& d, const double* Gnm, const double* LC, const double* U, double* Wp,
                  const int* skip, cudaStream_t s) {
  const int64_t tot = int64_t(d.N) * (d.N - 1) / 2 * d.RR * d.R;
  if (tot == 0) return CP_OK;
  k_core_w<<<unsigned((tot + 127) / 128), 128, 0, s>>>(d, Gnm, LC, U, Wp, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

// ---------------------------------------------------------------------------
// Matrix-free float64 operators on vectors of length N R^2
// ---------------------------------------------------------------------------

// out = K x  (or out = base - K x when base != null), one thread per entry.
//   (K x)_n[i + R j] = sum_{m != n} Gamma^(n,m)[i,j] X_m[j,i]
__global__ void k_apply_K(Dims d, const double* Gnm, const double* x, const double* base, double* out,
                          const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR, N = d.N;
  int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= d.ncore) return;
  const int n = int(idx / RR), e = int(idx % RR);
  const int i = e % R, j = e / R;
  double s = 0.0;
  for (int m = 0; m < N; ++m)
    if (m != n) s = fma(Gnm[(int64_t(n) * N + m) * RR + e], x[int64_t(m) * RR + j + R * i], s);
  out[idx] = base ? base[idx] - s : s;
}

// out_m = vec(L_m X_m U_m^T): CTA (m, q) computes column q with one warp.
__global__ void __launch_bounds__(32) k_apply_S(Dims d, const double* LC, const double* U,
                                                const double* x, double* out, const int* skip) {
  if (skip && *skip) return;
  __shared__ double t[CP_MAX_R];
  const int R = d.R, RR = d.RR;
  const int m = blockIdx.x / R, q = blockIdx.x % R;
  const int lane = threadIdx.x;
  const double* X = x + int64_t(m) * RR;
  const double* Um = U + int64_t(m) * RR;
  const double* Lm = LC + int64_t(m) * RR;
  if (lane < R) {   // t = X U_m[q, :]^T ; U_m upper: U_m[q,l] = 0 for l < q
    double s = 0.0;
    for (int l = q; l < R; ++l) s = fma(X[lane + R * l], Um[q + R * l], s);
    t[lane] = s;
  }
  __syncwarp();
  if (lane < R) {   // out[:, q] = L_m t ; L_m lower: L_m[p,k] = 0 for k > p
    double s = 0.0;
    for (int k = 0; k <= lane; ++k) s = fma(Lm[lane + R * k], t[k], s);
    out[int64_t(m) * RR + lane + R * q] = s;
  }
}

// out_n = vec(L_n^T V_n U_n) where V_n = x_n (kx = 0) or V_n = (K x)_n (kx = 1);
// if res != null: out = res_base - y - out  (refinement residual b - y - S^T K S y).
__global__ void __launch_bounds__(32) k_apply_ST(Dims d, const double* LC, const double* U,
                                                 const double* Gnm, const double* x, int kx,
                                                 const double* b, const double* y, double* out,
                                                 const int* skip) {
  if (skip && *skip) return;
  __shared__ double V[CP_MAX_R * CP_MAX_R];
  __shared__ double t[CP_MAX_R];
  const int R = d.R, RR = d.RR, N = d.N;
  const int n = blockIdx.x / R, q = blockIdx.x % R;
  const int lane = threadIdx.x;
  for (int e = lane; e < RR; e += 32) {
    if (kx) {
      const int i = e % R, j = e / R;
      double s = 0.0;
      for (int m = 0; m < N; ++m)
        if (m != n) s = fma(Gnm[(int64_t(n) * N + m) * RR + e], x[int64_t(m) * RR + j + R * i], s);
      V[e] = s;
    } else {
      V[e] = x[int64_t(n) * RR + e];
    }
  }
  __syncwarp();
  const double* Un = U + int64_t(n) * RR;
  const double* Ln = LC + int64_t(n) * RR;
  if (lane < R) {   // t = V U_n[:, q] ; U_n[l,q] = 0 for l > q
    double s = 0.0;
    for (int l = 0; l <= q; ++l) s = fma(V[lane + R * l], Un[l + R * q], s);
    t[lane] = s;
  }
  __syncwarp();
  if (lane < R) {   // out[:, q] = L_n^T t ; L_n[k,p] = 0 for k < p
    double s = 0.0;
    for (int k = lane; k < R; ++k) s = fma(Ln[k + R * lane], t[k], s);
    const int64_t o = int64_t(n) * RR + lane + R * q;
    out[o] = b ? (b[o] - y[o] - s) : s;
  }
}

int launch_apply_K(const Dims& d, const double* Gnm, const double* x, const double* base, double* out,
                   const int* skip, cudaStream_t s) {
  k_apply_K<<<unsigned((d.ncore + 127) / 128), 128, 0, s>>>(d, Gnm, x, base, out, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
int launch_apply_S(const Dims& d, const double* LC, const double* U, const double* x, double* out,
                   const int* skip, cudaStream_t s) {
  k_apply_S<<<d.N * d.R, 32, 0, s>>>(d, LC, U, x, out, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
int launch_apply_ST(const Dims& d, const double* LC, const double* U, const double* Gnm,
                    const double* x, int kx, const double* b, const double* y, double* out,
                    const int* skip, cudaStream_t s) {
  k_apply_ST<<<d.N * d.R, 32, 0, s>>>(d, LC, U, Gnm, x, kx, b, y, out, skip);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn
