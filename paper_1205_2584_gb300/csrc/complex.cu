// Complex-valued tensors (Sec. 5, Theorems 5-8): the damped Gauss-Newton
// step for a complex128 tensor with complex factors, all on the device.
//
// With C^(n) = A^(n)H A^(n) (Hermitian), Gamma^(n,m) = Hadamard_{k != n,m} C^(k),
// the Hessian J^H J = G + Z K Z^H (Theorem 7) with G = blkdiag(Gamma^(n) kron I),
// Z = blkdiag(I_R kron A^(n)), K^(n,m) = P_R diag(vec Gamma^(n,m)), and the
// gradient blocks G_n = E_(n) conj(KR_n) = Y_(n) conj(KR_n) - A^(n) Gamma^(n)T
// (Theorem 7, Eq. grad_complex_g).  The step (Theorem 8) in the Hermitian
// positive definite core form used for real tensors:
//   Gt^(n) = (Gamma^(n) + mu I)^{-1} = U_n U_n^H, U_n = L_G^{-H}, Gamma^(n) + mu I = L_G L_G^H,
//   C^(n) = L_n L_n^H,  S_n = U_n kron L_n  (S S^H = Psi_mu),
//   w_n = vec(A^(n)H G_n Gt^(n)T),  core = I + S^H K S,
//   f = K w - K S core^{-1} S^H K w,  Delta_n = (G_n - A^(n) F_n) Gt^(n)T
// (in matrix form the damped inverse acts as X -> X Gt^T).  The core is
// solved through its real representation [[Re, -Im], [Im, Re]] (symmetric
// positive definite, size 2 N R^2) by the float64 Cholesky of the real path.
// Control: accept iff the residual decreased, gain ratio with denominator
// Re(Delta^H (g + mu Delta)), Nielsen's rule, equal-energy normalisation with
// real positive scales, the same stop tests.
//
// Layout: complex numbers are interleaved (re, im) float64 pairs; Y is
// first-index-fastest like the real tensors; the factor vector a holds
// vec A^(1), ..., vec A^(N) (Eq. vecV) in complex entries.  Limits: R <= 16,
// I_1 <= 256, N R^2 <= 3200 (2 N R^2 <= 6400 for the real core).
#include <new>

#include "common.cuh"

namespace cpdgn {

int chol64_factor(double* A, int64_t n, double* dinv, int* info, void* sync, int* tmo, const int* skip,
                  cudaStream_t s);
int chol64_solve(const double* L, const double* dinv, int64_t n, const double* b, double* z, double* y,
                 void* sync, int* info, int* tmo, const int* skip, cudaStream_t s);
size_t chol64_sync_bytes(int64_t n);
size_t chol64_dinv_bytes(int64_t n);
int tc_timeout_counter(int** out);

constexpr int kCMaxR = 16;
constexpr int kCMaxI1 = 256;

typedef double2 cplx;
__device__ __forceinline__ cplx cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
// c + a b
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c + a conj(b)
__device__ __forceinline__ cplx cfmac(cplx a, cplx b, cplx c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.y, b.x, fma(-a.x, b.y, c.y)));
}
__device__ __forceinline__ cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ void catomic(cplx* p, cplx v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// scalar slots
enum { CS_R2 = 0, CS_R2T = 1, CS_YN2 = 2, CS_DEN = 3, CS_NRM = 8 };   // CS_NRM..: N R column norms^2
enum { CI_INFO = 0, CI_COMMIT = 1, CI_TOBASE = 2 };

struct CBufs {
  cp_status* status;
  cplx *G, *Gtr, *at, *delta;
  cplx *C, *Gnm, *P, *U, *LC, *Gt, *w, *Kw, *b, *Z, *KZ, *f;
  double *b2, *z2, *y2, *core2, *dinv, *scal, *scale;
  void* sync;
  int* info;
};

struct CLayout {
  size_t off[24];
  size_t total;
};

static void c_layout(const Dims& d, CLayout* L) {
  const size_t cs = sizeof(cplx);
  const size_t RT = size_t(d.T) * d.R, NRR = size_t(d.N) * d.RR, n = size_t(d.ncore), n2 = 2 * n;
  size_t sz[24] = {0};
  sz[0] = sizeof(cp_status);
  sz[1] = sz[2] = sz[3] = sz[4] = RT * cs;                // G, Gtr, at, delta
  sz[5] = NRR * cs;                                       // C
  sz[6] = size_t(d.N) * NRR * cs;                         // Gnm
  sz[7] = sz[8] = sz[9] = sz[10] = NRR * cs;              // P, U, LC, Gt
  sz[11] = sz[12] = sz[13] = sz[14] = sz[15] = sz[16] = n * cs;   // w, Kw, b, Z, KZ, f
  sz[17] = sz[18] = sz[19] = n2 * sizeof(double);         // b2, z2, y2
  sz[20] = n2 * n2 * sizeof(double);                      // core2
  sz[21] = chol64_dinv_bytes(int64_t(n2));                // dinv
  sz[22] = chol64_sync_bytes(int64_t(n2)) + 64 * sizeof(double) + size_t(d.N) * d.R * sizeof(double) +
           64 * sizeof(int) + 256;                        // sync, scal, scale, info
  size_t o = 0;
  for (int i = 0; i < 23; ++i) {
    L->off[i] = o;
    o += align256(sz[i]);
  }
  L->total = o;
}

static CBufs c_carve(const Dims& d, const CLayout& L, void* ws) {
  char* b = static_cast<char*>(ws);
  CBufs B;
  B.status = reinterpret_cast<cp_status*>(b + L.off[0]);
  B.G = reinterpret_cast<cplx*>(b + L.off[1]);
  B.Gtr = reinterpret_cast<cplx*>(b + L.off[2]);
  B.at = reinterpret_cast<cplx*>(b + L.off[3]);
  B.delta = reinterpret_cast<cplx*>(b + L.off[4]);
  B.C = reinterpret_cast<cplx*>(b + L.off[5]);
  B.Gnm = reinterpret_cast<cplx*>(b + L.off[6]);
  B.P = reinterpret_cast<cplx*>(b + L.off[7]);
  B.U = reinterpret_cast<cplx*>(b + L.off[8]);
  B.LC = reinterpret_cast<cplx*>(b + L.off[9]);
  B.Gt = reinterpret_cast<cplx*>(b + L.off[10]);
  B.w = reinterpret_cast<cplx*>(b + L.off[11]);
  B.Kw = reinterpret_cast<cplx*>(b + L.off[12]);
  B.b = reinterpret_cast<cplx*>(b + L.off[13]);
  B.Z = reinterpret_cast<cplx*>(b + L.off[14]);
  B.KZ = reinterpret_cast<cplx*>(b + L.off[15]);
  B.f = reinterpret_cast<cplx*>(b + L.off[16]);
  B.b2 = reinterpret_cast<double*>(b + L.off[17]);
  B.z2 = reinterpret_cast<double*>(b + L.off[18]);
  B.y2 = reinterpret_cast<double*>(b + L.off[19]);
  B.core2 = reinterpret_cast<double*>(b + L.off[20]);
  B.dinv = reinterpret_cast<double*>(b + L.off[21]);
  char* t = b + L.off[22];
  B.sync = t;
  t += align256(chol64_sync_bytes(2 * d.ncore));
  B.scal = reinterpret_cast<double*>(t);
  t += 64 * sizeof(double);
  B.scale = reinterpret_cast<double*>(t);
  t += size_t(d.N) * d.R * sizeof(double);
  B.info = reinterpret_cast<int*>(t);
  return B;
}

// ---------------------------------------------------------------------------
// Gramians: C^(n) = A^(n)H A^(n), P^(n) = A^(n)H G_n (if G), Gamma^(n,m).
// ---------------------------------------------------------------------------
__global__ void k_cgram(Dims d, const cplx* a, const cplx* G, cplx* C, cplx* P, const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int which = (G != nullptr) ? 2 : 1;
  if (e >= which * d.N * RR) return;
  const int part = e / (d.N * RR), q = e % (d.N * RR), n = q / RR, r = (q % RR) % R, s = (q % RR) / R;
  const int64_t In = d.I[n];
  const cplx* An = a + d.aoff[n];
  const cplx* Bn = (part == 0) ? An : G + d.aoff[n];
  cplx acc = cz();
  for (int64_t i = 0; i < In; ++i) acc = cfmac(Bn[i + In * s], An[i + In * r], acc);   // conj(A[i,r]) B[i,s]
  (part == 0 ? C : P)[int64_t(n) * RR + r + R * s] = acc;
}

__global__ void k_chad(Dims d, const cplx* C, cplx* Gnm, const int* skip) {
  if (skip && *skip) return;
  const int RR = d.RR, N = d.N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N * RR) return;
  const int nm = e / RR, q = e % RR, n = nm / N, m = nm % N;
  cplx v = make_double2(1.0, 0.0);
  for (int k = 0; k < N; ++k)
    if (k != n && k != m) v = cmul(v, C[int64_t(k) * RR + q]);
  Gnm[e] = v;
}

// lower Cholesky of the Hermitian R x R matrix M (column-major, in place, in
// shared memory) by one thread; false on a non-positive or non-finite pivot
__device__ bool cchol(cplx* M, int R) {
  bool ok = true;
  for (int j = 0; j < R; ++j) {
    double dj = M[j + R * j].x;
    for (int k = 0; k < j; ++k) dj -= M[j + R * k].x * M[j + R * k].x + M[j + R * k].y * M[j + R * k].y;
    if (!(dj > 0.0) || !isfinite(dj)) {
      ok = false;
      dj = 1.0;
    }
    const double ljj = sqrt(dj), inv = 1.0 / ljj;
    M[j + R * j] = make_double2(ljj, 0.0);
    for (int i = j + 1; i < R; ++i) {
      cplx s = M[i + R * j];
      for (int k = 0; k < j; ++k) s = csub(s, cmul(M[i + R * k], cconj(M[j + R * k])));
      M[i + R * j] = cscale(s, inv);
    }
    for (int i = 0; i < j; ++i) M[i + R * j] = cz();
  }
  return ok;
}

// inverse of the lower triangular R x R matrix L (column-major), one thread
__device__ void ctrinv(const cplx* L, cplx* X, int R) {
  for (int c = 0; c < R; ++c)
    for (int i = 0; i < R; ++i) {
      if (i < c) { X[i + R * c] = cz(); continue; }
      cplx s = (i == c) ? make_double2(1.0, 0.0) : cz();
      for (int k = c; k < i; ++k) s = csub(s, cmul(L[i + R * k], X[k + R * c]));
      const cplx l = L[i + R * i];
      X[i + R * c] = cscale(s, 1.0 / l.x);   // diagonal of a Cholesky factor is real positive
    }
}

// Per mode n (one CTA of 32 threads): U_n = L_G^{-H}, Gt^(n) = U U^H,
// L_n = chol(C^(n)), w_n = vec(P^(n) Gt^T) (P = A^H G).
__global__ void k_cprep(Dims d, const cplx* C, const cplx* Gnm, const cplx* P, const double* mu, cplx* U, cplx* LC,
                        cplx* Gt, cplx* w, int* info, const int* skip) {
  if (skip && *skip) return;
  __shared__ cplx M[kCMaxR * kCMaxR], X[kCMaxR * kCMaxR], Uu[kCMaxR * kCMaxR], Gs[kCMaxR * kCMaxR];
  const int n = blockIdx.x, R = d.R, RR = d.RR, tid = threadIdx.x;
  const double muv = *mu;
  for (int e = tid; e < RR; e += blockDim.x) {
    cplx v = Gnm[(int64_t(n) * d.N + n) * RR + e];
    if (e % R == e / R) v.x += muv;
    M[e] = v;
  }
  __syncthreads();
  if (tid == 0) {
    const bool ok = cchol(M, R);
    if (!ok && info) atomicCAS(info, 0, n + 1);
    ctrinv(M, X, R);                                  // L_G^{-1}
    for (int i = 0; i < R; ++i)
      for (int j = 0; j < R; ++j) Uu[i + R * j] = cconj(X[j + R * i]);   // U = L_G^{-H}
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) {
    const int i = e % R, j = e / R;
    U[int64_t(n) * RR + e] = Uu[e];
    cplx s = cz();
    for (int k = 0; k < R; ++k) s = cfmac(Uu[i + R * k], Uu[j + R * k], s);   // (U U^H)[i, j]
    Gs[e] = s;
    Gt[int64_t(n) * RR + e] = s;
  }
  __syncthreads();
  if (w) {
    for (int e = tid; e < RR; e += blockDim.x) {
      const int r = e % R, c = e / R;
      cplx s = cz();
      for (int k = 0; k < R; ++k) s = cfma(P[int64_t(n) * RR + r + R * k], Gs[c + R * k], s);   // P Gt^T
      w[int64_t(n) * RR + e] = s;
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int e = 0; e < RR; ++e) M[e] = C[int64_t(n) * RR + e];
    const bool ok = cchol(M, R);
    if (!ok && info) atomicCAS(info, 0, n + 1);
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) LC[int64_t(n) * RR + e] = M[e];
}

// out = K x (+ base - (K x) when base is given: out = base - K x).
// (K x)_n[i + R j] = sum_{m != n} Gamma^(n,m)[j, i] x_m[j + R i].
__global__ void k_capplyK(Dims d, const cplx* Gnm, const cplx* x, const cplx* base, cplx* out, const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR, N = d.N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.ncore) return;
  const int n = e / RR, q = e % RR, i = q % R, j = q / R;
  cplx s = cz();
  for (int m = 0; m < N; ++m)
    if (m != n) s = cfma(Gnm[(int64_t(n) * N + m) * RR + j + R * i], x[int64_t(m) * RR + j + R * i], s);
  out[e] = base ? csub(base[e], s) : s;
}

// out = S^H y: out_n[i + R j] = sum_{a,b} conj(L_n[a, i]) y_n[a + R b] conj(U_n[b, j]);
// also the real right-hand side b2 = [Re out; Im out] when b2 != null
__global__ void k_capplySH(Dims d, const cplx* LC, const cplx* U, const cplx* y, cplx* out, double* b2,
                           const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.ncore) return;
  const int n = e / RR, q = e % RR, i = q % R, j = q / R;
  const cplx* L = LC + int64_t(n) * RR;
  const cplx* Un = U + int64_t(n) * RR;
  const cplx* Y = y + int64_t(n) * RR;
  cplx s = cz();
  for (int b = 0; b < R; ++b) {
    cplx t = cz();
    for (int a = 0; a < R; ++a) t = cfmac(Y[a + R * b], L[a + R * i], t);   // conj(L[a, i]) Y[a, b]
    s = cfmac(t, Un[b + R * j], s);                                          // * conj(U[b, j])
  }
  out[e] = s;
  if (b2) {
    b2[e] = s.x;
    b2[e + d.ncore] = s.y;
  }
}

// out = S y (y from the real solution y2 when y2 != null): out_n[i + R j] =
// sum_{a,b} L_n[i, a] y_n[a + R b] U_n[j, b]
__global__ void k_capplyS(Dims d, const cplx* LC, const cplx* U, const double* y2, cplx* out, const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.ncore) return;
  const int n = e / RR, q = e % RR, i = q % R, j = q / R;
  const cplx* L = LC + int64_t(n) * RR;
  const cplx* Un = U + int64_t(n) * RR;
  cplx s = cz();
  for (int b = 0; b < R; ++b) {
    cplx t = cz();
    for (int a = 0; a < R; ++a) {
      const int64_t k = int64_t(n) * RR + a + R * b;
      t = cfma(L[i + R * a], make_double2(y2[k], y2[k + d.ncore]), t);
    }
    s = cfma(t, Un[j + R * b], s);
  }
  out[e] = s;
}

// Real representation of core = I + S^H K S, lower triangle of the 2n x 2n
// matrix [[Re, -Im], [Im, Re]] (column-major).  Thread = complex entry (p, q),
// p >= q: c_pq = delta_pq + sum_{a,b} conj(L_n[b,i]) conj(U_n[a,j]) Gamma^(n,m)[a,b] L_m[a,k] U_m[b,l]
// for p = (n, i + R j), q = (m, k + R l), n != m.
__global__ void k_ccore_fill(Dims d, const cplx* LC, const cplx* U, const cplx* Gnm, double* core2,
                             const int* skip) {
  if (skip && *skip) return;
  const int64_t n = d.ncore, n2 = 2 * n;
  const int R = d.R, RR = d.RR, N = d.N;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = e % n, q = e / n;
    if (p < q) continue;
    const int bn = int(p / RR), bm = int(q / RR);
    cplx c = (p == q) ? make_double2(1.0, 0.0) : cz();
    if (bn != bm) {
      const int x = int(p % RR), y = int(q % RR), i = x % R, j = x / R, k = y % R, l = y / R;
      const cplx* Ln = LC + int64_t(bn) * RR;
      const cplx* Un = U + int64_t(bn) * RR;
      const cplx* Lm = LC + int64_t(bm) * RR;
      const cplx* Um = U + int64_t(bm) * RR;
      const cplx* Gm = Gnm + (int64_t(bn) * N + bm) * RR;
      for (int b = 0; b < R; ++b) {
        cplx t = cz();
        for (int a = 0; a < R; ++a) {
          // conj(U_n[a, j]) Gamma[a, b] L_m[a, k]
          const cplx g = cmul(Gm[a + R * b], Lm[a + R * k]);
          t = cfmac(g, Un[a + R * j], t);
        }
        // conj(L_n[b, i]) t U_m[b, l]
        c = cfmac(cmul(t, Um[b + R * l]), Ln[b + R * i], c);
      }
    }
    core2[p + n2 * q] = c.x;
    core2[(p + n) + n2 * (q + n)] = c.x;
    core2[(p + n) + n2 * q] = c.y;
    if (p > q) core2[(q + n) + n2 * p] = -c.y;
  }
}

// The pass over a complex tensor at factors a: gradient blocks
// G_n = E_(n) conj(KR_n) (zeroed by the caller) and ||E||^2.  CTA = range of
// mode-1 fibres; thread i = row of the fibre (I_1 <= 256); per fibre the
// Khatri-Rao row kr_f, e = y_f - A^(1) kr_f, G_1 += e conj(kr_f) (registers),
// t_f = A^(1)H e (shared), G_n[i_n] += t_f conj(prod_{k >= 2, k != n} A^(k)[i_k]).
template <int RM>
__global__ void __launch_bounds__(kCMaxI1) k_cpass(Dims d, const cplx* Y, const cplx* a, cplx* G, double* r2,
                                                   int64_t fib_per_cta, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ cplx a1dyn[];
  cplx (*A1s)[RM] = reinterpret_cast<cplx (*)[RM]>(a1dyn);      // I_1 x RM
  __shared__ cplx kr[RM], t[RM], loo[CP_MAX_N][RM];
  __shared__ cplx es[kCMaxI1];
  __shared__ int idx[CP_MAX_N];
  __shared__ double red[kCMaxI1];
  const int R = d.R, N = d.N, tid = threadIdx.x;
  const int I1 = int(d.I[0]);
  for (int e = tid; e < I1 * R; e += blockDim.x) A1s[e % I1][e / I1] = a[e];
  cplx acc[RM];
#pragma unroll
  for (int r = 0; r < RM; ++r) acc[r] = cz();
  double e2 = 0.0;
  const int64_t f0 = int64_t(blockIdx.x) * fib_per_cta;
  int64_t f1 = f0 + fib_per_cta;
  if (f1 > d.nfib) f1 = d.nfib;
  __syncthreads();
  for (int64_t f = f0; f < f1; ++f) {
    if (tid == 0) {
      int64_t rem = f;
      for (int k = 1; k < N; ++k) {
        idx[k] = int(rem % d.I[k]);
        rem /= d.I[k];
      }
    }
    __syncthreads();
    if (tid < R) {
      const int r = tid;
      cplx v[CP_MAX_N];
      for (int k = 1; k < N; ++k) v[k] = a[d.aoff[k] + idx[k] + d.I[k] * r];
      cplx p = make_double2(1.0, 0.0);
      for (int k = 1; k < N; ++k) p = cmul(p, v[k]);
      kr[r] = p;
      for (int n = 1; n < N; ++n) {
        cplx l = make_double2(1.0, 0.0);
        for (int k = 1; k < N; ++k)
          if (k != n) l = cmul(l, v[k]);
        loo[n][r] = l;
      }
    }
    __syncthreads();
    if (tid < I1) {
      const cplx y = Y[int64_t(tid) + int64_t(I1) * f];
      cplx yh = cz();
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) yh = cfma(A1s[tid][r], kr[r], yh);
      const cplx e = csub(y, yh);
      e2 = fma(e.x, e.x, fma(e.y, e.y, e2));
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) acc[r] = cfmac(e, kr[r], acc[r]);
      es[tid] = e;
    }
    __syncthreads();
    if (G && tid < R) {
      cplx s = cz();
      for (int i = 0; i < I1; ++i) s = cfmac(es[i], A1s[i][tid], s);   // e_i conj(A1[i, r])
      t[tid] = s;
      for (int n = 1; n < N; ++n)
        catomic(G + d.aoff[n] + idx[n] + d.I[n] * tid, cmul(s, cconj(loo[n][tid])));
    }
    __syncthreads();
  }
  if (G && tid < I1) {
#pragma unroll
    for (int r = 0; r < RM; ++r)
      if (r < R) catomic(G + tid + int64_t(I1) * r, acc[r]);
  }
  red[tid] = e2;
  __syncthreads();
  for (int s = kCMaxI1 / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0 && r2) atomicAdd(r2, red[0]);
}

// Delta_n = (G_n - A^(n) F_n) Gt^(n)T, trial factors, Re(Delta^H (g + mu Delta)),
// squared column norms of the trial factors.  Thread = (mode, row).
__global__ void k_cupdate(Dims d, const cplx* a, const cplx* G, const cplx* f, const cplx* Gt, const double* mu,
                          cplx* delta, cplx* at, double* scal, const int* skip) {
  if (skip && *skip) return;
  const int R = d.R, RR = d.RR;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= d.T) return;
  int n = 0;
  while (n + 1 < d.N && e >= d.row0[n + 1]) ++n;
  const int64_t In = d.I[n], i = e - d.row0[n];
  const cplx* An = a + d.aoff[n];
  const cplx* Gn = G + d.aoff[n];
  const cplx* F = f + int64_t(n) * RR;
  const cplx* T = Gt + int64_t(n) * RR;
  cplx h[kCMaxR];
  for (int c = 0; c < R; ++c) {
    cplx s = Gn[i + In * c];
    for (int k = 0; k < R; ++k) s = csub(s, cmul(An[i + In * k], F[k + R * c]));
    h[c] = s;
  }
  const double muv = *mu;
  double den = 0.0;
  for (int r = 0; r < R; ++r) {
    cplx dl = cz();
    for (int c = 0; c < R; ++c) dl = cfma(h[c], T[r + R * c], dl);   // Gt^T[c, r] = Gt[r, c]
    const cplx g = Gn[i + In * r];
    const cplx gm = make_double2(g.x + muv * dl.x, g.y + muv * dl.y);
    den += dl.x * gm.x + dl.y * gm.y;                                 // Re(conj(dl) (g + mu dl))
    delta[d.aoff[n] + i + In * r] = dl;
    const cplx av = cadd(An[i + In * r], dl);
    at[d.aoff[n] + i + In * r] = av;
    atomicAdd(scal + CS_NRM + n * R + r, av.x * av.x + av.y * av.y);
  }
  atomicAdd(scal + CS_DEN, den);
}

__global__ void k_cbegin(Dims d, double* scal, int* info, cplx* Gtr, const cp_status* st) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i == 0) {
    info[CI_INFO] = 0;
    info[CI_COMMIT] = 0;
  }
  if (i < 64 && i != CS_R2 && i != CS_YN2) scal[i] = 0.0;
  for (int64_t e = i; e < d.T * d.R; e += int64_t(gridDim.x) * blockDim.x) Gtr[e] = cz();
}

__global__ void k_ccontrol(Dims d, cp_opts o, cp_status* st, double* scal, int* info, double* scale,
                           const int* tmo) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (st->stop != CP_RUNNING) return;
  const int R = d.R, N = d.N;
  const double r2 = st->resid2, r2t = scal[CS_R2T], den = scal[CS_DEN];
  const int bad = info[CI_INFO];
  const bool finite = isfinite(r2t) && isfinite(den);
  const bool accept = (bad == 0) && finite && (r2t < r2);
  const double rho = (bad == 0 && finite && den > 0.0) ? (r2 - r2t) / den : 0.0;
  if (bad == 0 && !finite && st->error == 0) st->error = CP_ENONFINITE;
  double mu = st->mu, nu = st->nu;
  if (rho > 0.0) {
    const double tt = 2.0 * rho - 1.0;
    const double fac = 1.0 - tt * tt * tt;
    mu *= (fac > 1.0 / 3.0) ? fac : 1.0 / 3.0;
    nu = 2.0;
  } else {
    mu *= nu;
    nu *= 2.0;
  }
  st->iters += 1;
  st->rho = rho;
  st->denom = den;
  st->resid2_trial = r2t;
  st->info = bad;
  st->mu = mu;
  st->nu = nu;
  st->last_accepted = accept ? 1 : 0;
  if (accept) {
    const double e_old = sqrt(r2 / st->y_norm2), e_new = sqrt(r2t / st->y_norm2);
    st->accepted += 1;
    st->resid2 = r2t;
    st->rel_err = e_new;
    scal[CS_R2] = r2t;
    if (e_old > 0.0 && fabs(e_old - e_new) < o.tol * e_old) st->stop = CP_STOP_TOL;
  }
  if (tmo && *reinterpret_cast<const volatile int*>(tmo) != info[CI_TOBASE]) {
    st->error = CP_ETIMEOUT;
    st->stop = CP_STOP_ERROR;
  }
  if (st->stop == CP_RUNNING && mu > o.mu_max) st->stop = CP_STOP_MU;
  if (st->stop == CP_RUNNING && st->iters >= o.max_iter) st->stop = CP_STOP_MAXIT;
  info[CI_COMMIT] = accept ? 1 : 0;
  // equal-energy scales (real positive: phases kept)
  for (int r = 0; r < R; ++r) {
    double lam = 1.0;
    bool pos = true;
    for (int n = 0; n < N; ++n) {
      const double nr = sqrt(scal[CS_NRM + n * R + r]);
      if (!(nr > 0.0)) pos = false;
      lam *= nr;
    }
    const double tgt = pos ? pow(lam, 1.0 / N) : 0.0;
    for (int n = 0; n < N; ++n) {
      const bool ok = o.normalize && accept && pos;
      scale[n * R + r] = ok ? tgt / sqrt(scal[CS_NRM + n * R + r]) : 1.0;
    }
  }
}

__global__ void k_ccommit(Dims d, const int* commit, const cplx* at, const cplx* Gtr, const double* scale, cplx* a,
                          cplx* G) {
  if (!*commit) return;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < d.T * d.R; e += int64_t(gridDim.x) * blockDim.x) {
    int n = 0;
    while (n + 1 < d.N && e >= d.aoff[n + 1]) ++n;
    const int r = int((e - d.aoff[n]) / d.I[n]);
    const double s = scale[n * d.R + r];
    a[e] = cscale(at[e], s);
    G[e] = cscale(Gtr[e], 1.0 / s);
  }
}

__global__ void k_csumsq(const cplx* Y, int64_t J, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < J; i += int64_t(gridDim.x) * 256)
    s = fma(Y[i].x, Y[i].x, fma(Y[i].y, Y[i].y, s));
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}

__global__ void k_cinit(Dims d, cp_opts o, const cplx* Gnm, double* scal, cp_status* st, int* info, const int* tmo) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mx = 0.0;
  for (int n = 0; n < d.N; ++n)
    for (int r = 0; r < d.R; ++r) {
      const double v = Gnm[(int64_t(n) * d.N + n) * d.RR + r + d.R * r].x;
      mx = v > mx ? v : mx;
    }
  cp_status s;
  s.mu = (o.mu0 > 0.0) ? o.mu0 : o.tau * mx;
  s.nu = 2.0;
  s.resid2 = scal[CS_R2];
  s.resid2_trial = scal[CS_R2];
  s.y_norm2 = scal[CS_YN2];
  s.rel_err = sqrt(scal[CS_R2] / scal[CS_YN2]);
  s.rho = s.denom = s.refine_resid = 0.0;
  s.reserved_d[0] = s.reserved_d[1] = s.reserved_d[2] = 0.0;
  s.iters = s.accepted = 0;
  s.stop = CP_RUNNING;
  s.error = 0;
  s.last_accepted = 0;
  s.info = 0;
  s.refine_sweeps = 0;
  s.core_f64 = 1;
  if (!isfinite(s.y_norm2) || !isfinite(s.resid2) || !isfinite(s.mu) || !(s.y_norm2 > 0.0)) {
    s.error = (isfinite(s.y_norm2) && isfinite(s.resid2) && isfinite(s.mu)) ? CP_EINVAL : CP_ENONFINITE;
    s.stop = CP_STOP_ERROR;
  }
  *st = s;
  info[CI_TOBASE] = tmo ? *reinterpret_cast<const volatile int*>(tmo) : 0;
}

static int cmake_dims(const cp_shape* shape, Dims* d) {
  if (!shape || shape->y_dtype != CP_C128) return CP_EINVAL;
  cp_shape s = *shape;
  s.y_dtype = CP_F64;
  CP_TRY(make_dims(&s, d));
  d->y_dtype = CP_C128;
  if (d->R > kCMaxR || d->I[0] > kCMaxI1 || 2 * d->ncore > 6400) return CP_EINVAL;
  return CP_OK;
}

template <int RM>
static void launch_cpass_t(const Dims& d, const cplx* Y, const cplx* a, cplx* G, double* r2, const int* skip,
                           cudaStream_t s) {
  int64_t grid = 8 * int64_t(kSMs);
  if (grid > d.nfib) grid = d.nfib;
  const int64_t per = (d.nfib + grid - 1) / grid;
  grid = (d.nfib + per - 1) / per;
  const size_t smem = size_t(d.I[0]) * RM * sizeof(cplx);
  cudaFuncSetAttribute(k_cpass<RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  k_cpass<RM><<<unsigned(grid), kCMaxI1, smem, s>>>(d, Y, a, G, r2, per, skip);
}

static void launch_cpass(const Dims& d, const cplx* Y, const cplx* a, cplx* G, double* r2, const int* skip,
                         cudaStream_t s) {
  if (d.R <= 4) launch_cpass_t<4>(d, Y, a, G, r2, skip, s);
  else if (d.R <= 8) launch_cpass_t<8>(d, Y, a, G, r2, skip, s);
  else launch_cpass_t<16>(d, Y, a, G, r2, skip, s);
}

}  // namespace cpdgn

using namespace cpdgn;

struct cp_cstate {
  Dims d;
  cp_opts o;
  cplx* a;
  CLayout L;
  CBufs B;
  int* tmo = nullptr;
};

extern "C" int cp_cstate_workspace_bytes(const cp_shape* shape, size_t* bytes) {
  Dims d;
  CP_TRY(cmake_dims(shape, &d));
  if (!bytes) return CP_EINVAL;
  CLayout L;
  c_layout(d, &L);
  *bytes = L.total;
  return CP_OK;
}

extern "C" int cp_cstate_create(const cp_shape* shape, const cp_opts* opts, double* a, void* ws, size_t ws_bytes,
                                cp_cstate** out) {
  if (!opts || !a || !ws || !out) return CP_EINVAL;
  Dims d;
  CP_TRY(cmake_dims(shape, &d));
  if (opts->max_iter < 0) return CP_EINVAL;
  CLayout L;
  c_layout(d, &L);
  if (ws_bytes < L.total) return CP_ENOMEM;
  cp_cstate* st = new (std::nothrow) cp_cstate;
  if (!st) return CP_ENOMEM;
  st->d = d;
  st->o = *opts;
  st->a = reinterpret_cast<cplx*>(a);
  st->L = L;
  st->B = c_carve(d, L, ws);
  if (tc_timeout_counter(&st->tmo) != CP_OK) {
    delete st;
    return CP_ECUDA;
  }
  *out = st;
  return CP_OK;
}

extern "C" int cp_cstate_destroy(cp_cstate* st) {
  delete st;
  return CP_OK;
}

extern "C" cp_status* cp_cstate_status(cp_cstate* st) { return st ? st->B.status : nullptr; }

extern "C" double* cp_cstate_buffer(cp_cstate* st, int id) {
  if (!st) return nullptr;
  switch (id) {
    case 0: return reinterpret_cast<double*>(st->B.G);
    case 1: return reinterpret_cast<double*>(st->B.delta);
    case 5: return reinterpret_cast<double*>(st->B.at);
    default: return nullptr;
  }
}

extern "C" int cp_cstate_init(cp_cstate* st, const void* Y, void* stream) {
  if (!st || !Y) return CP_EINVAL;
  const Dims& d = st->d;
  const CBufs& B = st->B;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cplx* Yc = static_cast<const cplx*>(Y);
  CP_CUDA(cudaMemsetAsync(B.G, 0, size_t(d.T) * d.R * sizeof(cplx), s));
  CP_CUDA(cudaMemsetAsync(B.scal, 0, 64 * sizeof(double), s));
  CP_CUDA(cudaMemsetAsync(B.info, 0, 64 * sizeof(int), s));
  launch_cpass(d, Yc, st->a, B.G, B.scal + CS_R2, nullptr, s);
  int64_t g = (d.J + 255) / 256;
  if (g > 4 * kSMs) g = 4 * kSMs;
  k_csumsq<<<unsigned(g), 256, 0, s>>>(Yc, d.J, B.scal + CS_YN2);
  k_cgram<<<unsigned((d.N * d.RR + 127) / 128), 128, 0, s>>>(d, st->a, nullptr, B.C, nullptr, nullptr);
  k_chad<<<unsigned((d.N * d.N * d.RR + 127) / 128), 128, 0, s>>>(d, B.C, B.Gnm, nullptr);
  k_cinit<<<1, 32, 0, s>>>(d, st->o, B.Gnm, B.scal, B.status, B.info, st->tmo);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" int cp_cdgn_step(cp_cstate* st, const void* Y, void* stream) {
  if (!st || !Y) return CP_EINVAL;
  const Dims& d = st->d;
  const CBufs& B = st->B;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cplx* Yc = static_cast<const cplx*>(Y);
  const int* skip = &B.status->stop;
  const double* mu = &B.status->mu;
  const int64_t n = d.ncore;
  const unsigned gn = unsigned((n + 127) / 128);
  k_cbegin<<<64, 256, 0, s>>>(d, B.scal, B.info, B.Gtr, B.status);
  k_cgram<<<unsigned((2 * d.N * d.RR + 127) / 128), 128, 0, s>>>(d, st->a, B.G, B.C, B.P, skip);
  k_chad<<<unsigned((d.N * d.N * d.RR + 127) / 128), 128, 0, s>>>(d, B.C, B.Gnm, skip);
  k_cprep<<<d.N, 32, 0, s>>>(d, B.C, B.Gnm, B.P, mu, B.U, B.LC, B.Gt, B.w, B.info + CI_INFO, skip);
  k_capplyK<<<gn, 128, 0, s>>>(d, B.Gnm, B.w, nullptr, B.Kw, skip);                     // K w
  k_capplySH<<<gn, 128, 0, s>>>(d, B.LC, B.U, B.Kw, B.b, B.b2, skip);                   // b = S^H K w
  int64_t gc = (n * n + 255) / 256;
  if (gc > 8 * kSMs) gc = 8 * kSMs;
  k_ccore_fill<<<unsigned(gc), 256, 0, s>>>(d, B.LC, B.U, B.Gnm, B.core2, skip);
  CP_TRY(chol64_factor(B.core2, 2 * n, B.dinv, B.info + CI_INFO, B.sync, st->tmo, skip, s));
  CP_TRY(chol64_solve(B.core2, B.dinv, 2 * n, B.b2, B.z2, B.y2, B.sync, B.info + CI_INFO, st->tmo, skip, s));
  k_capplyS<<<gn, 128, 0, s>>>(d, B.LC, B.U, B.y2, B.Z, skip);                          // S y
  k_capplyK<<<gn, 128, 0, s>>>(d, B.Gnm, B.Z, B.Kw, B.f, skip);                         // f = K w - K S y
  k_cupdate<<<unsigned((d.T + 127) / 128), 128, 0, s>>>(d, st->a, B.G, B.f, B.Gt, mu, B.delta, B.at, B.scal, skip);
  launch_cpass(d, Yc, B.at, B.Gtr, B.scal + CS_R2T, skip, s);
  k_ccontrol<<<1, 32, 0, s>>>(d, st->o, B.status, B.scal, B.info, B.scale, st->tmo);
  int64_t gm = (d.T * d.R + 255) / 256;
  if (gm > 4 * kSMs) gm = 4 * kSMs;
  k_ccommit<<<unsigned(gm), 256, 0, s>>>(d, B.info + CI_COMMIT, B.at, B.Gtr, B.scale, st->a, B.G);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
