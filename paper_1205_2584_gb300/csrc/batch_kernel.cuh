// Batched form: many small independent CP decompositions in ONE persistent
// launch.  Each CTA takes a problem from a device work queue (an atomic
// counter) and runs the damped Gauss-Newton iteration of Algorithm 1 with the
// Sec. 4.6 control on it until its stop rule fires (or a per-launch trial
// budget is spent), then takes the next problem.  Every phase is CTA-local,
// so there is no grid-wide synchronisation and the CTAs balance themselves.
//
// Per trial, inside one CTA (float32 tensor):
//   gram       C^(n) = A^(n)T A^(n), P^(n) = A^(n)T M_n      (float32, stored float64)
//   mode prep  Gamma^(n,m), chol(Gamma^(n) + mu I) and its inverse, Gt^(n),
//              U_n, chol(C^(n)), w                             (float64, one warp per mode)
//   core       W_nm, core = I + S^T K S (lower triangle)      (float32)
//   factor     blocked Cholesky of the core in global memory  (float32)
//   solve      y = core^{-1} S^T K w with float64 refinement of the residual
//              b - y - S^T K S y (matrix-free operator), f = K w - K S y
//   update     Delta A^(n) = (G_n - A^(n) F_n) Gt^(n)          (float32 products)
//   pass       MTTKRP and direct residual at the trial point  (float32, float64 sums)
//   control    gain ratio, accept iff the error decreased, Nielsen's mu, equal-
//              energy normalisation, stop test                (float64)
// The algebra is that of the single-problem path (SPD core, reading of w,
// Nielsen rule); only the placement differs.
#pragma once
#include "batch.cuh"
#include "small.cuh"

namespace cpdgn {

struct BCtx {
  int N, R, RR, n;
  int64_t I[BN], aoff[BN], T, J, nfib;
  const float* Y;
  double* a;
  double *M, *Mt, *At, *C, *P, *Gnm, *Gt, *U, *LC, *w, *Kw, *b, *y, *Z, *res, *f, *Wp, *delta;
  float* core;
  cp_status* st;
};

template <int TF>
struct BShared {
  // small float64 matrices of every mode
  double G[BN][BRR];
  double Linv[BN][BRR];
  double rinv[2 * BN][BR];
  double Cs[BN][BRR];
  double sc[BN * BR];              // column norms^2, then scales
  double red[BT];
  double scal[8];
  int flags[8];
  // MTTKRP tile and factor rows (float32)
  float A1[256 * BR];
  float Yt[2 * TF * 257];          // two alternating tiles of fibres (pitch I_1 | 1)
  float kr[TF * BR];
  float loo[(BN - 1) * TF * BR];
  float t[TF * BR];
  float Mn[3 * 256 * BR];          // partial M_n, n >= 2 (sum_{n>=2} I_n R <= 3 * 256 * 16)
  float blk[BNB * (BNB + 1)];      // Cholesky diagonal block / solve block
  float vec[1024];                 // right-hand side of the float32 solves
  int fix[(BN - 1) * TF];          // mode indices i_2.. of the tile's fibres
  float Af[3 * 256 * BR];          // factor rows of modes 2.. (float32), same layout as Mn
};

__device__ __forceinline__ void b_cp_async4(float* dst, const float* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void b_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void b_cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

static __device__ double bsum(double v, double* red) {
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = BT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Row i of a tile for rank RT: M_1 row i += sum_f y_f[i] kr_f, and the
// squared residual of y_f[i] against the model, fibre by fibre.  Four
// fibres at a time give independent chains; each sum keeps its fibre and
// column order.  RT is a template argument so that every loop is unrolled
// without guards and the loads can be issued ahead of their uses.
template <int RT>
__device__ __forceinline__ void b_rows_tile(const float* __restrict__ Yt, const float* __restrict__ kr,
                                            const float* __restrict__ a1, int ldy, int nf, int i,
                                            float (&acc)[BR], float& ee) {
  float arow[RT];
#pragma unroll
  for (int r = 0; r < RT; ++r) arow[r] = a1[r];
  int f = 0;
  for (; f + 4 <= nf; f += 4) {
    float yv[4], yh[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      yv[j] = Yt[(f + j) * ldy + i];
      yh[j] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < RT; ++r) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float k = kr[(f + j) * RT + r];
        acc[r] = fmaf(yv[j], k, acc[r]);
        yh[j] = fmaf(arow[r], k, yh[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float d = yv[j] - yh[j];
      ee = fmaf(d, d, ee);
    }
  }
  for (; f < nf; ++f) {
    const float yv = Yt[f * ldy + i];
    float yh = 0.f;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      const float k = kr[f * RT + r];
      acc[r] = fmaf(yv, k, acc[r]);
      yh = fmaf(arow[r], k, yh);
    }
    const float d = yv - yh;
    ee = fmaf(d, d, ee);
  }
}

// Column r of M_k (k >= 1): the tile's fibres in order, each adding
// t_f[r] * loo_f[r] to the row given by its mode-k index.  The running value
// stays in a register while consecutive fibres share a row.
__device__ __forceinline__ void b_mn_run(float* __restrict__ M, const int* __restrict__ fix,
                                         const float* __restrict__ t, const float* __restrict__ lo, int nf,
                                         int R) {
  int cur = fix[0];
  float v = M[cur * R];
#pragma unroll 4
  for (int f = 0; f < nf; ++f) {
    const int x = fix[f];
    const float tt = t[f * R], ll = lo[f * R];
    if (x != cur) {
      M[cur * R] = v;
      cur = x;
      v = M[cur * R];
    }
    v = fmaf(tt, ll, v);
  }
  M[cur * R] = v;
}

// ---------------------------------------------------------------------------
// pass over the tensor: M (if Mout) and ||Y - Y_hat||^2 at factors A
// ---------------------------------------------------------------------------
template <int TF>
__device__ double b_pass(const BCtx& c, BShared<TF>& sh, const double* A, double* Mout) {
  const int R = c.R, N = c.N, tid = threadIdx.x;
  const int I1 = int(c.I[0]);
  const int ldy = I1 | 1;
  for (int e = tid; e < I1 * R; e += BT) {
    const int i = e / R, r = e % R;
    sh.A1[i * R + r] = float(A[i + int64_t(r) * I1]);
  }
  int64_t moff[BN];
  int64_t mn = 0;
  for (int k = 1; k < N; ++k) { moff[k] = mn; mn += c.I[k] * R; }
  for (int64_t e = tid; e < mn; e += BT) sh.Mn[e] = 0.f;
  for (int k = 1; k < N; ++k) {                 // factor rows of modes 2.., row-major
    const int Ik = int(c.I[k]);
    for (int e = tid; e < Ik * R; e += BT) {
      const int i = e / R, r = e % R;
      sh.Af[moff[k] + e] = float(A[c.aoff[k] + i + int64_t(r) * Ik]);
    }
  }
  float acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.f;
  double e2 = 0.0;
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  // the tile's fibres go to one of two buffers by cp.async; the next tile's
  // copy is in flight while this tile is used
  auto load_tile = [&](int64_t f0, float* Yb) {
    const int nf = int((c.nfib - f0) < TF ? (c.nfib - f0) : TF);
    for (int f = warp; f < nf; f += BT / 32) {
      const float* src = c.Y + (f0 + f) * I1;
      for (int i = lane; i < I1; i += 32) b_cp_async4(&Yb[f * ldy + i], src + i);
    }
    b_cp_commit();
  };
  load_tile(0, sh.Yt);
  int buf = 0;
  for (int64_t f0 = 0; f0 < c.nfib; f0 += TF, buf ^= 1) {
    const int nf = int((c.nfib - f0) < TF ? (c.nfib - f0) : TF);
    const int yb = buf * (TF * 257);            // this tile's buffer
    // the tile's fibres: mode indices once per fibre (32-bit: nfib < 2^31 here)
    if (tid < nf) {
      int rem = int(f0) + tid;
#pragma unroll
      for (int k = 1; k < BN; ++k)
        if (k < N) {
          const int Ik = int(c.I[k]);
          const int q = rem / Ik;
          sh.fix[(k - 1) * TF + tid] = rem - q * Ik;
          rem = q;
        }
    }
    if (f0 + TF < c.nfib) load_tile(f0 + TF, sh.Yt + (buf ^ 1) * (TF * 257));
    else b_cp_commit();                         // empty group: the wait below is uniform
    b_cp_wait1();
    __syncthreads();
    for (int e = tid; e < nf * R; e += BT) {
      const int f = e / R, r = e % R;
      float v[BN];
#pragma unroll
      for (int k = 1; k < BN; ++k)
        if (k < N) v[k] = sh.Af[moff[k] + sh.fix[(k - 1) * TF + f] * R + r];
      float kr = 1.f;
#pragma unroll
      for (int k = 1; k < BN; ++k)
        if (k < N) kr *= v[k];
      sh.kr[f * R + r] = kr;
#pragma unroll
      for (int m = 1; m < BN; ++m)
        if (m < N) {
          float lo = 1.f;
#pragma unroll
          for (int k = 1; k < BN; ++k)
            if (k < N && k != m) lo *= v[k];
          sh.loo[((m - 1) * TF + f) * R + r] = lo;
        }
    }
    __syncthreads();
    // rows: M_1 and the residual
    for (int i = tid; i < I1; i += BT) {
      float ee = 0.f;
      const float* Yt = sh.Yt + yb;
      const float* a1 = sh.A1 + i * R;
      switch (R) {
#define CPDGN_ROWS(RT) \
  case RT: b_rows_tile<RT>(Yt, sh.kr, a1, ldy, nf, i, acc, ee); break;
        CPDGN_ROWS(1) CPDGN_ROWS(2) CPDGN_ROWS(3) CPDGN_ROWS(4) CPDGN_ROWS(5) CPDGN_ROWS(6)
        CPDGN_ROWS(7) CPDGN_ROWS(8) CPDGN_ROWS(9) CPDGN_ROWS(10) CPDGN_ROWS(11) CPDGN_ROWS(12)
        CPDGN_ROWS(13) CPDGN_ROWS(14) CPDGN_ROWS(15) CPDGN_ROWS(16)
#undef CPDGN_ROWS
        default: break;
      }
      e2 += double(ee);
    }
    // t_f = y_f^T A1 (a thread's two entries e, e + BT interleaved), then
    // the M_n, n >= 2, contributions
    if (Mout) {
      for (int e = tid; e < nf * R; e += 2 * BT) {
        const bool two = e + BT < nf * R;
        const int f = e / R, r = e % R;
        const int fb = two ? (e + BT) / R : f, rb = two ? (e + BT) % R : r;
        float s = 0.f, sb = 0.f;
#pragma unroll 8
        for (int i = 0; i < I1; ++i) {
          s = fmaf(sh.Yt[yb + f * ldy + i], sh.A1[i * R + r], s);
          sb = fmaf(sh.Yt[yb + fb * ldy + i], sh.A1[i * R + rb], sb);
        }
        sh.t[f * R + r] = s;
        if (two) sh.t[fb * R + rb] = sb;
      }
      __syncthreads();
      // M_k, k >= 1, in fibre order per (k, row, r).  When the tile's fibres
      // have distinct mode-1 indices (nf <= I_1), every M_1 row takes one
      // fibre and those updates run in parallel on warps 2..; the other
      // modes (all modes otherwise) run one thread per (k, r) on warps 0-1.
      const bool par1 = nf <= c.I[1];
      const int k0 = par1 ? 2 : 1;
      if (tid < (N - k0) * R) {
        const int k = k0 + tid / R, r = tid % R;
        b_mn_run(&sh.Mn[moff[k] + r], &sh.fix[(k - 1) * TF], sh.t + r, sh.loo + (k - 1) * TF * R + r, nf, R);
      }
      if (par1)
        for (int e = tid - 64; e >= 0 && e < nf * R; e += BT - 64) {
          const int f = e / R, r = e - f * R;
          float* dst = &sh.Mn[moff[1] + int64_t(sh.fix[f]) * R + r];
          *dst = fmaf(sh.t[f * R + r], sh.loo[f * R + r], *dst);
        }
    }
    __syncthreads();
  }
  if (Mout) {
    for (int i = tid; i < I1; i += BT)
      for (int r = 0; r < R; ++r) Mout[i + int64_t(r) * I1] = double(acc[r]);
    for (int k = 1; k < N; ++k) {
      const int Ik = int(c.I[k]);
      for (int e = tid; e < Ik * R; e += BT) {
        const int i = e % Ik, r = e / Ik;
        Mout[c.aoff[k] + i + int64_t(r) * Ik] = double(sh.Mn[moff[k] + int64_t(i) * R + r]);
      }
    }
  }
  return bsum(e2, sh.red);
}

// ---------------------------------------------------------------------------
// C^(n) and P^(n) (float32 products of float64 inputs, stored float64)
// ---------------------------------------------------------------------------
template <int TF>
__device__ void b_gram(const BCtx& c, BShared<TF>& sh, const double* A, const double* M) {
  const int R = c.R, RR = c.RR, N = c.N;
  for (int e = threadIdx.x; e < N * 2 * RR; e += BT) {
    const int n = e / (2 * RR), q = e % (2 * RR);
    const bool isP = q >= RR;
    const int rs = isP ? q - RR : q, r = rs % R, s2 = rs / R;
    if (!isP && r > s2) continue;
    const int64_t In = c.I[n];
    const double* x = A + c.aoff[n] + int64_t(r) * In;
    const double* y = (isP ? M : A) + c.aoff[n] + int64_t(s2) * In;
    float s0 = 0.f, s1 = 0.f;
    int64_t i = 0;
    for (; i + 1 < In; i += 2) {
      s0 = fmaf(float(x[i]), float(y[i]), s0);
      s1 = fmaf(float(x[i + 1]), float(y[i + 1]), s1);
    }
    if (i < In) s0 = fmaf(float(x[i]), float(y[i]), s0);
    const double v = double(s0) + double(s1);
    if (isP) {
      c.P[int64_t(n) * RR + rs] = v;
    } else {
      c.C[int64_t(n) * RR + r + R * s2] = v;
      c.C[int64_t(n) * RR + s2 + R * r] = v;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// per-mode float64 quantities: Gamma^(n,m), Gt, U, L_n, w
// ---------------------------------------------------------------------------
template <int TF>
__device__ bool b_mode_prep(const BCtx& c, BShared<TF>& sh, double mu) {
  const int R = c.R, RR = c.RR, N = c.N;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  for (int e = tid; e < N * N * RR; e += BT) {
    const int q = e % RR, nm = e / RR, n = nm / N, m = nm % N;
    double h = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != n && k != m) h *= c.C[int64_t(k) * RR + q];
    c.Gnm[e] = h;
  }
  __syncthreads();
  for (int e = tid; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR;
    sh.G[n][q] = c.Gnm[(int64_t(n) * N + n) * RR + q] + ((q % R) == (q / R) ? mu : 0.0);
    sh.Cs[n][q] = c.C[e];
  }
  if (tid == 0) sh.flags[0] = 1;
  __syncthreads();
  if (warp < N) {
    const bool ok = warp_chol(sh.G[warp], sh.rinv[warp], R);
    if (lane == 0 && !ok) sh.flags[0] = 0;
  } else if (warp < 2 * N) {
    const bool ok = warp_chol(sh.Cs[warp - N], sh.rinv[warp], R);
    if (lane == 0 && !ok) sh.flags[0] = 0;
  }
  __syncthreads();
  // Linv = L_G^{-1}: lane j of warp n solves L x = e_j (no synchronisation)
  if (warp < N && lane < R) {
    const double* L = sh.G[warp];
    const double* ri = sh.rinv[warp];
    double x[BR];
#pragma unroll
    for (int i = 0; i < BR; ++i) x[i] = 0.0;
#pragma unroll
    for (int i = 0; i < BR; ++i) {
      if (i < R) {
        double s = (i == lane) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < BR; ++k)
          if (k < i) s = fma(-L[i + R * k], x[k], s);
        x[i] = s * ri[i];
      }
    }
#pragma unroll
    for (int i = 0; i < BR; ++i)
      if (i < R) sh.Linv[warp][i + R * lane] = x[i];
  }
  __syncthreads();
  // U = Linv^T, Gt = U U^T = Linv^T Linv, L_n = chol(C^(n)) (lower)
  for (int e = tid; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR, i = q % R, j = q / R;
    const double* Li = sh.Linv[n];
    c.U[e] = Li[j + R * i];
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(Li[k + R * i], Li[k + R * j], s);
    c.Gt[e] = s;
    c.LC[e] = (i >= j) ? sh.Cs[n][q] : 0.0;
  }
  __syncthreads();
  // w_n = (P^(n) - C^(n) Gamma^(n)) Gt^(n): first V = P - C Gamma into sh.G
  for (int e = tid; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR, i = q % R, j = q / R;
    const double* Cn = c.C + int64_t(n) * RR;
    const double* Gm = c.Gnm + (int64_t(n) * N + n) * RR;
    double s = c.P[e];
    for (int k = 0; k < R; ++k) s = fma(-Cn[i + R * k], Gm[k + R * j], s);
    sh.G[n][q] = s;
  }
  __syncthreads();
  for (int e = tid; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR, i = q % R, j = q / R;
    const double* Gtn = c.Gt + int64_t(n) * RR;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(sh.G[n][i + R * k], Gtn[k + R * j], s);
    c.w[e] = s;
  }
  __syncthreads();
  return sh.flags[0] != 0;
}

__device__ __forceinline__ void bpair(int p, int* n, int* m) {
  int nn = 1;
  while ((nn * (nn + 1)) / 2 <= p) ++nn;
  *n = nn;
  *m = p - (nn * (nn - 1)) / 2;
}

// core = I + S^T K S, lower triangle, float32 (n x n, ld n)
template <int TF>
__device__ void b_core(const BCtx& c, BShared<TF>& sh) {
  const int R = c.R, RR = c.RR, N = c.N, n = c.n;
  const int npairs = N * (N - 1) / 2;
  const int R3 = RR * R;
  // Fast path: the float32 roundings the sums below take of float64 products
  // and values -- float(L_m[b,k] U_n[b,j]), float(Gamma^(n,m)), and for the
  // core blocks float(L_n[a,i] U_m[a,l]) -- are formed once per block pair in
  // the pass buffers (Af, Mn: unused here) instead of once per term (each a
  // float64 multiply and conversions on this part's slow float64 pipe), and
  // W stays in shared memory.  Same values, same order: results are those of
  // the per-term form below, which remains for shapes whose tables do not fit.
  const bool fast = 2 * npairs * R3 <= int(sizeof(sh.Af) / sizeof(float)) &&
                    npairs * (R3 + RR) <= int(sizeof(sh.Mn) / sizeof(float));
  if (fast) {
    float* P = sh.Af;                         // P[p][a][i][l] = float(L_n[a,i] U_m[a,l])
    float* W = sh.Af + npairs * R3;           // W[p][a + R (k + R j)]
    float* Q = sh.Mn;                         // Q[p][b][k][j] = float(L_m[b,k] U_n[b,j])
    float* Gf = sh.Mn + npairs * R3;          // Gf[p][a + R b] = float(Gamma^(n,m)[a,b])
    for (int e = threadIdx.x; e < npairs * R3; e += BT) {
      const int p = e / R3, q = e % R3, x = q / RR, y = (q / R) % R, z = q % R;
      int nn, m;
      bpair(p, &nn, &m);
      // P: (a, i, l) = (x, y, z); Q: (b, k, j) = (x, y, z)
      P[e] = float(c.LC[int64_t(nn) * RR + x + R * y] * c.U[int64_t(m) * RR + x + R * z]);
      Q[e] = float(c.LC[int64_t(m) * RR + x + R * y] * c.U[int64_t(nn) * RR + x + R * z]);
    }
    for (int e = threadIdx.x; e < npairs * RR; e += BT) {
      const int p = e / RR, q = e % RR;
      int nn, m;
      bpair(p, &nn, &m);
      Gf[e] = float(c.Gnm[(int64_t(nn) * N + m) * RR + q]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npairs * R3; e += BT) {
      const int p = e / R3, q = e % R3, aa = q % R, k = (q / R) % R, j = q / RR;
      const float* Qp = Q + p * R3;
      const float* Gp = Gf + p * RR;
      float s = 0.f;
      for (int bb = k; bb <= j; ++bb) s = fmaf(Gp[aa + R * bb], Qp[bb * RR + k * R + j], s);
      W[e] = s;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < int64_t(npairs) * RR * RR; e += BT) {
      const int p = int(e / (int64_t(RR) * RR));
      const int q = int(e % (int64_t(RR) * RR));
      const int rho = q % RR, kap = q / RR;
      int nn, m;
      bpair(p, &nn, &m);
      const int i = rho % R, j = rho / R, k = kap % R, l = kap / R;
      const float* Pp = P + p * R3;
      const float* Wq = W + p * R3;
      float s = 0.f;
      for (int aa = i; aa <= l; ++aa) s = fmaf(Pp[aa * RR + i * R + l], Wq[aa + R * (k + R * j)], s);
      c.core[(int64_t(nn) * RR + rho) + int64_t(n) * (int64_t(m) * RR + kap)] = s;
    }
  } else {
    for (int e = threadIdx.x; e < npairs * R3; e += BT) {
      const int p = e / R3, q = e % R3, aa = q % R, k = (q / R) % R, j = q / RR;
      int nn, m;
      bpair(p, &nn, &m);
      const double* G = c.Gnm + (int64_t(nn) * N + m) * RR;
      const double* Lm = c.LC + int64_t(m) * RR;
      const double* Un = c.U + int64_t(nn) * RR;
      float s = 0.f;
      for (int bb = k; bb <= j; ++bb) s = fmaf(float(G[aa + R * bb]), float(Lm[bb + R * k] * Un[bb + R * j]), s);
      c.Wp[e] = s;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < int64_t(npairs) * RR * RR; e += BT) {
      const int p = int(e / (int64_t(RR) * RR));
      const int q = int(e % (int64_t(RR) * RR));
      const int rho = q % RR, kap = q / RR;
      int nn, m;
      bpair(p, &nn, &m);
      const int i = rho % R, j = rho / R, k = kap % R, l = kap / R;
      const double* Ln = c.LC + int64_t(nn) * RR;
      const double* Um = c.U + int64_t(m) * RR;
      const double* W = c.Wp + int64_t(p) * R3;
      float s = 0.f;
      for (int aa = i; aa <= l; ++aa) s = fmaf(float(Ln[aa + R * i] * Um[aa + R * l]), float(W[aa + R * (k + R * j)]), s);
      c.core[(int64_t(nn) * RR + rho) + int64_t(n) * (int64_t(m) * RR + kap)] = s;
    }
  }
  for (int64_t e = threadIdx.x; e < int64_t(N) * RR * RR; e += BT) {
    const int nn = int(e / (int64_t(RR) * RR));
    const int q = int(e % (int64_t(RR) * RR));
    const int rho = q % RR, kap = q / RR;
    if (rho >= kap) c.core[(int64_t(nn) * RR + rho) + int64_t(n) * (int64_t(nn) * RR + kap)] = (rho == kap) ? 1.f : 0.f;
  }
  __syncthreads();
}

// In-CTA blocked right-looking Cholesky of the float32 core (lower, in global
// memory).  Returns false on a non-positive or non-finite pivot.  The solved
// panel of each block step (rows below the diagonal block) is also kept in
// shared memory -- in the pass buffers Af and Mn, unused during the
// factorisation -- so the trailing update reads its operands there instead
// of from global memory; rows beyond that space (cores above about 770) keep
// reading global memory.
// Panel rows are BNB + 1 floats apart: the threads of a warp read rows two
// apart at the same k, and a pitch of 33 puts them in different banks.
constexpr int kPanPitch = BNB + 1;
template <int TF>
__device__ __forceinline__ float* b_panel_row(BShared<TF>& sh, int r) {
  constexpr int cap = int(sizeof(sh.Af) / sizeof(float)) / kPanPitch;
  return r < cap ? sh.Af + r * kPanPitch : sh.Mn + (r - cap) * kPanPitch;
}
template <int TF>
__device__ bool b_chol(const BCtx& c, BShared<TF>& sh) {
  const int n = c.n, tid = threadIdx.x;
  float* A = c.core;
  constexpr int L = BNB + 1;
  constexpr int kPanRows = int(sizeof(sh.Af) / sizeof(float)) / kPanPitch +
                           int(sizeof(sh.Mn) / sizeof(float)) / kPanPitch;
  if (tid == 0) sh.flags[1] = 1;
  for (int k0 = 0; k0 < n; k0 += BNB) {
    const int kb = (n - k0) < BNB ? (n - k0) : BNB;
    __syncthreads();
    for (int e = tid; e < kb * kb; e += BT) {
      const int i = e % kb, j = e / kb;
      sh.blk[i + L * j] = A[(k0 + i) + int64_t(n) * (k0 + j)];
    }
    __syncthreads();
    for (int p = 0; p < kb; ++p) {        // right-looking factor of the diagonal block
      const float piv = sh.blk[p + L * p];
      if (tid == 0 && !(piv > 0.f && isfinite(piv))) sh.flags[1] = 0;
      const float dp = sqrtf(piv);
      const float ip = 1.f / dp;
      __syncthreads();
      if (tid == 0) sh.blk[p + L * p] = dp;
      if (tid > p && tid < kb) sh.blk[tid + L * p] *= ip;
      __syncthreads();
      const int m = kb - p - 1;
      for (int e = tid; e < m * m; e += BT) {
        const int i = p + 1 + e % m, j = p + 1 + e / m;
        if (j <= i) sh.blk[i + L * j] = fmaf(-sh.blk[i + L * p], sh.blk[j + L * p], sh.blk[i + L * j]);
      }
      __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += BT) {
      const int i = e % kb, j = e / kb;
      if (i >= j) A[(k0 + i) + int64_t(n) * (k0 + j)] = sh.blk[i + L * j];
    }
    // panel: rows below, X <- X L_kk^{-T}, one row per thread
    for (int r = k0 + kb + tid; r < n; r += BT) {
      float x[BNB];
#pragma unroll
      for (int j = 0; j < BNB; ++j) x[j] = (j < kb) ? A[r + int64_t(n) * (k0 + j)] : 0.f;
#pragma unroll
      for (int j = 0; j < BNB; ++j) {
        if (j < kb) {
          float s = x[j];
#pragma unroll
          for (int q = 0; q < BNB; ++q)
            if (q < j) s = fmaf(-x[q], sh.blk[j + L * q], s);
          x[j] = s / sh.blk[j + L * j];
        }
      }
#pragma unroll
      for (int j = 0; j < BNB; ++j)
        if (j < kb) A[r + int64_t(n) * (k0 + j)] = x[j];
      const int pr = r - (k0 + kb);
      if (pr < kPanRows) {
        float* dst = b_panel_row(sh, pr);
#pragma unroll
        for (int j = 0; j < BNB; ++j) dst[j] = (j < kb) ? x[j] : 0.f;
      }
    }
    __syncthreads();
    // trailing update of the lower triangle, 2 x 2 blocks per thread, the
    // panel read from shared memory (global memory past kPanRows rows)
    const int m0 = k0 + kb, rest = n - m0;
    const int nb2 = (rest + 1) / 2;
    for (int64_t e = tid; e < int64_t(nb2) * nb2; e += BT) {
      const int bi = int(e % nb2), bj = int(e / nb2);
      if (bj > bi) continue;
      const int i0 = m0 + 2 * bi, j0 = m0 + 2 * bj;
      float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
      const bool i1ok = i0 + 1 < n, j1ok = j0 + 1 < n;
      if (i0 + 1 - m0 < kPanRows) {      // i0 >= j0, so every row needed is staged
        const float* pa0 = b_panel_row(sh, i0 - m0);
        const float* pa1 = b_panel_row(sh, i0 + 1 - m0);
        const float* pb0 = b_panel_row(sh, j0 - m0);
        const float* pb1 = b_panel_row(sh, j0 + 1 - m0);
        for (int q = 0; q < kb; ++q) {
          const float a0 = pa0[q], a1 = i1ok ? pa1[q] : 0.f;
          const float b0 = pb0[q], b1 = j1ok ? pb1[q] : 0.f;
          c00 = fmaf(a0, b0, c00);
          c01 = fmaf(a0, b1, c01);
          c10 = fmaf(a1, b0, c10);
          c11 = fmaf(a1, b1, c11);
        }
      } else {
        for (int q = 0; q < kb; ++q) {
          const float* col = A + int64_t(n) * (k0 + q);
          const float a0 = col[i0], a1 = i1ok ? col[i0 + 1] : 0.f;
          const float b0 = col[j0], b1 = j1ok ? col[j0 + 1] : 0.f;
          c00 = fmaf(a0, b0, c00);
          c01 = fmaf(a0, b1, c01);
          c10 = fmaf(a1, b0, c10);
          c11 = fmaf(a1, b1, c11);
        }
      }
      A[i0 + int64_t(n) * j0] -= c00;
      if (j1ok && j0 + 1 <= i0) A[i0 + int64_t(n) * (j0 + 1)] -= c01;
      if (i1ok) A[(i0 + 1) + int64_t(n) * j0] -= c10;
      if (i1ok && j1ok) A[(i0 + 1) + int64_t(n) * (j0 + 1)] -= c11;
    }
  }
  __syncthreads();
  return sh.flags[1] != 0;
}

// v <- (L L^T)^{-1} v with the float32 factor, v in sh.vec (length n <= 1024)
template <int TF>
__device__ void b_tri_solve(const BCtx& c, BShared<TF>& sh) {
  // core = L L^T (float32, lower triangle in c.core): v <- L^{-T} L^{-1} v.
  // Each 32 x 32 diagonal block is staged in shared memory; one warp walks
  // it with the solution entries in registers (lane t holds entry k0 + t),
  // then all threads apply the block to the remaining rows.
  const int n = c.n, tid = threadIdx.x;
  const float* A = c.core;
  float* v = sh.vec;
  constexpr int L = BNB + 1;
  for (int k0 = 0; k0 < n; k0 += BNB) {          // forward: L z = v
    const int kb = (n - k0) < BNB ? (n - k0) : BNB;
    __syncthreads();
    for (int e = tid; e < kb * kb; e += BT) {
      const int i = e % kb, j = e / kb;
      if (i >= j) sh.blk[i + L * j] = A[(k0 + i) + int64_t(n) * (k0 + j)];
    }
    __syncthreads();
    if (tid < 32) {
      float vi = (tid < kb) ? v[k0 + tid] : 0.f;
      for (int p = 0; p < kb; ++p) {
        const float zp = __shfl_sync(0xffffffffu, vi, p) / sh.blk[p + L * p];
        if (tid == p) vi = zp;
        else if (tid > p && tid < kb) vi = fmaf(-sh.blk[tid + L * p], zp, vi);
      }
      if (tid < kb) v[k0 + tid] = vi;
    }
    __syncthreads();
    for (int r = k0 + kb + tid; r < n; r += BT) {
      float s = v[r];
      for (int q = 0; q < kb; ++q) s = fmaf(-A[r + int64_t(n) * (k0 + q)], v[k0 + q], s);
      v[r] = s;
    }
  }
  const int last = ((n - 1) / BNB) * BNB;
  for (int k0 = last; k0 >= 0; k0 -= BNB) {     // backward: L^T y = z
    const int kb = (n - k0) < BNB ? (n - k0) : BNB;
    __syncthreads();
    for (int e = tid; e < kb * kb; e += BT) {
      const int i = e % kb, j = e / kb;
      if (i >= j) sh.blk[i + L * j] = A[(k0 + i) + int64_t(n) * (k0 + j)];
    }
    __syncthreads();
    if (tid < 32) {
      float vi = (tid < kb) ? v[k0 + tid] : 0.f;
      for (int p = kb - 1; p >= 0; --p) {
        const float yp = __shfl_sync(0xffffffffu, vi, p) / sh.blk[p + L * p];
        if (tid == p) vi = yp;
        else if (tid < p) vi = fmaf(-sh.blk[p + L * tid], yp, vi);
      }
      if (tid < kb) v[k0 + tid] = vi;
    }
    __syncthreads();
    for (int r = tid; r < k0; r += BT) {
      float s = v[r];
      for (int q = 0; q < kb; ++q) s = fmaf(-A[(k0 + q) + int64_t(n) * r], v[k0 + q], s);
      v[r] = s;
    }
  }
  __syncthreads();
}

// out_n = S_n^T V_n with V = (K x) (kx) or x; then out = base - y - out if base.
// Also returns ||out||^2.  Float64, all N R^2 entries spread over the CTA.
template <int TF>
__device__ double b_apply_STK(const BCtx& c, BShared<TF>& sh, const double* x, int kx, const double* base,
                              const double* yv, double* out, double* kw) {
  const int R = c.R, RR = c.RR, N = c.N;
  // V into Z (scratch), V_n[i + R j] = sum_{m != n} Gamma^(n,m)[i,j] X_m[j,i]
  for (int e = threadIdx.x; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR, i = q % R, j = q / R;
    double s;
    if (kx) {
      s = 0.0;
      for (int m = 0; m < N; ++m)
        if (m != n) s = fma(c.Gnm[(int64_t(n) * N + m) * RR + q], x[int64_t(m) * RR + j + R * i], s);
    } else {
      s = x[e];
    }
    c.Z[e] = s;
    if (kw) kw[e] = s;
  }
  __syncthreads();
  // T = V U_n  (into res scratch if base==null else into sh.Linv as scratch)
  for (int e = threadIdx.x; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR, i = q % R, j = q / R;
    const double* V = c.Z + int64_t(n) * RR;
    const double* Un = c.U + int64_t(n) * RR;
    double s = 0.0;
    for (int l = 0; l <= j; ++l) s = fma(V[i + R * l], Un[l + R * j], s);
    sh.Linv[n][q] = s;
  }
  __syncthreads();
  double nrm = 0.0;
  for (int e = threadIdx.x; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR, p = q % R, j = q / R;
    const double* Ln = c.LC + int64_t(n) * RR;
    double s = 0.0;
    for (int k = p; k < R; ++k) s = fma(Ln[k + R * p], sh.Linv[n][k + R * j], s);
    const double v = base ? base[e] - yv[e] - s : s;
    out[e] = v;
    nrm = fma(v, v, nrm);
  }
  return bsum(nrm, sh.red);
}

// out_m = S_m x_m = vec(L_m X_m U_m^T)
template <int TF>
__device__ void b_apply_S(const BCtx& c, BShared<TF>& sh, const double* x, double* out) {
  const int R = c.R, RR = c.RR, N = c.N;
  for (int e = threadIdx.x; e < N * RR; e += BT) {       // T = X U^T
    const int m = e / RR, q = e % RR, i = q % R, j = q / R;
    const double* X = x + int64_t(m) * RR;
    const double* Um = c.U + int64_t(m) * RR;
    double s = 0.0;
    for (int l = j; l < R; ++l) s = fma(X[i + R * l], Um[j + R * l], s);
    sh.Linv[m][q] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * RR; e += BT) {       // out = L T
    const int m = e / RR, q = e % RR, p = q % R, j = q / R;
    const double* Lm = c.LC + int64_t(m) * RR;
    double s = 0.0;
    for (int k = 0; k <= p; ++k) s = fma(Lm[p + R * k], sh.Linv[m][k + R * j], s);
    out[e] = s;
  }
  __syncthreads();
}

// f = K w - K S core^{-1} S^T K w with refine_iters float64 refinement sweeps
template <int TF>
__device__ double b_solve(const BCtx& c, BShared<TF>& sh, int refine_iters) {
  const int n = c.n, tid = threadIdx.x;
  const double b2 = b_apply_STK(c, sh, c.w, 1, nullptr, nullptr, c.b, c.Kw);
  for (int e = tid; e < n; e += BT) sh.vec[e] = float(c.b[e]);
  b_tri_solve(c, sh);
  for (int e = tid; e < n; e += BT) c.y[e] = double(sh.vec[e]);
  __syncthreads();
  double rel = 0.0, prev = 0.0;
  for (int it = 0; it < refine_iters; ++it) {
    b_apply_S(c, sh, c.y, c.res);
    const double r2 = b_apply_STK(c, sh, c.res, 1, c.b, c.y, c.res, nullptr);
    rel = (b2 > 0.0) ? sqrt(r2 / b2) : 0.0;
    if (r2 <= 1e-30 * b2 || (prev > 0.0 && r2 > 0.0625 * prev)) break;
    prev = r2;
    for (int e = tid; e < n; e += BT) sh.vec[e] = float(c.res[e]);
    b_tri_solve(c, sh);
    for (int e = tid; e < n; e += BT) c.y[e] += double(sh.vec[e]);
    __syncthreads();
  }
  // f = Kw - K (S y)
  b_apply_S(c, sh, c.y, c.res);
  const int R = c.R, RR = c.RR, N = c.N;
  for (int e = tid; e < N * RR; e += BT) {
    const int nn = e / RR, q = e % RR, i = q % R, j = q / R;
    double s = 0.0;
    for (int m = 0; m < N; ++m)
      if (m != nn) s = fma(c.Gnm[(int64_t(nn) * N + m) * RR + q], c.res[int64_t(m) * RR + j + R * i], s);
    c.f[e] = c.Kw[e] - s;
  }
  __syncthreads();
  return rel;
}

// Delta A = (G - A F) Gt with G = M - A Gamma; trial factors; returns the
// gain-ratio denominator sum Delta (G + mu Delta); column norms^2 into sh.sc.
template <int TF>
__device__ double b_update(const BCtx& c, BShared<TF>& sh, double mu) {
  const int R = c.R, RR = c.RR, N = c.N;
  // Gamma^(n) + F_n and Gamma^(n) rounded to float32 once per mode, in the
  // pass buffer Mn (unused between passes); float64 -> float32 conversions
  // run on this part's slow float64 pipe, so none is repeated per row
  float* gf = sh.Mn;
  float* gg = sh.Mn + N * RR;
  for (int e = threadIdx.x; e < N * RR; e += BT) {
    const int n = e / RR, q = e % RR;
    const double gm = c.Gnm[(int64_t(n) * N + n) * RR + q];
    gf[e] = float(gm + c.f[int64_t(n) * RR + q]);
    gg[e] = float(gm);
  }
  __syncthreads();
  double den = 0.0;
  // The gain-ratio denominator sum_e Delta_e (g_e + mu Delta_e) is added in
  // the entry order e = tid, tid + BT, ... (then the fixed tree of bsum), so
  // that it does not depend on how entries are assigned to threads below:
  // the factors' trajectory, and so each problem's trial count, stays that of
  // the entry-per-thread form.  q_e = g_e + mu Delta_e waits in the pass
  // buffer Af when the T R entries fit.
  double* qs = reinterpret_cast<double*>(sh.Af);
  const bool replay = c.T * R <= int64_t(sizeof(sh.Af) / sizeof(double));
  // one factor row (mode n, index i) per thread: h[s] = (M - A Gamma - A F)[i, s]
  // and g[s] = (M - A Gamma)[i, s] once, then Delta[i, r] = h Gt[:, r]
  for (int64_t row = threadIdx.x; row < c.T; row += BT) {
    int n = 0;
    while (n + 1 < N && row >= c.aoff[n + 1] / R) ++n;
    const int64_t In = c.I[n];
    const int i = int(row - c.aoff[n] / R);
    const double* An = c.a + c.aoff[n];
    const double* Mn = c.M + c.aoff[n];
    const double* Gtn = c.Gt + int64_t(n) * RR;
    const float* gfn = gf + n * RR;
    const float* ggn = gg + n * RR;
    float ar[BR];
#pragma unroll
    for (int k = 0; k < BR; ++k) ar[k] = (k < R) ? float(An[i + In * k]) : 0.f;
    double h[BR], g[BR];
#pragma unroll
    for (int s2 = 0; s2 < BR; ++s2) {
      if (s2 < R) {
        float t1 = 0.f, t2 = 0.f;
        for (int k = 0; k < R; ++k) {
          t1 = fmaf(ar[k], gfn[k + R * s2], t1);
          t2 = fmaf(ar[k], ggn[k + R * s2], t2);
        }
        const double Ms = Mn[i + In * s2];
        h[s2] = Ms - double(t1);
        g[s2] = Ms - double(t2);
      }
    }
    for (int r = 0; r < R; ++r) {
      double dl = 0.0;
#pragma unroll
      for (int s2 = 0; s2 < BR; ++s2)
        if (s2 < R) dl = fma(h[s2], Gtn[s2 + R * r], dl);
      double gr = 0.0;
#pragma unroll
      for (int s2 = 0; s2 < BR; ++s2)
        if (s2 == r) gr = g[s2];
      const int64_t e = c.aoff[n] + i + In * r;
      if (replay) qs[e] = gr + mu * dl;
      else den = fma(dl, gr + mu * dl, den);
      c.delta[e] = dl;
      c.At[e] = An[i + In * r] + dl;
    }
  }
  if (replay) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < c.T * R; e += BT) den = fma(c.delta[e], qs[e], den);
  }
  const double dsum = bsum(den, sh.red);   // (ends with a barrier: At is complete)
  for (int e = threadIdx.x; e < N * R; e += BT) {   // column norms^2 in row order
    const int n = e / R, r = e % R;
    const double* col = c.At + c.aoff[n] + c.I[n] * r;
    double s = 0.0;
    for (int64_t i = 0; i < c.I[n]; ++i) s = fma(col[i], col[i], s);
    sh.sc[e] = s;
  }
  __syncthreads();
  return dsum;
}

template <int TF>
__global__ void __launch_bounds__(BT) k_batch_lm(const cp_batch_problem* probs, int count, const float* Y,
                                                 double* a, unsigned char* ws, cp_status* status, cp_opts o,
                                                 int trials, int* queue, const int* order) {
  extern __shared__ __align__(16) unsigned char bsmem[];
  BShared<TF>& sh = *reinterpret_cast<BShared<TF>*>(bsmem);
  __shared__ int s_p;
  for (;;) {
    if (threadIdx.x == 0) {
      const int q = atomicAdd(queue, 1);
      s_p = (q < count && order) ? order[q] : q;
    }
    __syncthreads();
    const int p = s_p;
    __syncthreads();
    if (p >= count) return;
    const cp_batch_problem pd = probs[p];
    BCtx c;
    c.N = pd.N;
    c.R = pd.R;
    c.RR = pd.R * pd.R;
    c.n = pd.N * c.RR;
    c.T = 0;
    c.J = 1;
    for (int k = 0; k < BN; ++k) c.I[k] = (k < pd.N) ? pd.I[k] : 1;
    for (int k = 0; k < pd.N; ++k) {
      c.aoff[k] = c.T * pd.R;
      c.T += pd.I[k];
      c.J *= pd.I[k];
    }
    c.nfib = c.J / c.I[0];
    c.Y = Y + pd.y_off;
    c.a = a + pd.a_off;
    double* base = reinterpret_cast<double*>(ws + pd.ws_off);
    const int64_t RT = c.T * c.R;
    const int64_t NRR = int64_t(c.N) * c.RR;
    c.M = base;
    c.Mt = c.M + RT;
    c.At = c.Mt + RT;
    c.delta = c.At + RT;
    c.C = c.delta + RT;
    c.P = c.C + NRR;
    c.Gt = c.P + NRR;
    c.U = c.Gt + NRR;
    c.LC = c.U + NRR;
    c.Gnm = c.LC + NRR;
    c.w = c.Gnm + int64_t(c.N) * NRR;
    c.Kw = c.w + c.n;
    c.b = c.Kw + c.n;
    c.y = c.b + c.n;
    c.Z = c.y + c.n;
    c.res = c.Z + c.n;
    c.f = c.res + c.n;
    c.Wp = c.f + c.n;
    c.core = reinterpret_cast<float*>(c.Wp + int64_t(c.N) * (c.N - 1) / 2 * c.RR * c.R);
    cp_status* st = status + p;
    c.st = st;
    if (st->stop != CP_RUNNING) continue;
    // start: one pass at the initial factors, ||Y||^2, mu_0
    if (st->iters == 0 && st->y_norm2 == 0.0) {
      const double r2 = b_pass(c, sh, c.a, c.M);
      double yn = 0.0;
      for (int64_t e = threadIdx.x; e < c.J; e += BT) {
        const double v = c.Y[e];
        yn = fma(v, v, yn);
      }
      yn = bsum(yn, sh.red);
      b_gram(c, sh, c.a, c.M);
      if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int n = 0; n < c.N; ++n) {
          for (int r = 0; r < c.R; ++r) {
            double g = 1.0;
            for (int k = 0; k < c.N; ++k)
              if (k != n) g *= c.C[int64_t(k) * c.RR + r + c.R * r];
            mx = g > mx ? g : mx;
          }
        }
        st->mu = (pd.mu0 > 0.0) ? pd.mu0 : o.tau * mx;
        st->nu = 2.0;
        st->resid2 = r2;
        st->resid2_trial = r2;
        st->y_norm2 = yn;
        st->rel_err = sqrt(r2 / yn);
        st->accepted = 0;
        st->last_accepted = 0;
        st->info = 0;
        // NaN / Inf in the tensor or the factors, or an all-zero tensor: stop
        if (!isfinite(yn) || !isfinite(r2) || !isfinite(st->mu) || !(yn > 0.0)) {
          st->error = (isfinite(yn) && isfinite(r2) && isfinite(st->mu)) ? CP_EINVAL : CP_ENONFINITE;
          st->stop = CP_STOP_ERROR;
        }
      }
      __syncthreads();
    }
    for (int t = 0; t < trials; ++t) {
      __syncthreads();
      if (st->stop != CP_RUNNING) break;
      const double mu = st->mu;
      b_gram(c, sh, c.a, c.M);
      bool ok = b_mode_prep(c, sh, mu);
      b_core(c, sh);
      ok = b_chol(c, sh) && ok;
      const double rel = b_solve(c, sh, o.refine_iters);
      const double den = b_update(c, sh, mu);
      __syncthreads();
      const double r2t = b_pass(c, sh, c.At, c.Mt);
      // control
      if (threadIdx.x == 0) {
        const double r2 = st->resid2;
        const bool finite = isfinite(r2t) && isfinite(den);
        const bool accept = ok && finite && (r2t < r2);
        // a failed factorisation or a non-finite trial is rejected as rho = 0
        // (mu grows), as in the single-problem control
        const double rho = (ok && finite && den > 0.0) ? (r2 - r2t) / den : 0.0;
        if (ok && !finite && st->error == 0) st->error = CP_ENONFINITE;
        double m2 = st->mu, nu = st->nu;
        if (rho > 0.0) {
          const double tt = 2.0 * rho - 1.0;
          const double fac = 1.0 - tt * tt * tt;
          m2 *= (fac > 1.0 / 3.0) ? fac : 1.0 / 3.0;
          nu = 2.0;
        } else {
          m2 *= nu;
          nu *= 2.0;
        }
        st->iters += 1;
        st->rho = rho;
        st->denom = den;
        st->resid2_trial = r2t;
        st->refine_resid = rel;
        st->info = ok ? 0 : 1;
        st->mu = m2;
        st->nu = nu;
        st->last_accepted = accept ? 1 : 0;
        if (accept) {
          const double e_old = sqrt(r2 / st->y_norm2), e_new = sqrt(r2t / st->y_norm2);
          st->accepted += 1;
          st->resid2 = r2t;
          st->rel_err = e_new;
          if (e_old > 0.0 && fabs(e_old - e_new) / e_old < o.tol) st->stop = CP_STOP_TOL;
        }
        if (st->stop == CP_RUNNING && m2 > o.mu_max) st->stop = CP_STOP_MU;
        if (st->stop == CP_RUNNING && st->iters >= o.max_iter) st->stop = CP_STOP_MAXIT;
        sh.flags[2] = accept ? 1 : 0;
      }
      __syncthreads();
      if (sh.flags[2]) {
        // equal-energy scales, then commit A and rescale M
        if (threadIdx.x < c.R) {
          const int r = threadIdx.x;
          bool okn = o.normalize != 0;
          double lam = 1.0;
          for (int n = 0; n < c.N; ++n) {
            const double nr = sqrt(sh.sc[n * c.R + r]);
            if (!(nr > 0.0)) okn = false;
            lam *= nr;
          }
          const double tgt = okn ? pow(lam, 1.0 / c.N) : 1.0;
          for (int n = 0; n < c.N; ++n) sh.sc[n * c.R + r] = okn ? tgt / sqrt(sh.sc[n * c.R + r]) : 1.0;
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < RT; e += BT) {
          int n = 0;
          while (n + 1 < c.N && e >= c.aoff[n + 1]) ++n;
          const int r = int((e - c.aoff[n]) / c.I[n]);
          const double s = sh.sc[n * c.R + r];
          c.a[e] = c.At[e] * s;
          c.M[e] = c.Mt[e] / s;
        }
      }
      __syncthreads();
    }
  }
}

template <int TF>
int batch_launch(const cp_batch_problem* probs_dev, int count, const float* Y, double* a, void* ws,
                 cp_status* status, const cp_opts* opts, int trials, int grid, const int* order,
                 cudaStream_t s) {
  const size_t smem = sizeof(BShared<TF>);
  if (cudaFuncSetAttribute(k_batch_lm<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return CP_ECUDA;
  k_batch_lm<TF><<<grid, BT, smem, s>>>(probs_dev, count, Y, a, static_cast<unsigned char*>(ws), status, *opts,
                                        trials, static_cast<int*>(ws), order);
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace cpdgn
