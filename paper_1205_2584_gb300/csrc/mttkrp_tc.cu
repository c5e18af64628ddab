// All-mode MTTKRP and direct residual of a 3-way float32 tensor on the
// 5th-generation tensor cores (tcgen05), one pass over the tensor.
//
// With Y(i1, f), f = (i2, i3) a fibre, and W(f, r) = A2(i2, r) A3(i3, r)
// (a Khatri-Rao row), the pass computes (Sec. 4, Eq. for the gradient blocks
// G_n = M_n - A^(n) Gamma^(n); the direct residual ||Y - Yhat||^2 of Sec. 4.6):
//   M1(i1, r) = sum_f Y(i1, f) W(f, r)                     (tensor cores)
//   V(f, r)   = sum_i1 Y(i1, f) A1(i1, r)                  (tensor cores)
//   M2(i2, r) = sum_i3 V(f, r) A3(i3, r),  M3(i3, r) = sum_i2 V(f, r) A2(i2, r)
//                                                          (dimension tree: V is
//                                                           shared by modes 2, 3)
//   Yhat(i1, f) = sum_r A1(i1, r) W(f, r)                  (tensor cores)
//   resid2 += sum (Y - Yhat)^2                             (exact float32 Y)
//
// Precision: the tensor cores take bf16 operands with f32 accumulation.
// Float64 factors and the f32 Khatri-Rao rows are split into three bf16
// pieces (x = x0 + x1 + x2, 24 significant bits); the tensor is split into two
// (y = y0 + y1, 16 significant bits, a fixed rounding of the data).  Products
// keep every term down to 2^-16 relative (5 piece pairs for Y W and Y A1, 6
// for A1 W), so the factor-dependent rounding is ~2^-22, below float32
// accumulation error.  The residual uses the exact float32 tensor.
//
// Work split: one CTA per (128-row chunk of i1, 128-row block of i2, segment
// of i3); per i3 step the CTA streams a 128 x 128 tile of Y as four 32 x 128
// float32 TMA boxes (128-byte swizzle) through a four-slot ring.  Warps:
//   4: TMA producer (full / empty mbarriers per slot);
//   5: MMA issuer, one thread: Yhat^T = W A1^T (M=128 f, N<=128 i1, K=32 r per
//      piece pair), V = Y^T A1 and M1 += Y W (N = 96 / 64: the factor pieces
//      concatenated along N);
//   0-3: SIMT, thread = fibre row f = TMEM lane: W pieces, e = y - yhat and
//      e^2, bf16 pieces of y, V epilogue (M2 in registers, M3 reduced).
// W and Yhat^T are double-buffered, so the model product of step s+1 runs
// while the SIMT warps consume step s; M1 stays in tensor memory for the
// CTA's whole segment.  Outputs are added to m / resid2 with float64 atomics
// (the caller zeroes them).  Every wait is bounded; a wait that runs out
// poisons the outputs with NaN and counts in g_tc_timeouts.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace cpdgn {

namespace {

constexpr int kTcThreads = 320;                  // warps 0-3 and 6-9 SIMT (two groups), 4 TMA, 5 MMA
constexpr int kSlots = 4;                        // TMA ring (16 KB boxes)
constexpr int kBoxBytes = 32 * 128 * 4;          // 32 i1 x 128 i2 float32
constexpr int kYpcBytes = 128 * 128 * 2;         // one bf16 piece of the tensor tile
// A1 chunk and W: 128 rows x (3 pieces x 32 columns) bf16, the piece index
// folded into the column so that [x0 x1 x2] is one 96-column operand.
constexpr int kArow = 3 * 4 * 128;               // bytes per 8-row group (12 column groups)
constexpr int kWrow = kArow;
constexpr int kFacBytes = 16 * kArow;            // 24 KB
constexpr int kWpcBytes = kFacBytes;
constexpr int kOffYpc = kSlots * kBoxBytes;
constexpr int kOffApc = kOffYpc + 2 * kYpcBytes;
constexpr int kOffWpc = kOffApc + kFacBytes;
constexpr int kSmemTc = kOffWpc + 2 * kWpcBytes;
// TMEM columns: Yhat^T x2 (128 each), V (3 x 32: one block per factor piece), M1 (3 x 32),
// the SIMT thread's A2 row and M2 accumulator (32 each)
constexpr uint32_t kColP = 0, kColV = 256, kColM1 = 352, kColA2 = 448, kColM2 = 480, kTmemCols = 512;

struct TcParams {
  int I1, I2, I3, R;
  int nc, nb, nseg;
  const double* a;     // A1 | A2 | A3, column-major, float64
  double* m;           // same layout, accumulated; may be null
  double* resid2;      // accumulated; may be null
  const int* skip;
  int grad;            // 1: the tensor-core products take e = y - y_hat (gradient blocks)
};

__device__ int g_tc_timeouts = 0;

// Byte offset of element (row, col) in a tile whose rows are 8-row groups of
// 16-byte core-matrix rows: group stride `gs`, column-group stride 128.
__device__ __forceinline__ uint32_t coff(int row, int col, int gs) {
  return uint32_t((row >> 3) * gs + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2);
}

// Pieces of row `row` of the A1 chunk (i1 = row index in A1): the R factor
// values are all loaded first, rounded once to float32 and split into three
// bfloat16 pieces in float32 arithmetic.  A float64 split would run its
// conversions and subtractions on this part's float64 pipe (about 2 results
// per clock per SM), which made the per-CTA setup of the pass cost ~10 us.
__device__ __forceinline__ void build_a1_row(const double* a, int64_t I1, int R, int i1, int row,
                                             unsigned char* apc) {
  float v[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = (i1 < I1 && r < R) ? float(a[i1 + I1 * r]) : 0.f;
#pragma unroll
  for (int rg = 0; rg < 4; ++rg) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      tc::split3x2(v[rg * 8 + h * 2], v[rg * 8 + h * 2 + 1], w0[h], w1[h], w2[h]);
    }
    *reinterpret_cast<uint4*>(apc + coff(row, rg * 8, kArow)) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(apc + coff(row, 32 + rg * 8, kArow)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(apc + coff(row, 64 + rg * 8, kArow)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
}

// lane l returns the sum over the warp of v[l] (recursive halving, 31 shuffles)
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = up ? v[i] : v[i + off];
      const float keep = up ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// Named barrier 1 over the 256 SIMT threads of the float32 pass (warps 0-3
// and 6-9); every SIMT thread reaches each call, so no decision that precedes
// one may differ per thread.
__device__ __forceinline__ void simt_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// The same barrier as a vote: true iff `v` holds in all 256 SIMT threads.
__device__ __forceinline__ bool simt_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(uint32_t(v))
      : "memory");
  return r != 0;
}

// W pieces of one step: row f = tid, W(f, r) = A2(i2, r) A3(i3, r) (float32),
// three bf16 pieces, written at the piece-interleaved layout (see kWrow).
__device__ __forceinline__ void build_w(unsigned char* wbuf, const float (&a2)[32], const float* a3, int tid) {
#pragma unroll
  for (int rg = 0; rg < 4; ++rg) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int r = rg * 8 + h * 2;
      tc::split3x2(a2[r] * a3[r], a2[r + 1] * a3[r + 1], w0[h], w1[h], w2[h]);
    }
    *reinterpret_cast<uint4*>(wbuf + coff(tid, rg * 8, kWrow)) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(wbuf + coff(tid, 32 + rg * 8, kWrow)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(wbuf + coff(tid, 64 + rg * 8, kWrow)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
}

// Half-row forms for the float32 pass, whose two SIMT warp groups each take
// 16 of the 32 rank columns (group g: ranks 16 g .. 16 g + 15).
__device__ __forceinline__ void build_a1_half(const double* a, int64_t I1, int R, int i1, int row, int g,
                                              unsigned char* apc) {
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int r = 16 * g + j;
    v[j] = (i1 < I1 && r < R) ? float(a[i1 + I1 * r]) : 0.f;
  }
#pragma unroll
  for (int rh = 0; rh < 2; ++rh) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      tc::split3x2(v[rh * 8 + h * 2], v[rh * 8 + h * 2 + 1], w0[h], w1[h], w2[h]);
    }
    const int c = 16 * g + rh * 8;
    *reinterpret_cast<uint4*>(apc + coff(row, c, kArow)) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(apc + coff(row, 32 + c, kArow)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(apc + coff(row, 64 + c, kArow)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
}

__device__ __forceinline__ void build_w_half(unsigned char* wbuf, const float (&a2)[16], const float* a3, int row,
                                             int g) {
#pragma unroll
  for (int rh = 0; rh < 2; ++rh) {
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int j = rh * 8 + h * 2;
      tc::split3x2(a2[j] * a3[16 * g + j], a2[j + 1] * a3[16 * g + j + 1], w0[h], w1[h], w2[h]);
    }
    const int c = 16 * g + rh * 8;
    *reinterpret_cast<uint4*>(wbuf + coff(row, c, kWrow)) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(wbuf + coff(row, 32 + c, kWrow)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(wbuf + coff(row, 64 + c, kWrow)) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
}

// lane l returns the sum over the warp of v[l % 16] (recursive halving over
// the 16 values, then the two half-warps added)
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 8; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const float send = up ? v[i] : v[i + off];
      const float keep = up ? v[i + off] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mttkrp_tc(const __grid_constant__ CUtensorMap tmap, TcParams p) {
  pdl_enter();
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar_full[kSlots], bar_empty[kSlots];
  __shared__ uint64_t bar_p[2], bar_mma, bar_ypc, bar_w[2];
  __shared__ uint32_t tbase_s;
  __shared__ float red[10][32];                    // per SIMT warp (indexed by warp number)
  __shared__ float a3s[3][32];
  __shared__ int abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int item = blockIdx.x;
  const int c = item % p.nc, b = (item / p.nc) % p.nb, seg = item / (p.nc * p.nb);
  const int s0 = int(int64_t(seg) * p.I3 / p.nseg), s1 = int(int64_t(seg + 1) * p.I3 / p.nseg);
  if (s0 >= s1) return;
  const int R = p.R;
  const int i1_0 = c * 128, i2_0 = b * 128;
  const int valid_i1 = min(128, p.I1 - i1_0);
  const int nbox = (valid_i1 + 31) / 32;
  const int ksteps_i1 = (valid_i1 + 15) / 16;
  const int n_p = nbox * 32;
  const int nsteps = s1 - s0;
  const int total_boxes = nsteps * nbox;
  const double* A3 = p.a + int64_t(p.I1 + p.I2) * R;

  unsigned char* stage = sm;
  unsigned char* ypc = sm + kOffYpc;
  unsigned char* apc = sm + kOffApc;
  unsigned char* wpc = sm + kOffWpc;

  if (tid == 0) {
    for (int k = 0; k < kSlots; ++k) {
      tc::mbar_init(&bar_full[k], 1);
      tc::mbar_init(&bar_empty[k], 4);
    }
    tc::mbar_init(&bar_p[0], 1);
    tc::mbar_init(&bar_p[1], 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init(&bar_ypc, 8);                    // every SIMT warp of both groups
    tc::mbar_init(&bar_w[0], 8);
    tc::mbar_init(&bar_w[1], 8);
    tc::fence_barrier_init();
    abort_s = 0;
  }
  if (warp == 5) {
    tc::tmem_alloc(&tbase_s, kTmemCols);
    tc::tmem_relinquish();
  }
  // SIMT groups: warps 0-3 (group 0) and 6-9 (group 1); a SIMT thread owns
  // row `srow` (TMEM lane) and the ranks 16 sg .. 16 sg + 15 of it, and
  // the tensor boxes 2 sg, 2 sg + 1 of every step
  const bool simt = warp < 4 || warp >= 6;
  const int sg = warp >= 6 ? 1 : 0;
  const int srow = 32 * (warp & 3) + lane;
  float a2[16];
  if (simt) {
    // zero the bf16 tensor pieces (columns past the valid i1 stay zero)
    uint4* z = reinterpret_cast<uint4*>(ypc);
    for (int e = srow + 128 * sg; e < 2 * kYpcBytes / 16; e += 256) z[e] = make_uint4(0, 0, 0, 0);
    // A1 chunk pieces, row t = i1 - i1_0, piece-interleaved (see kArow)
    build_a1_half(p.a, p.I1, R, i1_0 + srow, srow, sg, apc);
    const int i2 = i2_0 + srow;
    const double* A2 = p.a + int64_t(p.I1) * R;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int r = 16 * sg + j;
      a2[j] = (i2 < p.I2 && r < R) ? float(A2[i2 + int64_t(p.I2) * r]) : 0.f;
    }
    if (tid < 32) {
      a3s[0][tid] = (tid < R) ? float(A3[s0 + int64_t(p.I3) * tid]) : 0.f;
      if (nsteps > 1) a3s[1][tid] = (tid < R) ? float(A3[s0 + 1 + int64_t(p.I3) * tid]) : 0.f;
    }
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tb = tbase_s;

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int g = 0;
      for (; g < total_boxes; ++g) {
        const int slot = g % kSlots;
        if (g >= kSlots && !tc::mbar_wait(&bar_empty[slot], ((g / kSlots) - 1) & 1)) break;
        if (*reinterpret_cast<volatile int*>(&abort_s)) break;
        const int st = g / nbox, k = g % nbox;
        tc::mbar_expect_tx(&bar_full[slot], kBoxBytes);
        tc::tma_load_3d(stage + slot * kBoxBytes, &tmap, i1_0 + 32 * k, i2_0, s0 + st, &bar_full[slot]);
      }
      if (g < total_boxes) atomicExch(&abort_s, 1);
      // the last boxes issued must land before the CTA exits
      for (int h = max(0, g - kSlots); h < g; ++h) tc::mbar_wait(&bar_full[h % kSlots], (h / kSlots) & 1, 200000000ull);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t yb = tc::smem_u32(ypc), ab = tc::smem_u32(apc), wb = tc::smem_u32(wpc);
      const uint32_t idp = tc::idesc_bf16(128, n_p, false, false);
      const uint32_t idv = tc::idesc_bf16(128, 96, false, true);
      const uint32_t idv2 = tc::idesc_bf16(128, 64, false, true);
      const uint32_t idm = tc::idesc_bf16(128, 96, true, true);
      const uint32_t idm2 = tc::idesc_bf16(128, 64, true, true);
      // Yhat^T(step) = sum over piece pairs of W_p A1_q^T (K = 32 per piece)
      auto issue_p = [&](int st) {
        const uint32_t wbuf = wb + (st & 1) * kWpcBytes;
        const uint32_t dcol = tb + kColP + (st & 1) * 128;
        const int pw[6] = {0, 0, 1, 0, 1, 2}, pa[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
        for (int cmb = 0; cmb < 6; ++cmb)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ad = tc::sdesc(wbuf + pw[cmb] * 512 + ks * 256, 128, kWrow);
            const uint64_t bd = tc::sdesc(ab + pa[cmb] * 512 + ks * 256, 128, kArow);
            tc::mma_bf16(dcol, ad, bd, idp, (cmb | ks) ? 1u : 0u);
          }
        tc::mma_commit(&bar_p[st & 1]);
      };
      bool ok = tc::mbar_wait(&bar_w[0], 0);
      tc::tc_fence_after();
      if (ok) issue_p(0);
      for (int st = 0; st < nsteps && ok; ++st) {
        // model product of the next step first: it runs while the SIMT warps
        // consume this step
        if (st + 1 < nsteps) {
          ok = tc::mbar_wait(&bar_w[(st + 1) & 1], ((st + 1) >> 1) & 1);
          if (!ok) break;
          tc::tc_fence_after();
          issue_p(st + 1);
        }
        // V(st) and M1 += ... once the tensor pieces of step st are written
        ok = tc::mbar_wait(&bar_ypc, st & 1);
        if (!ok) break;
        tc::tc_fence_after();
        const uint32_t wbuf = wb + (st & 1) * kWpcBytes;
        const uint32_t vcol = tb + kColV;
        // V: y0 x [a0 a1 a2] (N = 96) and y1 x [a0 a1] (N = 64) into the same
        // column blocks (block q holds the products with piece q), K = i1
        for (int ks = 0; ks < ksteps_i1; ++ks) {
          tc::mma_bf16(vcol, tc::sdesc(yb + ks * 256, 128, 2048), tc::sdesc(ab + ks * 2 * kArow, kArow, 128), idv,
                       ks ? 1u : 0u);
          tc::mma_bf16(vcol, tc::sdesc(yb + kYpcBytes + ks * 256, 128, 2048),
                       tc::sdesc(ab + ks * 2 * kArow, kArow, 128), idv2, 1u);
        }
        // M1: y0 x [w0 w1 w2] and y1 x [w0 w1], K = f (128), accumulated over steps
        for (int ks = 0; ks < 8; ++ks) {
          tc::mma_bf16(tb + kColM1, tc::sdesc(yb + ks * 4096, 2048, 128), tc::sdesc(wbuf + ks * 2 * kWrow, kWrow, 128),
                       idm, (st > 0 || ks > 0) ? 1u : 0u);
          tc::mma_bf16(tb + kColM1, tc::sdesc(yb + kYpcBytes + ks * 4096, 2048, 128),
                       tc::sdesc(wbuf + ks * 2 * kWrow, kWrow, 128), idm2, 1u);
        }
        tc::mma_commit(&bar_mma);
      }
      if (!ok) atomicExch(&abort_s, 1);
      // let every issued MMA finish before TMEM is released
      tc::mbar_wait(&bar_mma, (nsteps - 1) & 1, 200000000ull);
    }
  } else {
    // ---------------- SIMT warps 0-3 and 6-9 (TMEM lanes 32 (w % 4) ..) ----------------
    const uint32_t lane_base = uint32_t((warp & 3) * 32) << 16;
    const uint32_t tl = tb + lane_base;
    const uint32_t hc = 16 * sg;                   // this group's first rank column
    {
      float z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0.f;
      tc::tmem_st16(tl + kColA2 + hc, a2);
      tc::tmem_st16(tl + kColM2 + hc, z);
    }
    double racc = 0.0;
    bool ok = true;
    auto make_w = [&](int st) {
      float a2r[16];
      tc::tmem_ld16(tl + kColA2 + hc, a2r);
      build_w_half(wpc + (st & 1) * kWpcBytes, a2r, a3s[st % 3], srow, sg);
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_w[st & 1]);
    };
    // V epilogue: M2 (+)= V A3(i3, :) in TMEM, M3(i3, :) = sum_f V A2 (atomics);
    // each group takes its 16 ranks
    auto v_epilogue = [&](int st) {
      float v[16], t[16];
      tc::tmem_ld16(tl + kColV + hc, v);
#pragma unroll
      for (int q = 1; q < 3; ++q) {
        tc::tmem_ld16(tl + kColV + 32 * q + hc, t);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += t[j];
      }
      const float* a3 = a3s[st % 3];
      tc::tmem_ld16(tl + kColM2 + hc, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) t[j] = fmaf(v[j], a3[hc + j], t[j]);
      tc::tmem_st16(tl + kColM2 + hc, t);
      tc::tmem_ld16(tl + kColA2 + hc, t);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] *= t[j];
      const float sum = warp_transpose_sum16(v);
      red[warp][lane] = sum;
      simt_sync();
      if (lane < 16 && (warp & 3) == 0) {          // warp 0: ranks 0-15, warp 8: ranks 16-31
        const int r = int(hc) + lane;
        const int w0 = sg ? 6 : 0;
        if (r < R && p.m) {
          const float tt = red[w0][lane] + red[w0 + 1][lane] + red[w0 + 2][lane] + red[w0 + 3][lane];
          atomicAdd(p.m + int64_t(p.I1 + p.I2) * R + (s0 + st) + int64_t(p.I3) * r, double(tt));
        }
      }
    };
    make_w(0);

    // boxes of this group: 2 sg, 2 sg + 1 (those below nbox)
    const int kb0 = 2 * sg, kb1 = (2 * sg + 2 < nbox) ? 2 * sg + 2 : nbox;
    for (int st = 0; st < nsteps; ++st) {
      // prefetch A3 row of step st + 2 (stored once V epilogue st - 1 is done)
      float a3next = 0.f;
      const bool pre = tid < 32 && st + 2 < nsteps;
      if (pre) a3next = (tid < R) ? float(A3[s0 + st + 2 + int64_t(p.I3) * tid]) : 0.f;
      // tensor pieces, V and the other W buffer are free once V/M1 of step st - 1 completed
      if (st > 0) {
        ok = simt_all(__all_sync(0xffffffffu, tc::mbar_wait(&bar_mma, (st - 1) & 1)) &&
                      !*reinterpret_cast<volatile int*>(&abort_s));
        if (!ok) break;
        tc::tc_fence_after();
        v_epilogue(st - 1);
      }
      if (pre) a3s[(st + 2) % 3][tid] = a3next;
      if (st + 1 < nsteps) {
        simt_sync();
        make_w(st + 1);
      }
      ok = simt_all(__all_sync(0xffffffffu, tc::mbar_wait(&bar_p[st & 1], (st >> 1) & 1)) &&
                    !*reinterpret_cast<volatile int*>(&abort_s));
      if (!ok) break;
      tc::tc_fence_after();
      const uint32_t pcol = tl + kColP + (st & 1) * 128;
      bool wok = true;
      uint32_t phr[32];
      if (kb0 < kb1) tc::tmem_ld32_async(pcol + 32 * kb0, phr);
      for (int k = kb0; k < kb1; ++k) {
        const int g = st * nbox + k;
        const int slot = g % kSlots;
        tc::tmem_wait_ld();
        float ph[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) ph[j] = __uint_as_float(phr[j]);
        if (k + 1 < kb1) tc::tmem_ld32_async(pcol + 32 * (k + 1), phr);
        wok = __all_sync(0xffffffffu, tc::mbar_wait(&bar_full[slot], (g / kSlots) & 1));
        if (!wok) break;
        const unsigned char* row = stage + slot * kBoxBytes + srow * 128;
        float y[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 v = *reinterpret_cast<const float4*>(row + ((j ^ (srow & 7)) << 4));
          y[4 * j] = v.x;
          y[4 * j + 1] = v.y;
          y[4 * j + 2] = v.z;
          y[4 * j + 3] = v.w;
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bar_empty[slot]);
        float e2 = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float e = y[j] - ph[j];
          e2 = fmaf(e, e, e2);
          if (p.grad) y[j] = e;        // the pieces below are then those of E
        }
        racc += double(e2);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          uint32_t h0[4], h1[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float ya = y[g8 * 8 + 2 * h], yb = y[g8 * 8 + 2 * h + 1];
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(ya, yb);
            const float2 f0 = __bfloat1622float2(p0);
            const __nv_bfloat162 p1 = __floats2bfloat162_rn(ya - f0.x, yb - f0.y);
            h0[h] = *reinterpret_cast<const uint32_t*>(&p0);
            h1[h] = *reinterpret_cast<const uint32_t*>(&p1);
          }
          const uint32_t o = coff(srow, 32 * k + 8 * g8, 2048);
          *reinterpret_cast<uint4*>(ypc + o) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
          *reinterpret_cast<uint4*>(ypc + kYpcBytes + o) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
        }
      }
      if (!wok) tc::tmem_wait_ld();
      ok = simt_all(wok);
      if (!ok) break;
      tc::fence_async_smem();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_ypc);
    }
    // one decision for all SIMT warps before the collective TMEM reads below
    if (ok) ok = __all_sync(0xffffffffu, tc::mbar_wait(&bar_mma, (nsteps - 1) & 1));
    ok = simt_all(ok && !*reinterpret_cast<volatile int*>(&abort_s));
    if (ok) {
      tc::tc_fence_after();
      v_epilogue(nsteps - 1);
      // M1 flush: lanes are i1 of the chunk; the three column blocks summed
      float v[16], t[16];
      tc::tmem_ld16(tl + kColM1 + hc, v);
#pragma unroll
      for (int q = 1; q < 3; ++q) {
        tc::tmem_ld16(tl + kColM1 + 32 * q + hc, t);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += t[j];
      }
      tc::tmem_ld16(tl + kColM2 + hc, t);
      if (p.m) {
        const int i1 = i1_0 + srow;
        if (i1 < p.I1) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (int(hc) + j < R) atomicAdd(p.m + i1 + int64_t(p.I1) * (int(hc) + j), double(v[j]));
        }
        const int i2 = i2_0 + srow;
        if (i2 < p.I2) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (int(hc) + j < R)
              atomicAdd(p.m + int64_t(p.I1) * R + i2 + int64_t(p.I2) * (int(hc) + j), double(t[j]));
        }
      }
      if (p.resid2) {
        double t2 = racc;
        for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
        if (lane == 0) atomicAdd(p.resid2, t2);
      }
    } else if (tid == 0) {
      atomicExch(&abort_s, 1);
      atomicAdd(&g_tc_timeouts, 1);
      if (p.resid2) atomicAdd(p.resid2, __longlong_as_double(0x7ff8000000000000ll));
      if (p.m) atomicAdd(p.m, __longlong_as_double(0x7ff8000000000000ll));
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 5) tc::tmem_dealloc(tb, kTmemCols);
}

// ---------------------------------------------------------------------------
// Two-plane bfloat16 tensors (CP_BF16X2: y = hi + lo; CP_BF16: y = hi).
// The planes are the tensor-core operands as TMA lands them (128-byte
// swizzle): V = Y^T A1 reads a plane tile K-major (rows f, K = i1) and
// M1 += Y W reads the same tile MN-major (M = i1, K = f), so no SIMT pass
// touches the tensor before the MMAs.  The SIMT warps only form the residual
// (y - yhat)^2 from the same tiles, concurrently with V / M1.  A step's tile
// slot is released by the four SIMT warps and by an MMA commit.
// ---------------------------------------------------------------------------
constexpr int kPlaneBox = 64 * 128 * 2;                // 64 i1 x 128 f bfloat16, 16 KB
constexpr int kStepBytes = 4 * kPlaneBox;              // 2 planes x 2 boxes
constexpr int kStages3 = 2;
constexpr int kOffApc3 = kStages3 * kStepBytes;
constexpr int kOffWpc3 = kOffApc3 + kFacBytes;
constexpr int kSmemTc3 = kOffWpc3 + 2 * kWpcBytes;

struct Tc3Params {
  TcParams t;
  int nplanes;         // 2: hi + lo, 1: hi only
};

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t kstride, uint32_t mnstride) {
  return tc::sdesc(saddr, kstride, mnstride) | (uint64_t(2) << 61);
}

constexpr int kTcThreads3 = 320;   // warps 0-3 residual, 4 TMA, 5 MMA, 6-9 epilogue / W

// Named barrier 2 over the 128 epilogue threads (warps 6-9).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }
__device__ __forceinline__ bool epi_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 2, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(uint32_t(v))
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kTcThreads3, 1)
    k_mttkrp_tc3(const __grid_constant__ CUtensorMap tmap_hi, const __grid_constant__ CUtensorMap tmap_lo,
                 Tc3Params p3) {
  pdl_enter();
  const TcParams& p = p3.t;
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar_full[kStages3], bar_empty[kStages3];
  __shared__ uint64_t bar_p[2], bar_mma, bar_w[2], bar_vfree;
  __shared__ uint32_t tbase_s;
  __shared__ float red[4][32];
  __shared__ float a3s[3][32];
  __shared__ int abort_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int item = blockIdx.x;
  const int c = item % p.nc, b = (item / p.nc) % p.nb, seg = item / (p.nc * p.nb);
  const int s0 = int(int64_t(seg) * p.I3 / p.nseg), s1 = int(int64_t(seg + 1) * p.I3 / p.nseg);
  if (s0 >= s1) return;
  const int R = p.R;
  const int nplanes = p3.nplanes;
  const int i1_0 = c * 128, i2_0 = b * 128;
  const int valid_i1 = min(128, p.I1 - i1_0);
  const int ksteps_i1 = (valid_i1 + 15) / 16;
  const int nsteps = s1 - s0;
  const double* A3 = p.a + int64_t(p.I1 + p.I2) * R;
  // fibre row of this thread in the residual (warps 0-3) and epilogue (6-9) groups
  const int row = (warp & 3) * 32 + lane;
  const uint32_t lane_off = uint32_t((warp & 3) * 32) << 16;

  unsigned char* stage = sm;
  unsigned char* apc = sm + kOffApc3;
  unsigned char* wpc = sm + kOffWpc3;

  if (tid == 0) {
    for (int k = 0; k < kStages3; ++k) {
      tc::mbar_init(&bar_full[k], 1);
      tc::mbar_init(&bar_empty[k], 5);          // 4 residual warps + the MMA commit
    }
    tc::mbar_init(&bar_p[0], 1);
    tc::mbar_init(&bar_p[1], 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_init(&bar_w[0], 4);
    tc::mbar_init(&bar_w[1], 4);
    tc::mbar_init(&bar_vfree, 4);
    tc::fence_barrier_init();
    abort_s = 0;
  }
  if (warp == 5) {
    tc::tmem_alloc(&tbase_s, kTmemCols);
    tc::tmem_relinquish();
  }
  if (warp < 4) {
    // A1 chunk pieces (rows i1 - i1_0), piece-interleaved
    build_a1_row(p.a, p.I1, R, i1_0 + row, row, apc);
  }
  if (warp == 6) {
    a3s[0][lane] = (lane < R) ? float(A3[s0 + int64_t(p.I3) * lane]) : 0.f;
    if (nsteps > 1) a3s[1][lane] = (lane < R) ? float(A3[s0 + 1 + int64_t(p.I3) * lane]) : 0.f;
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tb = tbase_s;

  if (warp == 4) {
    // ---------------- TMA producer: one step = nplanes x 2 boxes ----------------
    if (lane == 0) {
      const uint32_t bytes = uint32_t(nplanes) * 2 * kPlaneBox;
      int st = 0;
      for (; st < nsteps; ++st) {
        const int slot = st % kStages3;
        if (st >= kStages3 && !tc::mbar_wait(&bar_empty[slot], ((st / kStages3) - 1) & 1)) break;
        if (*reinterpret_cast<volatile int*>(&abort_s)) break;
        unsigned char* dst = stage + slot * kStepBytes;
        tc::mbar_expect_tx(&bar_full[slot], bytes);
        for (int k = 0; k < 2; ++k) {
          tc::tma_load_3d(dst + k * kPlaneBox, &tmap_hi, i1_0 + 64 * k, i2_0, s0 + st, &bar_full[slot]);
          if (nplanes == 2)
            tc::tma_load_3d(dst + 2 * kPlaneBox + k * kPlaneBox, &tmap_lo, i1_0 + 64 * k, i2_0, s0 + st,
                            &bar_full[slot]);
        }
      }
      if (st < nsteps) atomicExch(&abort_s, 1);
      for (int h = max(0, st - kStages3); h < st; ++h)
        tc::mbar_wait(&bar_full[h % kStages3], (h / kStages3) & 1, 200000000ull);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t sb = tc::smem_u32(stage), ab = tc::smem_u32(apc), wb = tc::smem_u32(wpc);
      const uint32_t idp = tc::idesc_bf16(128, 128, false, false);
      const uint32_t idv = tc::idesc_bf16(128, 96, false, true);
      const uint32_t idv2 = tc::idesc_bf16(128, 64, false, true);
      const uint32_t idm = tc::idesc_bf16(128, 96, true, true);
      const uint32_t idm2 = tc::idesc_bf16(128, 64, true, true);
      // descriptors are built once; a byte offset d moves the start field by d >> 4
      // (every operand lies below 256 KB, so the 14-bit field never carries)
      const uint64_t dWp = tc::sdesc(wb, 128, kWrow), dAp = tc::sdesc(ab, 128, kArow);
      const uint64_t dAv = tc::sdesc(ab, kArow, 128), dWm = tc::sdesc(wb, kWrow, 128);
      const uint64_t dYv = sdesc_sw128(sb, 16, 1024), dYm = sdesc_sw128(sb, kPlaneBox, 1024);
      auto issue_p = [&](int st) {
        const uint64_t wbuf = dWp + (((st & 1) * kWpcBytes) >> 4);
        const uint32_t dcol = tb + kColP + (st & 1) * 128;
        constexpr uint32_t offw[6] = {0, 0, 32, 0, 32, 64}, offa[6] = {0, 32, 0, 64, 32, 0};
#pragma unroll
        for (int cmb = 0; cmb < 6; ++cmb)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
            tc::mma_bf16(dcol, wbuf + offw[cmb] + ks * 16, dAp + offa[cmb] + ks * 16, idp, (cmb | ks) ? 1u : 0u);
        tc::mma_commit(&bar_p[st & 1]);
      };
      bool ok = tc::mbar_wait(&bar_w[0], 0);
      tc::tc_fence_after();
      if (ok) issue_p(0);
      for (int st = 0; st < nsteps && ok; ++st) {
        const int slot = st % kStages3;
        ok = tc::mbar_wait(&bar_full[slot], (st / kStages3) & 1);
        if (ok && st > 0) ok = tc::mbar_wait(&bar_vfree, (st - 1) & 1);
        if (!ok) break;
        tc::tc_fence_after();
        const uint32_t toff = (slot * kStepBytes) >> 4;
        const uint64_t wm = dWm + (((st & 1) * kWpcBytes) >> 4);
        // V(f, [q r]) = sum_i1 plane(i1, f) A1_q(i1, r): hi x [a0 a1 a2], lo x [a0 a1]
#pragma unroll 1
        for (int pl = 0; pl < nplanes; ++pl) {
          const uint64_t yv = dYv + toff + ((pl * 2 * kPlaneBox) >> 4);
          const uint32_t id = pl ? idv2 : idv;
#pragma unroll 1
          for (int ks = 0; ks < ksteps_i1; ++ks)
            tc::mma_bf16(tb + kColV, yv + (((ks >> 2) * kPlaneBox + (ks & 3) * 32) >> 4),
                         dAv + ((ks * 2 * kArow) >> 4), id, (pl | ks) ? 1u : 0u);
        }
        // M1(i1, [q r]) += sum_f plane(i1, f) W_q(f, r), the plane tile read MN-major
#pragma unroll 1
        for (int pl = 0; pl < nplanes; ++pl) {
          const uint64_t ym = dYm + toff + ((pl * 2 * kPlaneBox) >> 4);
          const uint32_t id = pl ? idm2 : idm;
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            tc::mma_bf16(tb + kColM1, ym + ks * 128, wm + ks * ((2 * kWrow) >> 4), id, (st | pl | ks) ? 1u : 0u);
        }
        tc::mma_commit(&bar_mma);
        tc::mma_commit(&bar_empty[slot]);
        if (st + 1 < nsteps) {
          ok = tc::mbar_wait(&bar_w[(st + 1) & 1], ((st + 1) >> 1) & 1);
          // the model buffer of step st + 1 was last read by the residual of step st - 1
          if (ok && st >= 1) ok = tc::mbar_wait(&bar_empty[(st - 1) % kStages3], ((st - 1) / kStages3) & 1);
          if (!ok) break;
          tc::tc_fence_after();
          issue_p(st + 1);
        }
      }
      if (!ok) atomicExch(&abort_s, 1);
      tc::mbar_wait(&bar_mma, (nsteps - 1) & 1, 200000000ull);
    }
  } else if (warp < 4) {
    // ---------------- residual warps: (hi + lo - yhat)^2 over the step tile ----------------
    const uint32_t tl = tb + lane_off;
    double racc = 0.0;
    bool ok = true;
    for (int st = 0; st < nsteps && ok; ++st) {
      const int slot = st % kStages3;
      ok = __all_sync(0xffffffffu, tc::mbar_wait(&bar_full[slot], (st / kStages3) & 1) &&
                                       tc::mbar_wait(&bar_p[st & 1], (st >> 1) & 1)) &&
           !*reinterpret_cast<volatile int*>(&abort_s);
      if (!ok) break;
      tc::tc_fence_after();
      const unsigned char* tile = stage + slot * kStepBytes;
      const uint32_t pcol = tl + kColP + (st & 1) * 128;
      float e2 = 0.f;
#pragma unroll 1
      for (int k = 0; k < 2; ++k) {
        const unsigned char* rh = tile + k * kPlaneBox + row * 128;
        const unsigned char* rl = rh + 2 * kPlaneBox;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float ph[32];
          tc::tmem_ld32(pcol + 64 * k + 32 * h, ph);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int ch = ((4 * h + j) ^ (row & 7)) << 4;
            const uint4 hv = *reinterpret_cast<const uint4*>(rh + ch);
            uint4 lv = make_uint4(0, 0, 0, 0);
            if (nplanes == 2) lv = *reinterpret_cast<const uint4*>(rl + ch);
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float y0 = __uint_as_float(hw[q] << 16) + __uint_as_float(lw[q] << 16);
              const float y1 = __uint_as_float(hw[q] & 0xffff0000u) + __uint_as_float(lw[q] & 0xffff0000u);
              const float ea = y0 - ph[8 * j + 2 * q], eb = y1 - ph[8 * j + 2 * q + 1];
              e2 = fmaf(ea, ea, e2);
              e2 = fmaf(eb, eb, e2);
            }
          }
        }
      }
      racc += double(e2);
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_empty[slot]);
    }
    if (!ok) {
      if (lane == 0) atomicExch(&abort_s, 1);
    } else if (p.resid2) {
      double t2 = racc;
      for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
      if (lane == 0) atomicAdd(p.resid2, t2);
    }
  } else {
    // ---------------- epilogue warps 6-9: W pieces, V epilogue, M1 / M2 flush ----------------
    const uint32_t tl = tb + lane_off;
    const int ew = warp - 6;                 // 0..3 within the group
    float a2[32], m2acc[32];
    {
      const int i2 = i2_0 + row;
      const double* A2 = p.a + int64_t(p.I1) * R;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        a2[r] = (i2 < p.I2 && r < R) ? float(A2[i2 + int64_t(p.I2) * r]) : 0.f;
        m2acc[r] = 0.f;
      }
    }
    bool ok = true;
    auto make_w = [&](int st) {
      build_w(wpc + (st & 1) * kWpcBytes, a2, a3s[st % 3], row);
      tc::fence_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_w[st & 1]);
    };
    make_w(0);
    for (int st = 0; st < nsteps; ++st) {
      float a3next = 0.f;
      const bool pre = ew == 0 && st + 2 < nsteps;
      if (pre) a3next = (lane < R) ? float(A3[s0 + st + 2 + int64_t(p.I3) * lane]) : 0.f;
      // W of the next step (its buffer was last read by M1 of step st - 1, done)
      if (st + 1 < nsteps) {
        epi_sync();
        make_w(st + 1);
      }
      ok = epi_all(__all_sync(0xffffffffu, tc::mbar_wait(&bar_mma, st & 1)) &&
                   !*reinterpret_cast<volatile int*>(&abort_s));
      if (!ok) break;
      tc::tc_fence_after();
      // V epilogue: M2 += V A3(i3, :) (registers), M3(i3, :) = sum_f V A2
      {
        float v[32], t[32];
        tc::tmem_ld32(tl + kColV, v);
#pragma unroll
        for (int q = 1; q < 3; ++q) {
          tc::tmem_ld32(tl + kColV + 32 * q, t);
#pragma unroll
          for (int r = 0; r < 32; ++r) v[r] += t[r];
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bar_vfree);     // V may be overwritten now
        const float* a3 = a3s[st % 3];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          m2acc[r] = fmaf(v[r], a3[r], m2acc[r]);
          v[r] *= a2[r];
        }
        const float sum = warp_transpose_sum(v);
        red[ew][lane] = sum;
        epi_sync();
        if (ew == 0 && lane < R && p.m) {
          const float tt = red[0][lane] + red[1][lane] + red[2][lane] + red[3][lane];
          atomicAdd(p.m + int64_t(p.I1 + p.I2) * R + (s0 + st) + int64_t(p.I3) * lane, double(tt));
        }
      }
      if (pre) a3s[(st + 2) % 3][lane] = a3next;
    }
    ok = epi_all(ok && !*reinterpret_cast<volatile int*>(&abort_s));
    if (ok) {
      float v[32], t[32];
      tc::tmem_ld32(tl + kColM1, v);
#pragma unroll
      for (int q = 1; q < 3; ++q) {
        tc::tmem_ld32(tl + kColM1 + 32 * q, t);
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] += t[r];
      }
      if (p.m) {
        const int i1 = i1_0 + row;
        if (i1 < p.I1) {
#pragma unroll
          for (int r = 0; r < 32; ++r)
            if (r < R) atomicAdd(p.m + i1 + int64_t(p.I1) * r, double(v[r]));
        }
        const int i2 = i2_0 + row;
        if (i2 < p.I2) {
#pragma unroll
          for (int r = 0; r < 32; ++r)
            if (r < R) atomicAdd(p.m + int64_t(p.I1) * R + i2 + int64_t(p.I2) * r, double(m2acc[r]));
        }
      }
    } else if (row == 0) {
      atomicExch(&abort_s, 1);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0 && *reinterpret_cast<volatile int*>(&abort_s)) {
    atomicAdd(&g_tc_timeouts, 1);
    if (p.resid2) atomicAdd(p.resid2, __longlong_as_double(0x7ff8000000000000ll));
    if (p.m) atomicAdd(p.m, __longlong_as_double(0x7ff8000000000000ll));
  }
  if (warp == 5) tc::tmem_dealloc(tb, kTmemCols);
}

__global__ void k_split_bf16x2(const float* __restrict__ Y, int64_t J, __nv_bfloat16* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < J; i += int64_t(gridDim.x) * blockDim.x) {
    const float y = Y[i];
    const __nv_bfloat16 hi = __float2bfloat16_rn(y);
    out[i] = hi;
    out[J + i] = __float2bfloat16_rn(y - __bfloat162float(hi));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

bool tc_disabled() {
  static const bool off = [] {
    const char* e = std::getenv("CPDGN_NO_TC");
    return e && e[0] && e[0] != '0';
  }();
  return off;
}

int launch_tc(const CUtensorMap& tm, const TcParams& p, int grid, cudaStream_t s) {
  if (cudaFuncSetAttribute(k_mttkrp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc) != cudaSuccess)
    return CP_ECUDA;
  CP_CUDA(launch_pdl(k_mttkrp_tc, grid, kTcThreads, kSmemTc, s, tm, p));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

}  // namespace

static int launch_tc3(const Dims& d, const void* Y, const double* a, double* m, double* resid2, const int* skip,
                      cudaStream_t s) {
  if (d.N != 3 || d.R > 32 || d.R < 1 || d.I[0] % 8 != 0 || (reinterpret_cast<uintptr_t>(Y) & 15) != 0)
    return CP_EINVAL;
  if (d.I[0] > (int64_t(1) << 30) || d.I[1] > (int64_t(1) << 30) || d.I[2] > (int64_t(1) << 30)) return CP_EINVAL;
  if (!m && !resid2) return CP_OK;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return CP_EINVAL;
  const int nplanes = d.y_dtype == CP_BF16X2 ? 2 : 1;
  CUtensorMap tm[2];
  cuuint64_t gdim[3] = {cuuint64_t(d.I[0]), cuuint64_t(d.I[1]), cuuint64_t(d.I[2])};
  cuuint64_t gstr[2] = {cuuint64_t(d.I[0]) * 2, cuuint64_t(d.I[0]) * d.I[1] * 2};
  cuuint32_t box[3] = {64, 128, 1}, es[3] = {1, 1, 1};
  for (int pl = 0; pl < 2; ++pl) {
    const __nv_bfloat16* base = static_cast<const __nv_bfloat16*>(Y) + (pl < nplanes ? pl : 0) * d.J;
    if (enc(&tm[pl], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base), gdim, gstr, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return CP_EINVAL;
  }
  Tc3Params p3;
  TcParams& p = p3.t;
  p.I1 = int(d.I[0]);
  p.I2 = int(d.I[1]);
  p.I3 = int(d.I[2]);
  p.R = d.R;
  p.nc = (p.I1 + 127) / 128;
  p.nb = (p.I2 + 127) / 128;
  p.nseg = kSMs / (p.nc * p.nb);
  if (p.nseg < 1) p.nseg = 1;
  if (p.nseg > p.I3) p.nseg = p.I3;
  p.a = a;
  p.m = m;
  p.resid2 = resid2;
  p.skip = skip;
  p.grad = 0;
  p3.nplanes = nplanes;
  const int64_t grid = int64_t(p.nc) * p.nb * p.nseg;
  if (grid > (int64_t(1) << 31) - 1) return CP_EINVAL;
  if (cudaFuncSetAttribute(k_mttkrp_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTc3) != cudaSuccess)
    return CP_ECUDA;
  CP_CUDA(launch_pdl(k_mttkrp_tc3, int(grid), kTcThreads3, kSmemTc3, s, tm[0], tm[1], p3));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

// Device address of g_tc_timeouts on the current device (looked up once per
// device; the counter counts the bounded waits of the tensor-core passes
// that ran out, over every call of the process on that device).
int tc_timeout_counter(int** out) {
  static std::mutex mu;
  static int* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CP_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_timeouts) != cudaSuccess) return CP_ECUDA;
    addr[dev] = static_cast<int*>(p);
  }
  *out = addr[dev];
  return CP_OK;
}

// CP_EINVAL when the shape or pointers do not suit a tensor-core pass (the
// caller falls back to the SIMT kernels); m and resid2 must be zeroed.
int launch_mttkrp_tc(const Dims& d, const void* Y, const double* a, double* m, double* resid2, const int* skip,
                     cudaStream_t s, int grad) {
  if (d.y_dtype == CP_BF16X2) return grad ? CP_EINVAL : launch_tc3(d, Y, a, m, resid2, skip, s);
  if (tc_disabled()) return CP_EINVAL;
  // the bfloat16 pass feeds Y's plane to the MMAs directly: no gradient form
  if (d.y_dtype == CP_BF16) return grad ? CP_EINVAL : launch_tc3(d, Y, a, m, resid2, skip, s);
  if (d.N != 3 || d.y_dtype != CP_F32 || d.R > 32 || d.R < 1) return CP_EINVAL;
  if (d.I[0] % 4 != 0 || (reinterpret_cast<uintptr_t>(Y) & 15) != 0) return CP_EINVAL;
  if (d.I[0] > (int64_t(1) << 30) || d.I[1] > (int64_t(1) << 30) || d.I[2] > (int64_t(1) << 30)) return CP_EINVAL;
  if (!m && !resid2) return CP_OK;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return CP_EINVAL;
  CUtensorMap tm;
  cuuint64_t gdim[3] = {cuuint64_t(d.I[0]), cuuint64_t(d.I[1]), cuuint64_t(d.I[2])};
  cuuint64_t gstr[2] = {cuuint64_t(d.I[0]) * 4, cuuint64_t(d.I[0]) * d.I[1] * 4};
  cuuint32_t box[3] = {32, 128, 1}, es[3] = {1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(Y), gdim, gstr, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return CP_EINVAL;
  TcParams p;
  p.I1 = int(d.I[0]);
  p.I2 = int(d.I[1]);
  p.I3 = int(d.I[2]);
  p.R = d.R;
  p.nc = (p.I1 + 127) / 128;
  p.nb = (p.I2 + 127) / 128;
  p.nseg = kSMs / (p.nc * p.nb);
  if (p.nseg < 1) p.nseg = 1;
  if (p.nseg > p.I3) p.nseg = p.I3;
  p.a = a;
  p.m = m;
  p.resid2 = resid2;
  p.skip = skip;
  p.grad = grad;
  const int64_t grid = int64_t(p.nc) * p.nb * p.nseg;
  if (grid > (int64_t(1) << 31) - 1) return CP_EINVAL;
  return launch_tc(tm, p, int(grid), s);
}

}  // namespace cpdgn

namespace cpdgn {
// An mbarrier that expects one arrival which never comes: the bounded wait
// gives up after limit_ns and the event is counted like a timed-out wait of
// the pass.  Nothing asynchronous is issued, so there is nothing to drain.
__global__ void k_selftest_wait(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) ok = tc::mbar_wait(&bar, 0, limit_ns);
  if (threadIdx.x == 0 && !ok) atomicAdd(&g_tc_timeouts, 1);
}
}  // namespace cpdgn

extern "C" int cp_selftest_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 10000000000ll) return CP_EINVAL;
  cpdgn::k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(uint64_t(limit_ns));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}

extern "C" int cp_tensor_split(const float* Y, int64_t J, void* out, void* stream) {
  if (!Y || !out || J < 1 || (reinterpret_cast<uintptr_t>(out) & 15) != 0) return CP_EINVAL;
  int64_t g = (J + 255) / 256;
  if (g > 8 * cpdgn::kSMs) g = 8 * cpdgn::kSMs;
  cpdgn::k_split_bf16x2<<<unsigned(g), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      Y, J, static_cast<__nv_bfloat16*>(out));
  return cudaGetLastError() == cudaSuccess ? CP_OK : CP_ECUDA;
}
