// Batched form, host side: problem checks, workspace layout and the launch
// dispatch over the tensor-tile width.  The kernel is in batch_kernel.cuh,
// compiled once per width (batch_tile8.cu, batch_tile16.cu, batch_tile32.cu).
#include "batch.cuh"

using namespace cpdgn;

static size_t batch_ws_one(const cp_batch_problem& p) {
  const int64_t RR = int64_t(p.R) * p.R;
  int64_t T = 0;
  for (int k = 0; k < p.N; ++k) T += p.I[k];
  const int64_t n = p.N * RR;
  size_t d = size_t(4 * T * p.R + 5 * p.N * RR + p.N * p.N * RR + 7 * n + p.N * (p.N - 1) / 2 * RR * p.R);
  size_t bytes = d * sizeof(double) + size_t(n) * n * sizeof(float);
  return (bytes + 255) & ~size_t(255);
}

extern "C" int cp_batch_check(const cp_batch_problem* p) {
  if (!p || p->N < 2 || p->N > BN || p->R < 1 || p->R > BR) return CP_EINVAL;
  int64_t mn = 0;
  for (int k = 0; k < p->N; ++k) {
    if (p->I[k] < 1) return CP_EINVAL;
    if (k > 0) mn += p->I[k] * p->R;
  }
  if (p->I[0] > BT || mn > 3 * 256 * BR) return CP_EINVAL;   // one row of M_1 per thread
  if (int64_t(p->N) * p->R * p->R > 1024) return CP_EINVAL;
  return CP_OK;
}

extern "C" int cp_batch_layout(cp_batch_problem* probs, int count, size_t* ws_bytes) {
  if (!probs || count < 0 || !ws_bytes) return CP_EINVAL;
  size_t off = 256;   // the first 256 bytes hold the work-queue counter
  for (int i = 0; i < count; ++i) {
    CP_TRY(cp_batch_check(&probs[i]));
    probs[i].ws_off = int64_t(off);
    off += batch_ws_one(probs[i]);
  }
  *ws_bytes = off;
  return CP_OK;
}

extern "C" int cp_batch_run(const cp_batch_problem* probs_dev, int count, const float* Y, double* a, void* ws,
                            cp_status* status, const cp_opts* opts, int trials, int ctas, int tile,
                            const int* order, void* stream) {
  if (!probs_dev || !Y || !a || !ws || !status || !opts || count < 0 || trials < 1) return CP_EINVAL;
  if (tile != 0 && tile != 8 && tile != 16 && tile != 32) return CP_EINVAL;
  if (count == 0) return CP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int grid = ctas > 0 ? ctas : kSMs;
  if (grid > count) grid = count;
  CP_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), s));
  switch (tile) {
    case 8: return batch_launch<8>(probs_dev, count, Y, a, ws, status, opts, trials, grid, order, s);
    case 32: return batch_launch<32>(probs_dev, count, Y, a, ws, status, opts, trials, grid, order, s);
    default: return batch_launch<16>(probs_dev, count, Y, a, ws, status, opts, trials, grid, order, s);
  }
}
