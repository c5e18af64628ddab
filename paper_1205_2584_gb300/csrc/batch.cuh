// Batched form: limits shared by the kernel and its host entry points, and
// the per-tile-width launcher (one translation unit per width).
#pragma once
#include "common.cuh"

namespace cpdgn {

constexpr int BT = 256;          // threads per CTA
constexpr int BN = 4;            // max order in the batched kernel
constexpr int BR = 16;           // max rank
constexpr int BRR = BR * BR;
constexpr int BNB = 32;          // Cholesky / triangular-solve block

// One persistent launch of k_batch_lm<TF> (TF = fibres per tensor tile).
template <int TF>
int batch_launch(const cp_batch_problem* probs_dev, int count, const float* Y, double* a, void* ws,
                 cp_status* status, const cp_opts* opts, int trials, int grid, const int* order,
                 cudaStream_t s);

}  // namespace cpdgn
