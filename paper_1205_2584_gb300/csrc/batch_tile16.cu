// The batched kernel for tensor tiles of 16 fibres.
#include "batch_kernel.cuh"

namespace cpdgn {
template int batch_launch<16>(const cp_batch_problem*, int, const float*, double*, void*, cp_status*,
                                const cp_opts*, int, int, const int*, cudaStream_t);
}  // namespace cpdgn
