// re_batched_f64.cu -- FP64 instantiations of the batched MD kernel,
// per-replica step budgets (lists in global or in shared memory).
#include "re_batched.cuh"

namespace re {
template cudaError_t launch_batched_t<true, 1, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 1, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 2, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 2, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 4, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 4, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 8, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 8, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
}  // namespace re
