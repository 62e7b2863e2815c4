// re_batched_mix.cu -- mixed-precision instantiations of the batched MD kernel,
// per-replica step budgets (lists in global or in shared memory).
#include "re_batched.cuh"

namespace re {
template cudaError_t launch_batched_t<false, 1, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 1, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 2, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 2, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 4, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 4, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 8, false, 0, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 8, true, 0, 1024>(BATCHED_LAUNCH_ARGS);
}  // namespace re
