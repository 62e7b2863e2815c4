// re_batched_mix_narrow.cu -- mixed-precision instantiations of the batched MD kernel,
// per-replica step budgets (lists in global or in shared memory).
// CTAs of at most kNarrowThreads threads (72 registers per thread).
#include "re_batched.cuh"

namespace re {
template cudaError_t launch_batched_t<false, 1, false, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 1, true, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 2, false, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 2, true, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 4, false, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 4, true, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 8, false, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 8, true, 0, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
}  // namespace re
