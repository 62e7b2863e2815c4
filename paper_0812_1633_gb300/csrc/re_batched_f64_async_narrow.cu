// re_batched_f64_async_narrow.cu -- FP64 instantiations of the batched MD kernel,
// master-stop and free-running modes (exchanges inside the launch).
// CTAs of at most kNarrowThreads threads (72 registers per thread).
#include "re_batched.cuh"

namespace re {
template cudaError_t launch_batched_t<true, 1, false, 1, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 1, false, 2, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<true, 1, false, kNarrowThreads>(const LaunchCfg&, int, int, size_t);
template cudaError_t launch_batched_t<true, 2, false, 1, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 2, false, 2, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<true, 2, false, kNarrowThreads>(const LaunchCfg&, int, int, size_t);
template cudaError_t launch_batched_t<true, 4, false, 1, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 4, false, 2, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<true, 4, false, kNarrowThreads>(const LaunchCfg&, int, int, size_t);
template cudaError_t launch_batched_t<true, 8, false, 1, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<true, 8, false, 2, kNarrowThreads>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<true, 8, false, kNarrowThreads>(const LaunchCfg&, int, int, size_t);
}  // namespace re
