// re_batched_mix_async.cu -- mixed-precision instantiations of the batched MD kernel,
// master-stop and free-running modes (exchanges inside the launch).
#include "re_batched.cuh"

namespace re {
template cudaError_t launch_batched_t<false, 1, false, 1, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 1, false, 2, 1024>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<false, 1, false, 1024>(const LaunchCfg&, int, int, size_t);
template cudaError_t launch_batched_t<false, 2, false, 1, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 2, false, 2, 1024>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<false, 2, false, 1024>(const LaunchCfg&, int, int, size_t);
template cudaError_t launch_batched_t<false, 4, false, 1, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 4, false, 2, 1024>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<false, 4, false, 1024>(const LaunchCfg&, int, int, size_t);
template cudaError_t launch_batched_t<false, 8, false, 1, 1024>(BATCHED_LAUNCH_ARGS);
template cudaError_t launch_batched_t<false, 8, false, 2, 1024>(BATCHED_LAUNCH_ARGS);
template int max_active_clusters_t<false, 8, false, 1024>(const LaunchCfg&, int, int, size_t);
}  // namespace re
