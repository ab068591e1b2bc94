// Instantiations of the Shouji filter for thresholds E = 24..27 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<24>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<25>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<26>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<27>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<24>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<25>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<26>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<27>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
