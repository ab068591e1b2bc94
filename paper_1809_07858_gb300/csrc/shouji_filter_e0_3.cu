// Instantiations of the Shouji filter for thresholds E = 0..3 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<0>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<1>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<2>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<3>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<0>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<1>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<2>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<3>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
