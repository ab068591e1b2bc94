// Instantiations of the Shouji filter for thresholds E = 4..7 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<4>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<5>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<6>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<7>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<4>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<5>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<6>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<7>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
