// Instantiations of the Shouji filter for thresholds E = 12..15 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<12>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<13>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<14>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<15>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<12>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<13>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<14>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<15>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
