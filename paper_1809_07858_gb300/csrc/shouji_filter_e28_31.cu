// Instantiations of the Shouji filter for thresholds E = 28..31 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<28>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<29>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<30>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<31>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<28>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<29>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<30>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<31>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
