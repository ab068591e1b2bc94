// Instantiations of the Shouji filter for thresholds E = 8..11 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<8>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<9>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<10>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<11>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<8>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<9>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<10>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<11>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
