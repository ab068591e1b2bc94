// Instantiations of the Shouji filter for thresholds E = 16..19 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<16>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<17>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<18>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<19>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<16>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<17>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<18>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<19>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
