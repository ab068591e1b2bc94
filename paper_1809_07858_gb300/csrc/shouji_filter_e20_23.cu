// Instantiations of the Shouji filter for thresholds E = 20..23 (one
// translation unit per range so that the build compiles them in parallel).
#include "shouji_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<20>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<21>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<22>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<23>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<20>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<21>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<22>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<23>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
