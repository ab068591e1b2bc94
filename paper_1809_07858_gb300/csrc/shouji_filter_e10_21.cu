// Instantiations of the Shouji filter for thresholds E = 10 and 21 (one
// translation unit per pair of thresholds of about equal total cost, so
// that the build compiles them in parallel).
#include "shouji_filter.cuh"
#include "shouji_batch_filter.cuh"

namespace shouji {
template cudaError_t launch_filter_E<10>(const FilterArgs &, cudaStream_t);
template cudaError_t launch_filter_E<21>(const FilterArgs &, cudaStream_t);
template cudaError_t batch::launch_filter_E<10>(const batch::FilterParams &, int, int, cudaStream_t);
template cudaError_t batch::launch_filter_E<21>(const batch::FilterParams &, int, int, cudaStream_t);
}  // namespace shouji
