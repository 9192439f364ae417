// Nearest-neighbour search kernels instantiated for one linkage (average);
// the search itself is in hac_query.cuh.
#include "hac_query.cuh"

namespace hacg {

cudaError_t launch_query_average(const QueryArgs &a, int dp, int prec, cudaStream_t s) {
  return prec == 0 ? launch_lk<LK_AVERAGE, 0>(a, dp, s) : launch_lk<LK_AVERAGE, 1>(a, dp, s);
}

}  // namespace hacg
