// Nearest-neighbour search kernels instantiated for one linkage (ward);
// the search itself is in hac_query.cuh.
#include "hac_query.cuh"

namespace hacg {

cudaError_t launch_query_ward(const QueryArgs &a, int dp, int prec, cudaStream_t s) {
  return prec == 0 ? launch_lk<LK_WARD, 0>(a, dp, s) : launch_lk<LK_WARD, 1>(a, dp, s);
}

}  // namespace hacg
