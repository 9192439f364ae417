// Dispatch of the nearest-neighbour search (Algorithms 2-4) by linkage; the
// kernels are in hac_query.cuh, instantiated per linkage in
// hac_query_<linkage>.cu.
#include "hac_query.cuh"

namespace hacg {

cudaError_t launch_query(const QueryArgs &a, int dp, int prec, cudaStream_t s) {
  if (a.nterm <= 0) return cudaSuccess;
  switch (a.linkage) {
    case LK_COMPLETE: return launch_query_complete(a, dp, prec, s);
    case LK_AVERAGE: return launch_query_average(a, dp, prec, s);
    case LK_WARD: return launch_query_ward(a, dp, prec, s);
    case LK_AVG2: return launch_query_avg2(a, dp, prec, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hacg
