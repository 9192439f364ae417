// Big-pair evaluation kernels instantiated for complete linkage (a
// translation unit of its own so the two linkages compile in parallel).
#include "hac_big.cuh"

namespace hacg {

int launch_big_complete(const State &s, int r0, cudaStream_t st) {
  return launch_big_lk<0>(s, r0, st);
}

}  // namespace hacg
