// Big-pair evaluation kernels instantiated for average linkage (a
// translation unit of its own so the two linkages compile in parallel).
#include "hac_big.cuh"

namespace hacg {

int launch_big_average(const State &s, int r0, cudaStream_t st) {
  return launch_big_lk<1>(s, r0, st);
}

}  // namespace hacg
