// FP16 instantiations of the tensor-core multi-right-hand-side hopping
// kernel (hop_tc.cuh), in a translation unit of their own so that they compile
// in parallel with the other stencils.
#include "hop_tc.cuh"

int hr_launch_hop_tc_f16(const hr_lattice *lat, const HopArgs &a, cudaStream_t s) {
  return hop_tc_dispatch<2>(lat, a, s);
}
