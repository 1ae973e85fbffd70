// FP64 instantiations of the hopping kernels: one site per thread for
// d_R <= 8 (hop.cuh), colour-split groups for the large representations
// (hop_split.cuh).
#include "hop_split.cuh"

int hr_launch_hop_f64(const hr_lattice *lat, const HopArgs &a, cudaStream_t s) {
  const int d = lat->d;
  if (d <= 8) return hop_dispatch<0>(lat, a, s);
  if (a.clover) return HR_ERR_UNSUPPORTED;
  const HopK k = make_hopk(lat, a);
  if (lat->is_real) {
    switch (d) {
      case 15: return launch_split<15, true, 0, 4>(k, a.nrhs, s);
      case 24: return launch_split<24, true, 0, 8>(k, a.nrhs, s);
      case 35: return launch_split<35, true, 0, 8>(k, a.nrhs, s);
    }
  } else {
    switch (d) {
      case 10: return launch_split<10, false, 0, 2>(k, a.nrhs, s);
      case 15: return launch_split<15, false, 0, 4>(k, a.nrhs, s);
      case 21: return launch_split<21, false, 0, 4>(k, a.nrhs, s);
    }
  }
  return HR_ERR_UNSUPPORTED;
}
