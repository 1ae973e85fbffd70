// FP16 instantiations of the site-per-thread hopping kernel (hop.cuh).
#include "hop.cuh"

int hr_launch_hop_f16(const hr_lattice *lat, const HopArgs &a, cudaStream_t s) { return hop_dispatch<2>(lat, a, s); }
