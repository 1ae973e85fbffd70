// FP32 instantiations of the site-per-thread hopping kernel (hop.cuh).
#include "hop.cuh"

int hr_launch_hop_f32(const hr_lattice *lat, const HopArgs &a, cudaStream_t s) { return hop_dispatch<1>(lat, a, s); }
