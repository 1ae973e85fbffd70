// Float-float instantiations of the rows kernel (hop_rows.cuh): the outer
// residuals of the mixed solvers for d_R >= 6 without clover.
#include "hop_rows.cuh"

int hr_launch_hop_ff_rows(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, int rows) {
  return rows_dispatch<3>(lat, a, s, rows);
}
