// Float-float instantiations of the rows kernel (hop_rows.cuh): the outer
// residuals of the mixed solvers for d_R >= 6 without clover.
#include "hop_rows.cuh"

int hr_launch_hop_ff_rows(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, int rows) {
  return rows_dispatch<3>(lat, a, s, rows);
}

// the multi-lattice rows kernel (batched solver) and its block and shared memory
const void *hr_ff_rows_multi(int d, int is_real, int rows, int *block, size_t *smem) {
  return rows_multi_ptr<3>(d, is_real, rows, block, smem);
}
