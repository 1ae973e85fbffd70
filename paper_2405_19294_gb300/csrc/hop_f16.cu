// FP16 instantiations of the hopping kernels: one site per thread for
// d_R <= 8 (hop.cuh), its multi-right-hand-side form (hop_mrhs.cuh) and
// colour-split groups (hop_split.cuh) for d_R >= 6;
// the autotuner in tune.cu chooses among the shapes listed by hr_hop_shapes.
#include "hop_mrhs.cuh"
#include "hop_rows.cuh"
#include "hop_split.cuh"

int hr_launch_hop_f16(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh) {
  const int d = lat->d;
  if (sh.mrhs >= HR_TC_MRHS) return hr_launch_hop_tc_f16(lat, a, s);
  if (sh.mrhs > 0) return hop_mrhs_dispatch<2>(lat, a, s, sh.mrhs);
  if (sh.rows > 0) return rows_dispatch<2>(lat, a, s, sh.rows);
  if (sh.split_g == 0) return hop_dispatch<2>(lat, a, s, sh.bs, sh.regs);
  if (a.clover) return HR_ERR_UNSUPPORTED;
  const HopK k = make_hopk(lat, a);
  const int g = sh.split_g;
  const bool real = lat->is_real != 0;
#define HR_SPLIT_CASE(DD, RE, GG) \
  if (d == DD && real == RE && g == GG) return launch_split<DD, RE, 2, GG>(k, make_skipk(a), a.nrhs, s);
  HR_SPLIT_SHAPES(HR_SPLIT_CASE)
#undef HR_SPLIT_CASE
  return HR_ERR_UNSUPPORTED;
}

int hr_launch_hop_multi_f16(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                            const int *frozen, cudaStream_t s) {
  return hop_multi_launch<2>(d, is_real, sh, descs, items, nitems, frozen, s);
}
