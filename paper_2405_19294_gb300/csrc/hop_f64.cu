// FP64 instantiations of the hopping kernels: one site per thread for
// d_R <= 8 (hop.cuh), its multi-right-hand-side form (hop_mrhs.cuh) and
// colour-split groups (hop_split.cuh) for d_R >= 6;
// the autotuner in tune.cu chooses among the shapes listed by hr_hop_shapes.
#include "hop_mrhs.cuh"
#include "hop_rows.cuh"
#include "hop_split.cuh"

int hr_launch_hop_f64(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh) {
  const int d = lat->d;
  if (sh.mrhs > 0) return hop_mrhs_dispatch<0>(lat, a, s, sh.mrhs);
  if (sh.rows > 0) return rows_dispatch<0>(lat, a, s, sh.rows);
  if (sh.split_g == 0) return hop_dispatch<0>(lat, a, s, sh.bs, sh.regs);
  if (a.clover) return HR_ERR_UNSUPPORTED;
  const HopK k = make_hopk(lat, a);
  const int g = sh.split_g;
  if (lat->is_real) {
    if (d == 8 && g == 2) return launch_split<8, true, 0, 2>(k, a.nrhs, s);
    if (d == 8 && g == 4) return launch_split<8, true, 0, 4>(k, a.nrhs, s);
    if (d == 15 && g == 4) return launch_split<15, true, 0, 4>(k, a.nrhs, s);
    if (d == 15 && g == 8) return launch_split<15, true, 0, 8>(k, a.nrhs, s);
    if (d == 24 && g == 8) return launch_split<24, true, 0, 8>(k, a.nrhs, s);
    if (d == 24 && g == 16) return launch_split<24, true, 0, 16>(k, a.nrhs, s);
    if (d == 35 && g == 8) return launch_split<35, true, 0, 8>(k, a.nrhs, s);
    if (d == 35 && g == 16) return launch_split<35, true, 0, 16>(k, a.nrhs, s);
  } else {
    if (d == 6 && g == 2) return launch_split<6, false, 0, 2>(k, a.nrhs, s);
    if (d == 10 && g == 2) return launch_split<10, false, 0, 2>(k, a.nrhs, s);
    if (d == 10 && g == 4) return launch_split<10, false, 0, 4>(k, a.nrhs, s);
    if (d == 15 && g == 4) return launch_split<15, false, 0, 4>(k, a.nrhs, s);
    if (d == 15 && g == 8) return launch_split<15, false, 0, 8>(k, a.nrhs, s);
    if (d == 21 && g == 4) return launch_split<21, false, 0, 4>(k, a.nrhs, s);
    if (d == 21 && g == 8) return launch_split<21, false, 0, 8>(k, a.nrhs, s);
  }
  return HR_ERR_UNSUPPORTED;
}

int hr_launch_hop_multi_f64(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                            const int *frozen, cudaStream_t s) {
  return hop_multi_launch<0>(d, is_real, sh, descs, items, nitems, frozen, s);
}
