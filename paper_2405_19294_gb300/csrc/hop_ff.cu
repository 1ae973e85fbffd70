// Float-float operator: the conversions that give it its links and clover
// blocks, and the dispatch over the per-class instantiations (hop_ff_*.cu) of
// its one-site-per-thread hopping kernel (hop_ff.cuh), d_R <= 8, and of the
// rows kernel (hop_rows.cuh) for the larger representations.
//
// The float-float operator is the FP64-accurate Dhat of the mixed solvers'
// outer residuals (Sec. 3.3): the FP64 kernel's stencil with every real a pair
// of FP32 numbers (cplx.cuh), about 48 significant bits.  Its links and clover
// blocks are float-float copies of the FP64 ones, made once per gauge field
// (and per m0 for the clover blocks).
#include "hop_ff.cuh"

// out[j] = (h, l) with h + l = in[j] to 48 bits
__global__ void f64_to_ff_kernel(float2 *out, const double *in, size_t n) {
  for (size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const ff v(in[j]);
    out[j] = make_float2(v.h, v.l);
  }
}

int hr_f64_to_ff(void *out, const void *in, size_t nreal, cudaStream_t s) {
  if (nreal == 0) return HR_OK;
  const size_t nb = (nreal + 255) / 256;
  const unsigned grid = (unsigned)(nb < 4096 ? nb : 4096);
  f64_to_ff_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<float2 *>(out), reinterpret_cast<const double *>(in), nreal);
  return hr_check_launch("f64_to_ff_kernel");
}

int hr_ff_prepare(hr_lattice *lat, int clover, double m0, cudaStream_t st) {
  if (!lat->ff_links_ok) {
    // the FP64 links were made on the lattice's stream, which was synchronised
    const size_t nreal = (size_t)2 * 4 * lat->nch_link * (size_t)lat->Vh * 2;
    if (!lat->links[HR_FF]) HR_TRY(hr_dev_alloc(&lat->links[HR_FF], nreal * 8));
    HR_TRY(hr_f64_to_ff(lat->links[HR_FF], lat->links[HR_F64], nreal, st));
    if (lat->rlinks[HR_F64]) {  // the rows kernel's layout, slack rows included
      const size_t nr = ((size_t)16 * hr_rows_nch(lat->d, lat->is_real) + HR_ROWS_SLACK) * (size_t)lat->Vh * 2;
      if (!lat->rlinks[HR_FF]) HR_TRY(hr_dev_alloc(&lat->rlinks[HR_FF], nr * 8));
      HR_TRY(hr_f64_to_ff(lat->rlinks[HR_FF], lat->rlinks[HR_F64], nr, st));
    }
    lat->ff_links_ok = 1;
  }
  if (clover) {
    HR_TRY(hr_clover_prepare(lat, m0));
    if (!lat->clover_ff_ok) {
      // the FP64 blocks may still be in flight on the lattice's stream
      HrEvent ev;
      HR_CUDA(cudaEventCreateWithFlags(&ev.e, cudaEventDisableTiming));
      HR_CUDA(cudaEventRecord(ev.e, lat->stream));
      HR_CUDA(cudaStreamWaitEvent(st, ev.e, 0));
      const size_t nreal = (size_t)2 * 4 * lat->d * lat->d * (size_t)lat->Vh * 2;
      if (!lat->clover_A[2]) HR_TRY(hr_dev_alloc(&lat->clover_A[2], nreal * 8));
      if (!lat->clover_Ainv[2]) HR_TRY(hr_dev_alloc(&lat->clover_Ainv[2], nreal * 8));
      HR_TRY(hr_f64_to_ff(lat->clover_A[2], lat->clover_A[0], nreal, st));
      HR_TRY(hr_f64_to_ff(lat->clover_Ainv[2], lat->clover_Ainv[0], nreal, st));
      lat->clover_ff_ok = 1;
    }
  }
  return HR_OK;
}

int hr_ff_outer_usable(hr_lattice *lat, int clover, double m0, int nrhs, cudaStream_t st, int *use) {
  *use = 0;
  HopShape sh[HR_MAX_SHAPES];
  if (lat->dom || hr_hop_shapes(lat->d, lat->is_real, HR_FF, clover, nrhs > 1, sh) < 1) return HR_OK;
  const int rc = hr_ff_prepare(lat, clover, m0, st);
  if (rc == HR_ERR_NOMEM) {  // no room for the float-float copies: the solver keeps FP64
    cudaGetLastError();
    return HR_OK;
  }
  HR_TRY(rc);
  *use = 1;
  return HR_OK;
}

#define HR_FF_CLASS(DD, RE, NAME)                                   \
  void NAME(const HopK &, SkipK, dim3, int, int, cudaStream_t, int); \
  const void *NAME##_multi();                                        \
  size_t NAME##_smem(int bs);
HR_FF_CLASSES(HR_FF_CLASS)
#undef HR_FF_CLASS
const void *hr_ff_rows_multi(int d, int is_real, int rows, int *block, size_t *smem);

// Persistent multi-lattice launch (grid = min(work items, SMs x resident
// blocks)): the site kernel of the class, or the rows kernel.
int hr_launch_hop_multi_ff(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                           const int *frozen, cudaStream_t s) {
  int block = sh.bs;
  size_t smem = 0;
  const void *fn = nullptr;
  if (sh.rows) {
    fn = hr_ff_rows_multi(d, is_real, sh.rows, &block, &smem);
  } else if (!sh.split_g && !sh.mrhs) {
    const bool real = is_real != 0;
#define HR_FF_CLASS(DD, RE, NAME) \
  if (d == DD && real == RE) {    \
    fn = NAME##_multi();          \
    smem = NAME##_smem(block);    \
  }
    HR_FF_CLASSES(HR_FF_CLASS)
#undef HR_FF_CLASS
  }
  if (!fn) return HR_ERR_UNSUPPORTED;
  if (nitems <= 0) return HR_OK;
  int dev = 0, sms = 0, per_sm = 0;
  HR_CUDA(cudaGetDevice(&dev));
  HR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem));
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > nitems) grid = nitems;
  void *args[] = {(void *)&descs, (void *)&items, (void *)&nitems, (void *)&frozen};
  HR_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s));
  return HR_OK;
}

int hr_launch_hop_ff_rows(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, int rows);

int hr_launch_hop_ff(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh) {
  if (sh.rows && !sh.mrhs && !sh.split_g && !a.tmask) return hr_launch_hop_ff_rows(lat, a, s, sh.rows);
  if (sh.mrhs || sh.rows || sh.split_g || a.tmask || (sh.regs != 0 && sh.regs != 1)) return HR_ERR_UNSUPPORTED;
  const HopK k = make_hopk(lat, a);
  const SkipK sk = make_skipk(a);
  const int bs = sh.bs;
  dim3 grid((unsigned)(((lat->Vh + bs - 1) / bs) * a.nrhs));
  const bool real = lat->is_real != 0;
#define HR_FF_CLASS(DD, RE, NAME)             \
  if (lat->d == DD && real == RE) {           \
    NAME(k, sk, grid, bs, sh.regs, s, a.pdl); \
    return hr_check_launch("hop_kernel");     \
  }
  HR_FF_CLASSES(HR_FF_CLASS)
#undef HR_FF_CLASS
  return HR_ERR_UNSUPPORTED;
}
