// Site-wise linear algebra and reductions on internal spinor fields
// (Sec. 3.2: copy, scale-and-add kernels and inner products / norms).
//
// The paper reduces with a site-wise kernel followed by a library reduction,
// two passes over global memory.  Here every reduction is fused into the
// kernel that produces its operand: each block folds its sites with warp
// shuffles into one FP64 partial, writes it, and the last block to finish
// (an atomic arrival counter per right-hand side) adds the partials in block
// order, so results are deterministic run to run.  That final step also
// derives the CG scalars (alpha = rr / pAp, beta = rr_new / rr) on the
// device, so a CG iteration needs no host round trip.
//
// Thread mapping: a fixed grid of `hr_blas_blocks` blocks x 256 threads per
// right-hand side, grid-striding over the V/2 sites of one parity; each site
// is processed colour by colour with the precision-specific chunk helpers.
#include <math.h>
#include <string.h>

#include "blas_dev.cuh"

int hr_blas_blocks(int64_t Vh) {
  int64_t nb = (Vh + 255) / 256;
  if (nb > HR_RED_MAXBLK) nb = HR_RED_MAXBLK;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// ---------------------------------------------------------------- kernels --
// grid: (blocks, nrhs * nsub); result slot = blockIdx.y / nsub; the parts of a
// slot are its nsub sub-fields x gridDim.x blocks.
#define SLOT_ARGS(nsub) (blockIdx.y / (nsub)), ((blockIdx.y % (nsub)) * gridDim.x + blockIdx.x), (gridDim.x * (nsub))
#define SITE_RANGE ((int64_t)blockIdx.x * blockDim.x + threadIdx.x), ((int64_t)gridDim.x * blockDim.x)

template <int P>
__global__ void norm2_kernel(const void *x, FieldDesc f, RedArgs red, int finish) {
  const char *base = reinterpret_cast<const char *>(x) + (size_t)blockIdx.y * f.fb;
  const double acc = norm2_sites<P>(base, f.Vh, f.d, SITE_RANGE);
  reduce_publish(acc, red, finish, SLOT_ARGS(f.nsub));
}

template <int PR, int PP>
__global__ void cg_xr_kernel(void *x, void *r, const void *p, const void *Ap, FieldDesc fr, FieldDesc fp,
                             RedArgs red) {
  typedef typename PT<PR>::A AR;
  const int rhs = blockIdx.y / fr.nsub;
  const AR al = (AR)red.alpha[rhs];
  double acc = 0.0;
  if (al != (AR)0)
    acc = cg_xr_sites<PR, PP>(reinterpret_cast<char *>(x) + (size_t)blockIdx.y * fr.fb,
                              reinterpret_cast<char *>(r) + (size_t)blockIdx.y * fr.fb,
                              reinterpret_cast<const char *>(p) + (size_t)blockIdx.y * fp.fb,
                              reinterpret_cast<const char *>(Ap) + (size_t)blockIdx.y * fp.fb, fr.Vh, fr.d, al,
                              SITE_RANGE);
  reduce_publish(acc, red, RED_BETA, SLOT_ARGS(fr.nsub));
}

template <int PR, int PP>
__global__ void cg_p_kernel(const void *r, void *p, FieldDesc fr, FieldDesc fp, const double *beta,
                            const double *alpha) {
  const int rhs = blockIdx.y / fr.nsub;
  if (alpha && alpha[rhs] == 0.0) return;  // frozen right-hand side
  cg_p_sites<PR, PP>(reinterpret_cast<const char *>(r) + (size_t)blockIdx.y * fr.fb,
                     reinterpret_cast<char *>(p) + (size_t)blockIdx.y * fp.fb, fr.Vh, fr.d,
                     (typename PT<PP>::A)beta[rhs], SITE_RANGE);
}

template <int PX, int PY>
__global__ void axpby_kernel(const void *x, void *y, FieldDesc fx, FieldDesc fy, const double *a, const double *b,
                             RedArgs red, int want_norm) {
  typedef typename PT<PY>::A AY;
  const int rhs = blockIdx.y / fx.nsub;
  const double acc = axpby_sites<PX, PY>(reinterpret_cast<const char *>(x) + (size_t)blockIdx.y * fx.fb,
                                         reinterpret_cast<char *>(y) + (size_t)blockIdx.y * fy.fb, fx.Vh, fx.d,
                                         (AY)a[rhs], (AY)b[rhs], SITE_RANGE);
  if (want_norm) reduce_publish(acc, red, RED_PLAIN, SLOT_ARGS(fx.nsub));
}

// ---------------------------------------------------------------- launchers
int hr_blas_norm2(const FieldDesc &f, int prec, const void *x, int nrhs, const RedArgs &red, int finish,
                  cudaStream_t s) {
  dim3 grid(hr_blas_blocks(f.Vh), nrhs * f.nsub);
  if (prec == HR_F64) norm2_kernel<0><<<grid, 256, 0, s>>>(x, f, red, finish);
  else if (prec == HR_FF) norm2_kernel<3><<<grid, 256, 0, s>>>(x, f, red, finish);
  else if (prec == HR_F32) norm2_kernel<1><<<grid, 256, 0, s>>>(x, f, red, finish);
  else norm2_kernel<2><<<grid, 256, 0, s>>>(x, f, red, finish);
  return hr_check_launch("norm2_kernel");
}

int hr_blas_cg_xr(int pr, int pp, void *x, void *r, const void *p, const void *Ap, const FieldDesc &fr,
                  const FieldDesc &fp, int nrhs, const RedArgs &red, cudaStream_t s) {
  dim3 grid(hr_blas_blocks(fr.Vh), nrhs * fr.nsub);
  if (pr == HR_F64 && pp == HR_F64) cg_xr_kernel<0, 0><<<grid, 256, 0, s>>>(x, r, p, Ap, fr, fp, red);
  else if (pr == HR_F32 && pp == HR_F32) cg_xr_kernel<1, 1><<<grid, 256, 0, s>>>(x, r, p, Ap, fr, fp, red);
  else if (pr == HR_F32 && pp == HR_F16) cg_xr_kernel<1, 2><<<grid, 256, 0, s>>>(x, r, p, Ap, fr, fp, red);
  else return HR_ERR_UNSUPPORTED;
  return hr_check_launch("cg_xr_kernel");
}

int hr_blas_cg_p(int pr, int pp, const void *r, void *p, const FieldDesc &fr, const FieldDesc &fp, int nrhs,
                 const double *beta, const double *alpha, cudaStream_t s) {
  dim3 grid(hr_blas_blocks(fr.Vh), nrhs * fr.nsub);
  if (pr == HR_F64 && pp == HR_F64) cg_p_kernel<0, 0><<<grid, 256, 0, s>>>(r, p, fr, fp, beta, alpha);
  else if (pr == HR_F32 && pp == HR_F32) cg_p_kernel<1, 1><<<grid, 256, 0, s>>>(r, p, fr, fp, beta, alpha);
  else if (pr == HR_F32 && pp == HR_F16) cg_p_kernel<1, 2><<<grid, 256, 0, s>>>(r, p, fr, fp, beta, alpha);
  else return HR_ERR_UNSUPPORTED;
  return hr_check_launch("cg_p_kernel");
}

int hr_blas_axpby(int px, int py, const void *x, void *y, const FieldDesc &fx, const FieldDesc &fy, int nrhs,
                  const double *a, const double *b, const RedArgs &red, int want_norm, cudaStream_t s) {
  dim3 grid(hr_blas_blocks(fx.Vh), nrhs * fx.nsub);
#define AXPBY(A, B) axpby_kernel<A, B><<<grid, 256, 0, s>>>(x, y, fx, fy, a, b, red, want_norm)
  if (px == 0 && py == 0) AXPBY(0, 0);
  else if (px == 0 && py == 1) AXPBY(0, 1);
  else if (px == 0 && py == 2) AXPBY(0, 2);
  else if (px == 1 && py == 0) AXPBY(1, 0);
  else if (px == 1 && py == 1) AXPBY(1, 1);
  else if (px == 1 && py == 2) AXPBY(1, 2);
  else if (px == 2 && py == 0) AXPBY(2, 0);
  else if (px == 2 && py == 1) AXPBY(2, 1);
  else if (px == 2 && py == 2) AXPBY(2, 2);
  // float-float: conversions from / to FP64 and FP32, and updates
  else if (px == 0 && py == 3) AXPBY(0, 3);
  else if (px == 3 && py == 0) AXPBY(3, 0);
  else if (px == 1 && py == 3) AXPBY(1, 3);
  else if (px == 3 && py == 1) AXPBY(3, 1);
  else if (px == 3 && py == 3) AXPBY(3, 3);
  else return HR_ERR_UNSUPPORTED;
#undef AXPBY
  return hr_check_launch("axpby_kernel");
}

// ------------------------------------------------------------ public norm2 --
int hr_red_scratch(hr_lattice *lat, int nrhs) {
  (void)nrhs;
  if (!lat->red_partials) {
    HR_CUDA(cudaMalloc(&lat->red_partials, sizeof(double) * 2 * HR_RED_MAXBLK * HR_MAX_RHS));
    HR_CUDA(cudaMalloc(&lat->red_count, sizeof(unsigned) * HR_MAX_RHS));
    HR_CUDA(cudaMemset(lat->red_count, 0, sizeof(unsigned) * HR_MAX_RHS));
    // red_out: [HR_MAX_RHS] results, then the a and b coefficients of hr_axpby
    HR_CUDA(cudaMalloc(&lat->red_out, sizeof(double) * 3 * HR_MAX_RHS));
    HR_CUDA(cudaMallocHost(&lat->red_out_host, sizeof(double) * HR_MAX_RHS));
  }
  return HR_OK;
}

extern "C" int hr_norm2(hr_lattice *lat, const void *x, int parity, int prec, int nrhs, double *out_host) {
  if (!lat || !x || !out_host || nrhs < 1 || nrhs > HR_MAX_RHS || prec < HR_F64 || prec > HR_F16 ||
      parity < HR_EVEN || parity > HR_FULL)
    return HR_ERR_ARG;
  HR_TRY(hr_red_scratch(lat, nrhs));
  const size_t fb = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  FieldDesc f;
  f.Vh = lat->Vh;
  f.d = lat->d;
  f.fb = fb;
  f.nsub = parity == HR_FULL ? 2 : 1;
  RedArgs red;
  memset(&red, 0, sizeof(red));
  red.partials = lat->red_partials;
  red.count = lat->red_count;
  red.out = lat->red_out;
  red.err = lat->dev_err;
  HR_TRY(hr_blas_norm2(f, prec, x, nrhs, red, RED_PLAIN, lat->stream));
  HR_CUDA(cudaMemcpyAsync(lat->red_out_host, lat->red_out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost,
                          lat->stream));
  HR_CUDA(cudaStreamSynchronize(lat->stream));
  for (int r = 0; r < nrhs; ++r) out_host[r] = lat->red_out_host[r];
  return HR_OK;
}

extern "C" int hr_axpby(hr_lattice *lat, const void *x, void *y, const double *a, const double *b, int parity,
                        int prec, int nrhs) {
  if (!lat || !x || !y || !a || !b || nrhs < 1 || nrhs > HR_MAX_RHS || prec < HR_F64 || prec > HR_F16 ||
      parity < HR_EVEN || parity > HR_FULL)
    return HR_ERR_ARG;
  HR_TRY(hr_red_scratch(lat, nrhs));
  // the coefficients go to the device through a pageable copy, which has
  // taken them from the caller's arrays by the time it returns
  double coef[2 * HR_MAX_RHS];
  for (int r = 0; r < nrhs; ++r) {
    coef[r] = a[r];
    coef[HR_MAX_RHS + r] = b[r];
  }
  double *ad = lat->red_out + HR_MAX_RHS, *bd = lat->red_out + 2 * HR_MAX_RHS;
  HR_CUDA(cudaMemcpyAsync(ad, coef, sizeof(double) * 2 * HR_MAX_RHS, cudaMemcpyHostToDevice, lat->stream));
  FieldDesc f;
  f.Vh = lat->Vh;
  f.d = lat->d;
  f.fb = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  f.nsub = parity == HR_FULL ? 2 : 1;
  RedArgs red;
  memset(&red, 0, sizeof(red));
  return hr_blas_axpby(prec, prec, x, y, f, f, nrhs, ad, bd, red, 0, lat->stream);
}
