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

#include "blas.cuh"
#include "cplx.cuh"
#include "hr_internal.h"

int hr_blas_blocks(int64_t Vh) {
  int64_t nb = (Vh + 255) / 256;
  if (nb > HR_RED_MAXBLK) nb = HR_RED_MAXBLK;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// block-wide FP64 sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = (l < nw) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Publish this block's partial; the last block of this rhs sums all partials in
// block order and applies `finish`.  Returns nothing; writes red.out[rhs].
__device__ void reduce_publish(double v, const RedArgs &red, int finish, int nsub) {
  const int rhs = blockIdx.y / nsub;
  const int nparts = gridDim.x * nsub;
  double s = block_sum(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    red.partials[(size_t)rhs * 2 * HR_RED_MAXBLK + (blockIdx.y % nsub) * gridDim.x + blockIdx.x] = s;
    __threadfence();
    const unsigned prev = atomicAdd(&red.count[rhs], 1u);
    last = (prev == (unsigned)nparts - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order sum of the partials by one warp
  double t = 0.0;
  if (threadIdx.x < 32) {
    for (int b = threadIdx.x; b < nparts; b += 32)
      t += ((volatile double *)red.partials)[(size_t)rhs * 2 * HR_RED_MAXBLK + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  if (threadIdx.x == 0) {
    red.out[rhs] = t;
    red.count[rhs] = 0u;
    if (finish == RED_ALPHA) {
      // alpha = rr / pAp, frozen (0) once rr reached the stop threshold or on breakdown
      const double rr = red.rr[rhs];
      double al = 0.0;
      if (rr > red.stop[rhs]) {
        if (t > 0.0 && isfinite(t)) al = rr / t;
        else atomicExch(red.err, 1);
      }
      red.alpha[rhs] = al;
      if (red.iters && al != 0.0) red.iters[rhs] += 1;
    } else if (finish == RED_BETA) {
      const double rr = red.rr[rhs];
      red.beta[rhs] = (rr > 0.0 && red.alpha[rhs] != 0.0) ? t / rr : 0.0;
      red.rr_next[rhs] = (red.alpha[rhs] != 0.0) ? t : rr;
    }
  }
}

// ---------------------------------------------------------------- kernels --
template <int P>
__global__ void norm2_kernel(const void *x, FieldDesc f, RedArgs red, int finish) {
  typedef typename PT<P>::A A;
  const char *base = reinterpret_cast<const char *>(x) + (size_t)blockIdx.y * f.fb;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f.Vh; i += (int64_t)gridDim.x * blockDim.x) {
    A s = 0;
    for (int c = 0; c < f.d; ++c) {
      cx<A> v[4];
      ld_colour<P>(base, f.Vh, i, c, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) s += v[q].x * v[q].x + v[q].y * v[q].y;
    }
    double sd = (double)s;
    if (P == 2) {
      const double sc = (double)f16_scales(base, f.Vh, f.d)[i];
      sd *= sc * sc;
    }
    acc += sd;
  }
  reduce_publish(acc, red, finish, f.nsub);
}

// load colour c of site i (FP16 scaled back)
template <int P>
__device__ __forceinline__ void ldc(const char *f, int64_t Vh, int d, int64_t i, int c,
                                    cx<typename PT<P>::A> v[4]) {
  ld_colour<P>(f, Vh, i, c, v);
  if (P == 2) {
    const float s = f16_scales(f, Vh, d)[i];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = scale((typename PT<P>::A)s, v[q]);
  }
}

// store colour c (FP16: divided by the given site scale, `inv` = 1/scale)
template <int P>
__device__ __forceinline__ void stc(char *f, int64_t Vh, int64_t i, int c, const cx<typename PT<P>::A> v[4],
                                    float inv) {
  if (P == 0) st_colour64(f, Vh, i, c, reinterpret_cast<const cx<double> *>(v));
  else if (P == 1) st_colour32(f, Vh, i, c, reinterpret_cast<const cx<float> *>(v));
  else {
    cx<float> w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = mk((float)v[q].x * inv, (float)v[q].y * inv);
    st_colour16(f, Vh, i, c, w);
  }
}

// x += alpha p ; r -= alpha Ap ; rr_new = |r|^2   (x, r: precision PR; p, Ap: PP)
template <int PR, int PP>
__global__ void cg_xr_kernel(void *x, void *r, const void *p, const void *Ap, FieldDesc fr, FieldDesc fp,
                             RedArgs red) {
  typedef typename PT<PR>::A AR;
  const int rhs = blockIdx.y / fr.nsub;
  char *xb = reinterpret_cast<char *>(x) + (size_t)blockIdx.y * fr.fb;
  char *rb = reinterpret_cast<char *>(r) + (size_t)blockIdx.y * fr.fb;
  const char *pb = reinterpret_cast<const char *>(p) + (size_t)blockIdx.y * fp.fb;
  const char *ab = reinterpret_cast<const char *>(Ap) + (size_t)blockIdx.y * fp.fb;
  const AR al = (AR)red.alpha[rhs];
  double acc = 0.0;
  if (al != (AR)0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fr.Vh;
         i += (int64_t)gridDim.x * blockDim.x) {
      AR s = 0;
      for (int c = 0; c < fr.d; ++c) {
        cx<AR> xv[4], rv[4];
        cx<typename PT<PP>::A> pv[4], av[4];
        ldc<PR>(xb, fr.Vh, fr.d, i, c, xv);
        ldc<PR>(rb, fr.Vh, fr.d, i, c, rv);
        ldc<PP>(pb, fp.Vh, fp.d, i, c, pv);
        ldc<PP>(ab, fp.Vh, fp.d, i, c, av);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xv[q] = mk(fma(al, (AR)pv[q].x, xv[q].x), fma(al, (AR)pv[q].y, xv[q].y));
          rv[q] = mk(fma(-al, (AR)av[q].x, rv[q].x), fma(-al, (AR)av[q].y, rv[q].y));
          s += rv[q].x * rv[q].x + rv[q].y * rv[q].y;
        }
        stc<PR>(xb, fr.Vh, i, c, xv, 1.f);
        stc<PR>(rb, fr.Vh, i, c, rv, 1.f);
      }
      acc += (double)s;
    }
  }
  reduce_publish(acc, red, RED_BETA, fr.nsub);
}

// p = r + beta p   (r: PR, p: PP)
template <int PR, int PP>
__global__ void cg_p_kernel(const void *r, void *p, FieldDesc fr, FieldDesc fp, const double *beta,
                            const double *alpha) {
  typedef typename PT<PP>::A AP;
  const int rhs = blockIdx.y / fr.nsub;
  if (alpha && alpha[rhs] == 0.0) return;  // frozen right-hand side
  const char *rb = reinterpret_cast<const char *>(r) + (size_t)blockIdx.y * fr.fb;
  char *pb = reinterpret_cast<char *>(p) + (size_t)blockIdx.y * fp.fb;
  const AP be = (AP)beta[rhs];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fr.Vh; i += (int64_t)gridDim.x * blockDim.x) {
    float inv = 1.f;
    if (PP == 2) {  // first pass: the new site maximum
      float m = 0.f;
      for (int c = 0; c < fr.d; ++c) {
        cx<typename PT<PR>::A> rv[4];
        cx<AP> pv[4];
        ldc<PR>(rb, fr.Vh, fr.d, i, c, rv);
        ldc<PP>(pb, fp.Vh, fp.d, i, c, pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          m = fmaxf(m, fabsf((float)fma(be, pv[q].x, (AP)rv[q].x)));
          m = fmaxf(m, fabsf((float)fma(be, pv[q].y, (AP)rv[q].y)));
        }
      }
      inv = m > 0.f ? 1.f / m : 0.f;
      // second pass below reads the old p again before overwriting it, so the
      // scale is written last
      for (int c = 0; c < fr.d; ++c) {
        cx<typename PT<PR>::A> rv[4];
        cx<AP> pv[4];
        ldc<PR>(rb, fr.Vh, fr.d, i, c, rv);
        ldc<PP>(pb, fp.Vh, fp.d, i, c, pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) pv[q] = mk(fma(be, pv[q].x, (AP)rv[q].x), fma(be, pv[q].y, (AP)rv[q].y));
        stc<PP>(pb, fp.Vh, i, c, pv, inv);
      }
      f16_scales_w(pb, fp.Vh, fp.d)[i] = m;
    } else {
      for (int c = 0; c < fr.d; ++c) {
        cx<typename PT<PR>::A> rv[4];
        cx<AP> pv[4];
        ldc<PR>(rb, fr.Vh, fr.d, i, c, rv);
        ldc<PP>(pb, fp.Vh, fp.d, i, c, pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) pv[q] = mk(fma(be, pv[q].x, (AP)rv[q].x), fma(be, pv[q].y, (AP)rv[q].y));
        stc<PP>(pb, fp.Vh, i, c, pv, inv);
      }
    }
  }
}

// y = a * x + b * y   with per-rhs a, b (host scalars in arrays), precisions PX -> PY;
// b == 0 overwrites y (y may hold anything).  Optional |y|^2 reduction.
template <int PX, int PY>
__global__ void axpby_kernel(const void *x, void *y, FieldDesc fx, FieldDesc fy, const double *a, const double *b,
                             RedArgs red, int want_norm) {
  typedef typename PT<PY>::A AY;
  const int rhs = blockIdx.y / fx.nsub;
  const char *xb = reinterpret_cast<const char *>(x) + (size_t)blockIdx.y * fx.fb;
  char *yb = reinterpret_cast<char *>(y) + (size_t)blockIdx.y * fy.fb;
  const AY av = (AY)a[rhs], bv = (AY)b[rhs];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fx.Vh; i += (int64_t)gridDim.x * blockDim.x) {
    float inv = 1.f;
    if (PY == 2) {
      float m = 0.f;
      for (int c = 0; c < fx.d; ++c) {
        cx<typename PT<PX>::A> xv[4];
        cx<AY> yv[4];
        ldc<PX>(xb, fx.Vh, fx.d, i, c, xv);
        if (bv != (AY)0) ldc<PY>(yb, fy.Vh, fy.d, i, c, yv);
        else
#pragma unroll
          for (int q = 0; q < 4; ++q) yv[q] = mk((AY)0, (AY)0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          m = fmaxf(m, fabsf((float)(av * (AY)xv[q].x + bv * yv[q].x)));
          m = fmaxf(m, fabsf((float)(av * (AY)xv[q].y + bv * yv[q].y)));
        }
      }
      inv = m > 0.f ? 1.f / m : 0.f;
      AY s = 0;
      for (int c = 0; c < fx.d; ++c) {
        cx<typename PT<PX>::A> xv[4];
        cx<AY> yv[4];
        ldc<PX>(xb, fx.Vh, fx.d, i, c, xv);
        if (bv != (AY)0) ldc<PY>(yb, fy.Vh, fy.d, i, c, yv);
        else
#pragma unroll
          for (int q = 0; q < 4; ++q) yv[q] = mk((AY)0, (AY)0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          yv[q] = mk(av * (AY)xv[q].x + bv * yv[q].x, av * (AY)xv[q].y + bv * yv[q].y);
          s += yv[q].x * yv[q].x + yv[q].y * yv[q].y;
        }
        stc<PY>(yb, fy.Vh, i, c, yv, inv);
      }
      f16_scales_w(yb, fy.Vh, fy.d)[i] = m;
      acc += (double)s;
    } else {
      AY s = 0;
      for (int c = 0; c < fx.d; ++c) {
        cx<typename PT<PX>::A> xv[4];
        cx<AY> yv[4];
        ldc<PX>(xb, fx.Vh, fx.d, i, c, xv);
        if (bv != (AY)0) ldc<PY>(yb, fy.Vh, fy.d, i, c, yv);
        else
#pragma unroll
          for (int q = 0; q < 4; ++q) yv[q] = mk((AY)0, (AY)0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          yv[q] = mk(fma(av, (AY)xv[q].x, bv * yv[q].x), fma(av, (AY)xv[q].y, bv * yv[q].y));
          s += yv[q].x * yv[q].x + yv[q].y * yv[q].y;
        }
        stc<PY>(yb, fy.Vh, i, c, yv, inv);
      }
      acc += (double)s;
    }
  }
  if (want_norm) reduce_publish(acc, red, RED_PLAIN, fx.nsub);
}

// ---------------------------------------------------------------- launchers
int hr_blas_norm2(const FieldDesc &f, int prec, const void *x, int nrhs, const RedArgs &red, int finish,
                  cudaStream_t s) {
  dim3 grid(hr_blas_blocks(f.Vh), nrhs * f.nsub);
  if (prec == HR_F64) norm2_kernel<0><<<grid, 256, 0, s>>>(x, f, red, finish);
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
  else AXPBY(2, 2);
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
    HR_CUDA(cudaMalloc(&lat->red_out, sizeof(double) * HR_MAX_RHS));
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
