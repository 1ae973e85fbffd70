// Device-side building blocks of the site-wise linear algebra (Sec. 3.2):
// the fused FP64 block reduction with deterministic last-block finish, the
// precision-generic colour loads/stores, and the per-site loops of the CG
// vector updates.  Each loop processes sites i0, i0 + stride, ... of one
// single-parity field and returns this thread's FP64 partial sum, so the
// single-lattice kernels (blas.cu) and the multi-lattice kernels (batch.cu)
// share one body.
#pragma once

#include <math.h>

#include "blas.cuh"
#include "cplx.cuh"
#include "hr_internal.h"

// block-wide FP64 sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // sh may still be read by a previous call
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

// Publish this block's partial `v` as part `part` of `nparts` for result slot
// `slot`; the last block to arrive sums the parts in part order (deterministic)
// and applies `finish` (plain sum, alpha, or beta / rr_next / frozen).
__device__ __forceinline__ void reduce_publish(double v, const RedArgs &red, int finish, int slot, int part,
                                               int nparts) {
  double s = block_sum(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    red.partials[(size_t)slot * 2 * HR_RED_MAXBLK + part] = s;
    __threadfence();
    const unsigned prev = atomicAdd(&red.count[slot], 1u);
    last = (prev == (unsigned)nparts - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  if (threadIdx.x < 32) {
    for (int b = threadIdx.x; b < nparts; b += 32)
      t += ((volatile double *)red.partials)[(size_t)slot * 2 * HR_RED_MAXBLK + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  if (threadIdx.x == 0) {
    red.out[slot] = t;
    red.count[slot] = 0u;
    if (finish == RED_ALPHA) {
      // alpha = rr / pAp, frozen (0) once rr reached the stop threshold or on breakdown
      const double rr = red.rr[slot];
      double al = 0.0;
      if (rr > red.stop[slot]) {
        if (t > 0.0 && isfinite(t)) al = rr / t;
        else atomicExch(red.err, 1);
      }
      red.alpha[slot] = al;
      if (red.iters && al != 0.0) red.iters[slot] += 1;
    } else if (finish == RED_BETA) {
      const double rr = red.rr[slot];
      red.beta[slot] = (rr > 0.0 && red.alpha[slot] != 0.0) ? t / rr : 0.0;
      const double nx = (red.alpha[slot] != 0.0) ? t : rr;
      red.rr_next[slot] = nx;
      if (red.frozen) red.frozen[slot] = (nx <= red.stop[slot]) ? 1 : 0;
    }
  }
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

// store colour c (FP16: multiplied by `inv` = 1/site scale first)
template <int P>
__device__ __forceinline__ void stc(char *f, int64_t Vh, int64_t i, int c, const cx<typename PT<P>::A> v[4],
                                    float inv) {
  if constexpr (P == 0) st_colour64(f, Vh, i, c, reinterpret_cast<const cx<double> *>(v));
  else if constexpr (P == 1) st_colour32(f, Vh, i, c, reinterpret_cast<const cx<float> *>(v));
  else if constexpr (P == 3) st_colour_ff(f, Vh, i, c, v);
  else {
    cx<float> w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = mk((float)v[q].x * inv, (float)v[q].y * inv);
    st_colour16(f, Vh, i, c, w);
  }
}

// sum |x|^2 over the sites
template <int P>
__device__ __forceinline__ double norm2_sites(const char *base, int64_t Vh, int d, int64_t i0, int64_t stride) {
  typedef typename PT<P>::A A;
  double acc = 0.0;
  for (int64_t i = i0; i < Vh; i += stride) {
    A s[4] = {0, 0, 0, 0};  // one chain per spin: four independent FMA chains (GB300's FP64 latency)
    for (int c = 0; c < d; ++c) {
      cx<A> v[4];
      ld_colour<P>(base, Vh, i, c, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] = fma(v[q].y, v[q].y, fma(v[q].x, v[q].x, s[q]));
    }
    double sd = (double)((s[0] + s[1]) + (s[2] + s[3]));
    if (P == 2) {
      const double sc = (double)f16_scales(base, Vh, d)[i];
      sd *= sc * sc;
    }
    acc += sd;
  }
  return acc;
}

// x += alpha p ; r -= alpha Ap ; returns sum |r_new|^2   (x, r: PR; p, Ap: PP)
template <int PR, int PP>
__device__ __forceinline__ double cg_xr_sites(char *xb, char *rb, const char *pb, const char *ab, int64_t Vh, int d,
                                              typename PT<PR>::A al, int64_t i0, int64_t stride) {
  typedef typename PT<PR>::A AR;
  double acc = 0.0;
  for (int64_t i = i0; i < Vh; i += stride) {
    AR s[4] = {0, 0, 0, 0};  // one chain per spin
    for (int c = 0; c < d; ++c) {
      cx<AR> xv[4], rv[4];
      cx<typename PT<PP>::A> pv[4], av[4];
      ldc<PR>(xb, Vh, d, i, c, xv);
      ldc<PR>(rb, Vh, d, i, c, rv);
      ldc<PP>(pb, Vh, d, i, c, pv);
      ldc<PP>(ab, Vh, d, i, c, av);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xv[q] = mk(fma(al, (AR)pv[q].x, xv[q].x), fma(al, (AR)pv[q].y, xv[q].y));
        rv[q] = mk(fma(-al, (AR)av[q].x, rv[q].x), fma(-al, (AR)av[q].y, rv[q].y));
        s[q] = fma(rv[q].y, rv[q].y, fma(rv[q].x, rv[q].x, s[q]));
      }
      stc<PR>(xb, Vh, i, c, xv, 1.f);
      stc<PR>(rb, Vh, i, c, rv, 1.f);
    }
    acc += (double)((s[0] + s[1]) + (s[2] + s[3]));
  }
  return acc;
}

// p = r + beta p   (r: PR, p: PP).  FP16 p: a first pass finds the new site
// maximum, the second reads the old p again and writes the new one (the old
// scale is overwritten last).
template <int PR, int PP>
__device__ __forceinline__ void cg_p_sites(const char *rb, char *pb, int64_t Vh, int d, typename PT<PP>::A be,
                                           int64_t i0, int64_t stride) {
  typedef typename PT<PP>::A AP;
  for (int64_t i = i0; i < Vh; i += stride) {
    float inv = 1.f, m = 0.f;
    if (PP == 2) {
      for (int c = 0; c < d; ++c) {
        cx<typename PT<PR>::A> rv[4];
        cx<AP> pv[4];
        ldc<PR>(rb, Vh, d, i, c, rv);
        ldc<PP>(pb, Vh, d, i, c, pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          m = fmaxf(m, fabsf((float)fma(be, pv[q].x, (AP)rv[q].x)));
          m = fmaxf(m, fabsf((float)fma(be, pv[q].y, (AP)rv[q].y)));
        }
      }
      inv = m > 0.f ? 1.f / m : 0.f;
    }
    for (int c = 0; c < d; ++c) {
      cx<typename PT<PR>::A> rv[4];
      cx<AP> pv[4];
      ldc<PR>(rb, Vh, d, i, c, rv);
      ldc<PP>(pb, Vh, d, i, c, pv);
#pragma unroll
      for (int q = 0; q < 4; ++q) pv[q] = mk(fma(be, pv[q].x, (AP)rv[q].x), fma(be, pv[q].y, (AP)rv[q].y));
      stc<PP>(pb, Vh, i, c, pv, inv);
    }
    if (PP == 2) f16_scales_w(pb, Vh, d)[i] = m;
  }
}

// y = a x + b y (b == 0: y overwritten); returns sum |y_new|^2   (x: PX, y: PY)
template <int PX, int PY>
__device__ __forceinline__ double axpby_sites(const char *xb, char *yb, int64_t Vh, int d, typename PT<PY>::A av,
                                              typename PT<PY>::A bv, int64_t i0, int64_t stride) {
  typedef typename PT<PY>::A AY;
  double acc = 0.0;
  for (int64_t i = i0; i < Vh; i += stride) {
    float inv = 1.f, m = 0.f;
    if (PY == 2) {
      for (int c = 0; c < d; ++c) {
        cx<typename PT<PX>::A> xv[4];
        cx<AY> yv[4];
        ldc<PX>(xb, Vh, d, i, c, xv);
        if (bv != (AY)0) ldc<PY>(yb, Vh, d, i, c, yv);
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
    }
    AY s[4] = {0, 0, 0, 0};  // one chain per spin
    for (int c = 0; c < d; ++c) {
      cx<typename PT<PX>::A> xv[4];
      cx<AY> yv[4];
      ldc<PX>(xb, Vh, d, i, c, xv);
      if (bv != (AY)0) ldc<PY>(yb, Vh, d, i, c, yv);
      else
#pragma unroll
        for (int q = 0; q < 4; ++q) yv[q] = mk((AY)0, (AY)0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (PY == 2) yv[q] = mk(av * (AY)xv[q].x + bv * yv[q].x, av * (AY)xv[q].y + bv * yv[q].y);
        else yv[q] = mk(fma(av, (AY)xv[q].x, bv * yv[q].x), fma(av, (AY)xv[q].y, bv * yv[q].y));
        if constexpr (PY == 3) yv[q] = mk(ff_norm(yv[q].x), ff_norm(yv[q].y));  // after a cancellation |l| ~ |h|
        s[q] = fma(yv[q].y, yv[q].y, fma(yv[q].x, yv[q].x, s[q]));
      }
      stc<PY>(yb, Vh, i, c, yv, inv);
    }
    if (PY == 2) f16_scales_w(yb, Vh, d)[i] = m;
    acc += (double)((s[0] + s[1]) + (s[2] + s[3]));
  }
  return acc;
}
