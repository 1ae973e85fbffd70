// Small complex-arithmetic helpers and the per-precision load/store of the
// internal spinor, link and clover chunks (layouts in hr_internal.h).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

template <typename R>
struct cx {
  R x, y;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R x, R y) {
  cx<R> c;
  c.x = x;
  c.y = y;
  return c;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.x - b.x, a.y - b.y); }
// a + s*b, s real
template <typename R>
__device__ __forceinline__ cx<R> axpy_r(R s, cx<R> b, cx<R> a) { return mk(fma(s, b.x, a.x), fma(s, b.y, a.y)); }
// a + i*s*b, s real:  i s (bx + i by) = -s by + i s bx
template <typename R>
__device__ __forceinline__ cx<R> axpy_i(R s, cx<R> b, cx<R> a) { return mk(fma(-s, b.y, a.x), fma(s, b.x, a.y)); }
// acc + u * v
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> u, cx<R> v, cx<R> acc) {
  acc.x = fma(u.x, v.x, acc.x);
  acc.x = fma(-u.y, v.y, acc.x);
  acc.y = fma(u.x, v.y, acc.y);
  acc.y = fma(u.y, v.x, acc.y);
  return acc;
}
// acc + conj(u) * v
template <typename R>
__device__ __forceinline__ cx<R> cfmac(cx<R> u, cx<R> v, cx<R> acc) {
  acc.x = fma(u.x, v.x, acc.x);
  acc.x = fma(u.y, v.y, acc.x);
  acc.y = fma(u.x, v.y, acc.y);
  acc.y = fma(-u.y, v.x, acc.y);
  return acc;
}
// acc + r * v, r real
template <typename R>
__device__ __forceinline__ cx<R> rfma(R r, cx<R> v, cx<R> acc) { return mk(fma(r, v.x, acc.x), fma(r, v.y, acc.y)); }
template <typename R>
__device__ __forceinline__ cx<R> scale(R s, cx<R> a) { return mk(s * a.x, s * a.y); }

// ----------------------------------------------------------- float-float ----
// A real number as the unevaluated sum h + l of two FP32 numbers (Dekker's
// double-length arithmetic with Knuth's exact two-sum): about 48 significant
// bits, the FP32 exponent range, and every operation a handful of FP32
// instructions.  This part's FP64 pipe runs at about 1/64 of its FP32 pipe, so
// a stencil in this arithmetic can outrun the same stencil in FP64.
//
// Inside a kernel the pairs are not renormalised after every sum (|l| may
// exceed half an ulp of h, e.g. after a cancellation); products therefore take
// all four partial products h*h (exactly, as p + fma(h, h, -p)), h*l, l*h and
// l*l, so the error of every result stays about 2^-47 of the size of its
// operands.  Stores and norms renormalise.  All operations use the _rn
// intrinsics, so the compiler neither contracts a product into a following add
// nor reorders the error terms.
struct ff {
  float h, l;
  ff() = default;
  __device__ __forceinline__ ff(float x) : h(x), l(0.f) {}
  __device__ __forceinline__ ff(int x) : h((float)x), l(0.f) {}
  // the FP64 value to 48 bits: FP64 instructions, so for kernel parameters
  // and one-off conversions only
  __device__ __forceinline__ explicit ff(double x) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(h, l); }
};
__device__ __forceinline__ ff mkff(float h, float l) {
  ff r;
  r.h = h;
  r.l = l;
  return r;
}
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// the same value with |l| at most half an ulp of h
__device__ __forceinline__ ff ff_norm(ff a) {
  float s, e;
  two_sum(a.h, a.l, s, e);
  return mkff(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return mkff(-a.h, -a.l); }
__device__ __forceinline__ ff operator+(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return mkff(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.l, b.l, e);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return mkff(p, e);
}
// a*b + c
__device__ __forceinline__ ff fma(ff a, ff b, ff c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  float s, t;
  two_sum(p, c.h, s, t);
  e = __fadd_rn(e, t);
  e = __fadd_rn(e, c.l);
  e = __fmaf_rn(a.l, b.l, e);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return mkff(s, e);
}
__device__ __forceinline__ bool operator!=(ff a, ff b) { return a.h != b.h || a.l != b.l; }

// ------------------------------------------------------------ precisions ----
// P = 0 (FP64), 1 (FP32), 2 (FP16), 3 (float-float); A = accumulation type.
// Float-float fields, links and clover blocks have the FP64 layouts, each
// 16-byte chunk holding (re.h, re.l, im.h, im.l) in place of (re, im).
template <int P> struct PT;
template <> struct PT<0> { typedef double A; typedef double2 S2; };   // S2: one stored 2-real chunk
template <> struct PT<1> { typedef float A; typedef float2 S2; };
template <> struct PT<2> { typedef float A; typedef __half2 S2; };
template <> struct PT<3> { typedef ff A; typedef float4 S2; };

// 2-real chunk k (link or clover) of site i, converted to the accumulation type
template <int P>
__device__ __forceinline__ cx<typename PT<P>::A> ld2(const void *base, int64_t idx);
template <>
__device__ __forceinline__ cx<double> ld2<0>(const void *base, int64_t idx) {
  double2 v = __ldg(reinterpret_cast<const double2 *>(base) + idx);
  return mk(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<float> ld2<1>(const void *base, int64_t idx) {
  float2 v = __ldg(reinterpret_cast<const float2 *>(base) + idx);
  return mk(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<float> ld2<2>(const void *base, int64_t idx) {
  __half2 h = reinterpret_cast<const __half2 *>(base)[idx];
  float2 v = __half22float2(h);
  return mk(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<ff> ld2<3>(const void *base, int64_t idx) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(base) + idx);
  return mk(mkff(v.x, v.y), mkff(v.z, v.w));
}

// the four spin components of colour c of site i of a spinor field
template <int P>
__device__ __forceinline__ void ld_colour(const void *f, int64_t Vh, int64_t i, int c,
                                          cx<typename PT<P>::A> psi[4]);
template <>
__device__ __forceinline__ void ld_colour<0>(const void *f, int64_t Vh, int64_t i, int c, cx<double> psi[4]) {
  const double2 *p = reinterpret_cast<const double2 *>(f);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    double2 v = __ldg(p + (int64_t)(4 * c + s) * Vh + i);
    psi[s] = mk(v.x, v.y);
  }
}
template <>
__device__ __forceinline__ void ld_colour<1>(const void *f, int64_t Vh, int64_t i, int c, cx<float> psi[4]) {
  const float4 *p = reinterpret_cast<const float4 *>(f);
  float4 a = __ldg(p + (int64_t)(2 * c) * Vh + i);
  float4 b = __ldg(p + (int64_t)(2 * c + 1) * Vh + i);
  psi[0] = mk(a.x, a.y);
  psi[1] = mk(a.z, a.w);
  psi[2] = mk(b.x, b.y);
  psi[3] = mk(b.z, b.w);
}
template <>
__device__ __forceinline__ void ld_colour<2>(const void *f, int64_t Vh, int64_t i, int c, cx<float> psi[4]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(f);
  uint4 u = __ldg(p + (int64_t)c * Vh + i);
  __half2 h0 = *reinterpret_cast<__half2 *>(&u.x);
  __half2 h1 = *reinterpret_cast<__half2 *>(&u.y);
  __half2 h2 = *reinterpret_cast<__half2 *>(&u.z);
  __half2 h3 = *reinterpret_cast<__half2 *>(&u.w);
  float2 f0 = __half22float2(h0), f1 = __half22float2(h1), f2 = __half22float2(h2), f3 = __half22float2(h3);
  psi[0] = mk(f0.x, f0.y);
  psi[1] = mk(f1.x, f1.y);
  psi[2] = mk(f2.x, f2.y);
  psi[3] = mk(f3.x, f3.y);
}
template <>
__device__ __forceinline__ void ld_colour<3>(const void *f, int64_t Vh, int64_t i, int c, cx<ff> psi[4]) {
  const float4 *p = reinterpret_cast<const float4 *>(f);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    float4 v = __ldg(p + (int64_t)(4 * c + s) * Vh + i);
    psi[s] = mk(mkff(v.x, v.y), mkff(v.z, v.w));
  }
}

// per-site scale of an FP16 field (stored after the d chunk arrays)
__device__ __forceinline__ const float *f16_scales(const void *f, int64_t Vh, int d) {
  return reinterpret_cast<const float *>(reinterpret_cast<const char *>(f) + (size_t)d * 16u * (size_t)Vh);
}
__device__ __forceinline__ float *f16_scales_w(void *f, int64_t Vh, int d) {
  return reinterpret_cast<float *>(reinterpret_cast<char *>(f) + (size_t)d * 16u * (size_t)Vh);
}

// store colour c (4 spins) of an FP64 / FP32 field
__device__ __forceinline__ void st_colour64(void *f, int64_t Vh, int64_t i, int c, const cx<double> v[4]) {
  double2 *p = reinterpret_cast<double2 *>(f);
#pragma unroll
  for (int s = 0; s < 4; ++s) p[(int64_t)(4 * c + s) * Vh + i] = make_double2(v[s].x, v[s].y);
}
__device__ __forceinline__ void st_colour32(void *f, int64_t Vh, int64_t i, int c, const cx<float> v[4]) {
  float4 *p = reinterpret_cast<float4 *>(f);
  p[(int64_t)(2 * c) * Vh + i] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  p[(int64_t)(2 * c + 1) * Vh + i] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}
// store colour c of a float-float field, each pair renormalised
__device__ __forceinline__ void st_colour_ff(void *f, int64_t Vh, int64_t i, int c, const cx<ff> v[4]) {
  float4 *p = reinterpret_cast<float4 *>(f);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const ff x = ff_norm(v[s].x), y = ff_norm(v[s].y);
    p[(int64_t)(4 * c + s) * Vh + i] = make_float4(x.h, x.l, y.h, y.l);
  }
}
// store colour c of an FP16 field, values already divided by the site scale
__device__ __forceinline__ void st_colour16(void *f, int64_t Vh, int64_t i, int c, const cx<float> v[4]) {
  uint4 u;
  __half2 h0 = __floats2half2_rn(v[0].x, v[0].y);
  __half2 h1 = __floats2half2_rn(v[1].x, v[1].y);
  __half2 h2 = __floats2half2_rn(v[2].x, v[2].y);
  __half2 h3 = __floats2half2_rn(v[3].x, v[3].y);
  u.x = *reinterpret_cast<unsigned *>(&h0);
  u.y = *reinterpret_cast<unsigned *>(&h1);
  u.z = *reinterpret_cast<unsigned *>(&h2);
  u.w = *reinterpret_cast<unsigned *>(&h3);
  reinterpret_cast<uint4 *>(f)[(int64_t)c * Vh + i] = u;
}

// -------------------------------------------------------------- geometry ----
// Coordinates of checkerboard index i of parity p.
struct Site {
  int t, x, y, z;
};
__device__ __forceinline__ Site site_of(int64_t i, int p, int L, int Lh) {
  Site s;
  int xh = (int)(i % Lh);
  int64_t r = i / Lh;
  s.y = (int)(r % L);
  r /= L;
  s.z = (int)(r % L);
  s.t = (int)(r / L);
  s.x = 2 * xh + ((s.t + s.y + s.z + p) & 1);
  return s;
}
// checkerboard index of a site (any parity)
__device__ __forceinline__ int64_t cb_index(int t, int x, int y, int z, int L, int Lh) {
  return (((int64_t)t * L + z) * L + y) * Lh + (x >> 1);
}
__device__ __forceinline__ int64_t lex_index(int t, int x, int y, int z, int L) {
  return (((int64_t)t * L + z) * L + y) * L + x;
}
