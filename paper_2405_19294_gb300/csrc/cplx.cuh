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

// ------------------------------------------------------------ precisions ----
// P = 0 (FP64), 1 (FP32), 2 (FP16); A = accumulation type.
template <int P> struct PT;
template <> struct PT<0> { typedef double A; typedef double2 S2; };   // S2: one stored 2-real chunk
template <> struct PT<1> { typedef float A; typedef float2 S2; };
template <> struct PT<2> { typedef float A; typedef __half2 S2; };

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
