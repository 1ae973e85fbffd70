// The spin-projected 8-neighbour hopping kernel (one output site per thread).
//
// For output parity p and each output site x it computes
//   H(x) = sum_mu [ (1 - s g_mu) U_R,mu(x) psi(x+mu) + (1 + s g_mu) U_R,mu(x-mu)^+ psi(x-mu) ]
// (s = +1 for D, -1 for D^+ = g5 D g5) and applies the epilogue
//   HOP_SCALED:  out = coef * H            or  A^{-1} (coef * H)   (clover)
//   HOP_SELF  :  out = diag * self + coef*H or  A self + coef * H   (clover)
// which covers the two halves of the Schur complement and the full operator
// (Sec. 3.1, even-odd preconditioning and clover).
//
// Each neighbour spinor is projected to a half-spinor (two spin rows) before
// the colour multiply, the projection of Sec. 2.2, so each U_R (or U_R^+)
// multiplies 2 instead of 4 colour vectors; the two lower spin rows are
// rebuilt from the products.  With the chiral gammas and projector
// (1 + sig g_mu):
//   mu=0: h0 = p0 - sig p2,    h1 = p1 - sig p3;    row2 = -sig r0,   row3 = -sig r1
//   mu=1: h0 = p0 - i sig p3,  h1 = p1 - i sig p2;  row2 = i sig r1,  row3 = i sig r0
//   mu=2: h0 = p0 - sig p3,    h1 = p1 + sig p2;    row2 = sig r1,    row3 = -sig r0
//   mu=3: h0 = p0 - i sig p2,  h1 = p1 + i sig p3;  row2 = i sig r0,  row3 = -i sig r1
// where r0, r1 are the colour products of h0, h1.  The sign sig is a runtime
// +-1 so D and D^+ share one kernel (the adds become FMAs with +-1).
#pragma once

#include "cplx.cuh"
#include "hr_internal.h"

struct HopK {
  void *out;
  const void *in;
  const void *self;
  const void *links;
  const void *clover;
  int T, L, Lh, p, mode, nch, nrhs;
  int64_t Vh;
  size_t stride;
  double sgn, coef, diag;
  const void *rlinks;  // rows-kernel link layout (rows kernel only)
  int tmask;           // time-slab bulk pass (site kernel only)
};

// Converged-rhs skip (see HopArgs), a kernel parameter of its own: growing
// HopK moved the compiler's register and load scheduling of the stencils.
struct SkipK {
  const double *rr, *stop;
};
static inline SkipK make_skipk(const HopArgs &a) { return SkipK{a.skip_rr, a.skip_stop}; }

// true when right-hand side rhs has converged and its hop is not needed
__device__ __forceinline__ bool rhs_done(const SkipK &sk, int rhs) { return sk.rr && sk.rr[rhs] <= sk.stop[rhs]; }

// Blocks are numbered right-hand side fastest: block b handles tile b / nrhs
// of right-hand side b % nrhs, so the nrhs blocks that read the same links run
// back to back and all but the first find them in L2.
__device__ __forceinline__ void block_tile(const HopK &k, int64_t &tile, int &rhs) {
  rhs = (int)(blockIdx.x % (unsigned)k.nrhs);
  tile = blockIdx.x / (unsigned)k.nrhs;
}

template <int MU, typename R>
__device__ __forceinline__ void project(R sig, const cx<R> psi[4], cx<R> &h0, cx<R> &h1) {
  if (MU == 0) {
    h0 = axpy_r(-sig, psi[2], psi[0]);
    h1 = axpy_r(-sig, psi[3], psi[1]);
  } else if (MU == 1) {
    h0 = axpy_i(-sig, psi[3], psi[0]);
    h1 = axpy_i(-sig, psi[2], psi[1]);
  } else if (MU == 2) {
    h0 = axpy_r(-sig, psi[3], psi[0]);
    h1 = axpy_r(sig, psi[2], psi[1]);
  } else {
    h0 = axpy_i(-sig, psi[2], psi[0]);
    h1 = axpy_i(sig, psi[3], psi[1]);
  }
}

template <int MU, typename R>
__device__ __forceinline__ void reconstruct(R sig, cx<R> r0, cx<R> r1, cx<R> acc[4]) {
  acc[0] = acc[0] + r0;
  acc[1] = acc[1] + r1;
  if (MU == 0) {
    acc[2] = axpy_r(-sig, r0, acc[2]);
    acc[3] = axpy_r(-sig, r1, acc[3]);
  } else if (MU == 1) {
    acc[2] = axpy_i(sig, r1, acc[2]);
    acc[3] = axpy_i(sig, r0, acc[3]);
  } else if (MU == 2) {
    acc[2] = axpy_r(sig, r1, acc[2]);
    acc[3] = axpy_r(-sig, r0, acc[3]);
  } else {
    acc[2] = axpy_i(sig, r0, acc[2]);
    acc[3] = axpy_i(-sig, r1, acc[3]);
  }
}

// reconstruct with the neighbour's FP16 site scale w folded in:
// acc += w * (rebuilt 4-spinor), the scale riding on the FMAs that add the
// rows anyway instead of a separate multiply of the half-spinor.
template <int MU, typename R>
__device__ __forceinline__ void reconstruct_w(R sig, R w, cx<R> r0, cx<R> r1, cx<R> acc[4]) {
  const R sw = sig * w;
  acc[0] = axpy_r(w, r0, acc[0]);
  acc[1] = axpy_r(w, r1, acc[1]);
  if (MU == 0) {
    acc[2] = axpy_r(-sw, r0, acc[2]);
    acc[3] = axpy_r(-sw, r1, acc[3]);
  } else if (MU == 1) {
    acc[2] = axpy_i(sw, r1, acc[2]);
    acc[3] = axpy_i(sw, r0, acc[3]);
  } else if (MU == 2) {
    acc[2] = axpy_r(sw, r1, acc[2]);
    acc[3] = axpy_r(-sw, r0, acc[3]);
  } else {
    acc[2] = axpy_i(sw, r0, acc[2]);
    acc[3] = axpy_i(-sw, r1, acc[3]);
  }
}

// ---- FP16 fields: half2 projection, mixed-precision FMAs ----
// The projected half-spinor is formed in half2 arithmetic straight from the
// stored FP16 components (the +-1 and +-i factors are exact; the one add rounds
// to FP16), and the link products use fma.rn.f32.f16: both factors FP16, the
// product and the accumulation in FP32.  Neither the spinor nor the link
// entries pass through conversions to FP32.
__device__ __forceinline__ float fma_f16(unsigned a, unsigned b, float c, bool hi_a, bool hi_b) {
  const unsigned short ah = (unsigned short)(hi_a ? (a >> 16) : (a & 0xffffu));
  const unsigned short bh = (unsigned short)(hi_b ? (b >> 16) : (b & 0xffffu));
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(ah), "h"(bh), "f"(c));
  return d;
}
__device__ __forceinline__ unsigned h2u(__half2 h) { return *reinterpret_cast<unsigned *>(&h); }
__device__ __forceinline__ __half2 u2h(unsigned u) { return *reinterpret_cast<__half2 *>(&u); }
// a + s b and a + i s b on half2 complex numbers; s2 = (s, s), si2 = (-s, s)
__device__ __forceinline__ unsigned h2_axpy_r(__half2 s2, unsigned b, unsigned a) {
  return h2u(__hfma2(s2, u2h(b), u2h(a)));
}
__device__ __forceinline__ unsigned h2_axpy_i(__half2 si2, unsigned b, unsigned a) {
  return h2u(__hfma2(si2, __lowhigh2highlow(u2h(b)), u2h(a)));
}
// acc + u h (ADJ: conj(u) h) with u, h FP16 complex and hr = i h (ADJ: -i h)
__device__ __forceinline__ cx<float> cfma_f16(unsigned u, unsigned h, unsigned hr, cx<float> acc) {
  acc.x = fma_f16(u, h, acc.x, false, false);
  acc.x = fma_f16(u, hr, acc.x, true, false);
  acc.y = fma_f16(u, h, acc.y, false, true);
  acc.y = fma_f16(u, hr, acc.y, true, true);
  return acc;
}

// half-spinor rows h0, h1 of the projection (1 -+ gamma_mu) of one colour's
// stored FP16 components v = (psi0, psi1, psi2, psi3), as half2 complex numbers
template <int MU>
__device__ __forceinline__ void project_h2(float sig, const uint4 &v, unsigned &h0, unsigned &h1) {
  if (MU == 0) {
    const __half2 m_r = __float2half2_rn(-sig);
    h0 = h2_axpy_r(m_r, v.z, v.x);
    h1 = h2_axpy_r(m_r, v.w, v.y);
  } else if (MU == 1) {
    const __half2 m_i = __floats2half2_rn(sig, -sig);
    h0 = h2_axpy_i(m_i, v.w, v.x);
    h1 = h2_axpy_i(m_i, v.z, v.y);
  } else if (MU == 2) {
    h0 = h2_axpy_r(__float2half2_rn(-sig), v.w, v.x);
    h1 = h2_axpy_r(__float2half2_rn(sig), v.z, v.y);
  } else {
    h0 = h2_axpy_i(__floats2half2_rn(sig, -sig), v.z, v.x);
    h1 = h2_axpy_i(__floats2half2_rn(-sig, sig), v.w, v.y);
  }
}
// i h = (-h.y, h.x), or -i h = (h.y, -h.x) when NEG
template <bool NEG>
__device__ __forceinline__ unsigned rot_h2(unsigned h) {
  const __half2 rot = NEG ? __floats2half2_rn(1.f, -1.f) : __floats2half2_rn(-1.f, 1.f);
  return h2u(__hmul2(rot, __lowhigh2highlow(u2h(h))));
}

template <int D, int MU, bool ADJ>
__device__ __forceinline__ void hop_dir_f16(cx<float> acc[D][4], const void *in, int64_t Vh, int64_t j,
                                            const void *lk, int64_t li, float sig, float scl) {
  unsigned h0[D], h1[D], g0[D], g1[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    project_h2<MU>(sig, __ldg(reinterpret_cast<const uint4 *>(in) + (int64_t)c * Vh + j), h0[c], h1[c]);
    g0[c] = rot_h2<ADJ>(h0[c]);
    g1[c] = rot_h2<ADJ>(h1[c]);
  }
  const unsigned *lu = reinterpret_cast<const unsigned *>(lk);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<float> r0 = mk(0.f, 0.f), r1 = mk(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const unsigned u = __ldg(lu + (int64_t)(ADJ ? (c * D + a) : (a * D + c)) * Vh + li);
      r0 = cfma_f16(u, h0[c], g0[c], r0);
      r1 = cfma_f16(u, h1[c], g1[c], r1);
    }
    reconstruct_w<MU>(sig, scl, r0, r1, acc[a]);
  }
}

// the same for real (adjoint) links: entry e of the d x d matrix is half
// (e & 1) of 2-real chunk e >> 1; U^T for the backward hop
template <int D, int MU, bool ADJ>
__device__ __forceinline__ void hop_dir_f16_real(cx<float> acc[D][4], const void *in, int64_t Vh, int64_t j,
                                                 const void *lk, int64_t li, float sig, float scl) {
  constexpr int NC = (D * D + 1) / 2;
  unsigned h0[D], h1[D];
#pragma unroll
  for (int c = 0; c < D; ++c)
    project_h2<MU>(sig, __ldg(reinterpret_cast<const uint4 *>(in) + (int64_t)c * Vh + j), h0[c], h1[c]);
  const unsigned *lu = reinterpret_cast<const unsigned *>(lk);
  unsigned u[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) u[k] = __ldg(lu + (int64_t)k * Vh + li);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<float> r0 = mk(0.f, 0.f), r1 = mk(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int e = ADJ ? (c * D + a) : (a * D + c);
      const bool hi = (e & 1) != 0;
      r0.x = fma_f16(u[e >> 1], h0[c], r0.x, hi, false);
      r0.y = fma_f16(u[e >> 1], h0[c], r0.y, hi, true);
      r1.x = fma_f16(u[e >> 1], h1[c], r1.x, hi, false);
      r1.y = fma_f16(u[e >> 1], h1[c], r1.y, hi, true);
    }
    reconstruct_w<MU>(sig, scl, r0, r1, acc[a]);
  }
}

// One direction, one side: project psi(j), multiply by U (or U^+ when ADJ),
// accumulate.  `lk` points at chunk 0 of the link slot, `li` is the link's
// site index in that slot.
template <int D, bool REAL, int P, int MU, bool ADJ>
__device__ __forceinline__ void hop_dir(cx<typename PT<P>::A> acc[D][4], const void *in, int64_t Vh,
                                        int64_t j, const void *lk, int64_t li,
                                        typename PT<P>::A sig, typename PT<P>::A scl) {
  typedef typename PT<P>::A A;
  // FP16: half2 projection and mixed-precision FMAs, except for complex d_R = 5
  // and 7, where the extra live half-spinor copies made the kernel spill and run
  // 3-6 % slower than converting to FP32 first (d_R = 2, 3, 6 and the real
  // classes gained 5-12 %)
  if constexpr (P == 2 && (REAL || (D != 5 && D != 7))) {
    if constexpr (REAL) hop_dir_f16_real<D, MU, ADJ>(acc, in, Vh, j, lk, li, sig, scl);
    else hop_dir_f16<D, MU, ADJ>(acc, in, Vh, j, lk, li, sig, scl);
    return;
  }
  // FP16: the neighbour's site scale scl is applied in the reconstruction
  cx<A> h0[D], h1[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    cx<A> psi[4];
    ld_colour<P>(in, Vh, j, c, psi);
    project<MU>(sig, psi, h0[c], h1[c]);
  }
  auto rebuild = [&](cx<A> r0, cx<A> r1, cx<A> a4[4]) {
    if (P == 2) reconstruct_w<MU>(sig, scl, r0, r1, a4);
    else reconstruct<MU>(sig, r0, r1, a4);
  };
  if (REAL) {
    constexpr int NC = (D * D + 1) / 2;
    cx<A> u[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) u[k] = ld2<P>(lk, (int64_t)k * Vh + li);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      cx<A> r0 = mk(A(0), A(0)), r1 = mk(A(0), A(0));
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const int e = ADJ ? (c * D + a) : (a * D + c);
        const A ue = (e & 1) ? u[e >> 1].y : u[e >> 1].x;
        r0 = rfma(ue, h0[c], r0);
        r1 = rfma(ue, h1[c], r1);
      }
      rebuild(r0, r1, acc[a]);
    }
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      cx<A> r0 = mk(A(0), A(0)), r1 = mk(A(0), A(0));
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (ADJ) {
          const cx<A> ue = ld2<P>(lk, (int64_t)(c * D + a) * Vh + li);
          r0 = cfmac(ue, h0[c], r0);
          r1 = cfmac(ue, h1[c], r1);
        } else {
          const cx<A> ue = ld2<P>(lk, (int64_t)(a * D + c) * Vh + li);
          r0 = cfma(ue, h0[c], r0);
          r1 = cfma(ue, h1[c], r1);
        }
      }
      rebuild(r0, r1, acc[a]);
    }
  }
}

// w = B v for one packed Hermitian 2D x 2D block (chunk offset `off`):
// D chunks of diagonal pairs, then the strictly lower triangle row by row.
template <int D, int P>
__device__ __forceinline__ void herm_apply(const void *cl, int64_t Vh, int64_t i, int off,
                                           const cx<typename PT<P>::A> v[2 * D],
                                           cx<typename PT<P>::A> w[2 * D]) {
  typedef typename PT<P>::A A;
  constexpr int n = 2 * D;
  constexpr int PC = (P == 0 || P == 3) ? P : 1;  // clover storage: FP64 / float-float, else FP32
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const cx<A> dg = ld2<PC>(cl, (int64_t)(off + q) * Vh + i);
    w[2 * q] = scale(dg.x, v[2 * q]);
    w[2 * q + 1] = scale(dg.y, v[2 * q + 1]);
  }
#pragma unroll
  for (int r = 1; r < n; ++r) {
#pragma unroll
    for (int c = 0; c < r; ++c) {
      const cx<A> a = ld2<PC>(cl, (int64_t)(off + D + r * (r - 1) / 2 + c) * Vh + i);
      w[r] = cfma(a, v[c], w[r]);
      w[c] = cfmac(a, v[r], w[c]);
    }
  }
}

// out = B acc (B = both chiral blocks of A or A^{-1}), in place on acc
template <int D, int P>
__device__ __forceinline__ void clover_apply(const void *cl, int64_t Vh, int64_t i,
                                             cx<typename PT<P>::A> acc[D][4]) {
  typedef typename PT<P>::A A;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    cx<A> v[2 * D], w[2 * D];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int c = 0; c < D; ++c) v[s * D + c] = acc[c][2 * b + s];
    herm_apply<D, P>(cl, Vh, i, b * 2 * D * D, v, w);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c][2 * b + s] = w[s * D + c];
  }
}

// The whole stencil for output site i (< Vh) of right-hand side rhs.  MASK:
// on a time slab, leave out the t hops that cross its faces (they arrive
// later from the halo); a template flag so that the ordinary kernels carry no
// branch that would keep the compiler from hoisting the t-direction loads.
template <int D, bool REAL, int P, bool MASK = false>
__device__ __forceinline__ void hop_site(const HopK &k, int64_t i, int rhs) {
  typedef typename PT<P>::A A;
  const size_t roff = (size_t)rhs * k.stride;
  const void *in = reinterpret_cast<const char *>(k.in) + roff;
  void *out = reinterpret_cast<char *>(k.out) + roff;
  const int64_t Vh = k.Vh;
  const int L = k.L, Lh = k.Lh, T = k.T, p = k.p;
  const Site s = site_of(i, p, L, Lh);
  const A sg = (A)k.sgn;
  const int64_t slab = (int64_t)k.nch * Vh;  // chunks per [parity][mu] slot
  auto slot = [&](int par, int mu) -> const void * {
    const size_t es = (P == 0) ? 16 : (P == 1 ? 8 : 4);
    return reinterpret_cast<const char *>(k.links) + (size_t)((par * 4 + mu) * slab) * es;
  };
  const float *isc = (P == 2) ? f16_scales(in, Vh, D) : nullptr;

  cx<A> acc[D][4];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[c][q] = mk(A(0), A(0));

  const int64_t LLh = (int64_t)L * Lh;
  // mu = 0 (t); on a time slab (tmask) the hops across its faces come later from the halo
  {
    const int tf = (s.t + 1 == T) ? 0 : s.t + 1, tb = (s.t == 0) ? T - 1 : s.t - 1;
    const int64_t jf = i + (int64_t)(tf - s.t) * L * LLh, jb = i + (int64_t)(tb - s.t) * L * LLh;
    if (!(MASK && s.t == T - 1))
      hop_dir<D, REAL, P, 0, false>(acc, in, Vh, jf, slot(p, 0), i, -sg, P == 2 ? (A)isc[jf] : A(1));
    if (!(MASK && s.t == 0))
      hop_dir<D, REAL, P, 0, true>(acc, in, Vh, jb, slot(1 - p, 0), jb, sg, P == 2 ? (A)isc[jb] : A(1));
  }
  // mu = 1 (x)
  {
    const int xf = (s.x + 1 == L) ? 0 : s.x + 1, xb = (s.x == 0) ? L - 1 : s.x - 1;
    const int64_t jf = i - (s.x >> 1) + (xf >> 1), jb = i - (s.x >> 1) + (xb >> 1);
    hop_dir<D, REAL, P, 1, false>(acc, in, Vh, jf, slot(p, 1), i, -sg, P == 2 ? (A)isc[jf] : A(1));
    hop_dir<D, REAL, P, 1, true>(acc, in, Vh, jb, slot(1 - p, 1), jb, sg, P == 2 ? (A)isc[jb] : A(1));
  }
  // mu = 2 (y)
  {
    const int yf = (s.y + 1 == L) ? 0 : s.y + 1, yb = (s.y == 0) ? L - 1 : s.y - 1;
    const int64_t jf = i + (int64_t)(yf - s.y) * Lh, jb = i + (int64_t)(yb - s.y) * Lh;
    hop_dir<D, REAL, P, 2, false>(acc, in, Vh, jf, slot(p, 2), i, -sg, P == 2 ? (A)isc[jf] : A(1));
    hop_dir<D, REAL, P, 2, true>(acc, in, Vh, jb, slot(1 - p, 2), jb, sg, P == 2 ? (A)isc[jb] : A(1));
  }
  // mu = 3 (z)
  {
    const int zf = (s.z + 1 == L) ? 0 : s.z + 1, zb = (s.z == 0) ? L - 1 : s.z - 1;
    const int64_t jf = i + (int64_t)(zf - s.z) * LLh, jb = i + (int64_t)(zb - s.z) * LLh;
    hop_dir<D, REAL, P, 3, false>(acc, in, Vh, jf, slot(p, 3), i, -sg, P == 2 ? (A)isc[jf] : A(1));
    hop_dir<D, REAL, P, 3, true>(acc, in, Vh, jb, slot(1 - p, 3), jb, sg, P == 2 ? (A)isc[jb] : A(1));
  }

  // ---- epilogue ----
  const A coef = (A)k.coef;
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[c][q] = scale(coef, acc[c][q]);
  if (k.mode == HOP_SCALED) {
    if (k.clover) clover_apply<D, P>(k.clover, Vh, i, acc);
  } else {
    const void *self = reinterpret_cast<const char *>(k.self) + roff;
    const A ssc = (P == 2) ? (A)f16_scales(self, Vh, D)[i] : A(1);
    cx<A> sv[D][4];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      ld_colour<P>(self, Vh, i, c, sv[c]);
      if (P == 2 && k.clover)  // without clover the scale joins the diagonal factor below
#pragma unroll
        for (int q = 0; q < 4; ++q) sv[c][q] = scale(ssc, sv[c][q]);
    }
    if (k.clover) {
      clover_apply<D, P>(k.clover, Vh, i, sv);
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[c][q] = acc[c][q] + sv[c][q];
    } else {
      const A dg = (A)k.diag * ssc;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[c][q] = axpy_r(dg, sv[c][q], acc[c][q]);
    }
  }
  if (P == 0) {
#pragma unroll
    for (int c = 0; c < D; ++c) st_colour64(out, Vh, i, c, reinterpret_cast<const cx<double> *>(acc[c]));
  } else if (P == 1) {
#pragma unroll
    for (int c = 0; c < D; ++c) st_colour32(out, Vh, i, c, reinterpret_cast<const cx<float> *>(acc[c]));
  } else {
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) m = fmaxf(m, fmaxf(fabsf((float)acc[c][q].x), fabsf((float)acc[c][q].y)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<float> v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = mk((float)acc[c][q].x * inv, (float)acc[c][q].y * inv);
      st_colour16(out, Vh, i, c, v);
    }
    f16_scales_w(out, Vh, D)[i] = m;
  }
}

// Register budget variants (the autotuner picks one with the block size):
// MAXT x MINB = 256 x 1 (compiler's choice), 128 x 3 (up to ~170 registers: more
// loads in flight per thread), 64 x 12 (at most ~85 registers: more warps),
// 128 x 4 (at most 128 registers, between the two), and variant 4: the budget
// of 1 as a one-wave PERSIST launch (FP32; 1-2 % faster on 24^3 x 48).
// Programmatic dependent launch: every block lets the next kernel of the
// stream start launching, and waits for the previous kernel's results (it
// reads the fields that kernel wrote) before anything else; both are no-ops
// unless the kernels were launched with programmatic stream serialisation.
__device__ __forceinline__ void pdl_start() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// PERSIST: a grid of at most one wave of resident blocks, each block taking
// work items (tile, rhs) blockIdx.x, + gridDim.x, ... (the launcher sizes the
// grid so that every block gets the same number of items): no partly filled
// last wave, which on small lattices leaves SMs idle for a sizeable part of
// a launch of a few tens of microseconds.
template <int D, bool REAL, int P, int MAXT, int MINB, bool MASK = false, bool PERSIST = false>
__global__ void __launch_bounds__(MAXT, MINB) hop_kernel(HopK k, SkipK sk) {
  pdl_start();
  if constexpr (PERSIST) {
    const int64_t nwork = ((k.Vh + blockDim.x - 1) / blockDim.x) * k.nrhs;
    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
      const int rhs = (int)(w % k.nrhs);
      if (rhs_done(sk, rhs)) continue;
      const int64_t i = (w / k.nrhs) * blockDim.x + threadIdx.x;
      if (i < k.Vh) hop_site<D, REAL, P, MASK>(k, i, rhs);
    }
  } else {
    int64_t tile;
    int rhs;
    block_tile(k, tile, rhs);
    if (rhs_done(sk, rhs)) return;
    const int64_t i = tile * blockDim.x + threadIdx.x;
    if (i < k.Vh) hop_site<D, REAL, P, MASK>(k, i, rhs);
  }
}

// Persistent multi-lattice form: every block walks the work list (lattice,
// tile) with stride gridDim.x; each lattice brings its own descriptor
// (geometry, fields, links, epilogue).  A lattice whose `frozen` flag is set
// (its CG has converged) is skipped.
template <int D, bool REAL, int P>
__global__ void __launch_bounds__(256) hop_multi_kernel(const HopK *descs, const int2 *items, int nitems,
                                                        const int *frozen) {
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    if (frozen && frozen[it.x]) continue;
    const HopK k = descs[it.x];
    const int64_t i = (int64_t)it.y * blockDim.x + threadIdx.x;
    if (i < k.Vh) hop_site<D, REAL, P>(k, i, 0);
  }
}

static inline HopK make_hopk(const hr_lattice *lat, const HopArgs &a) {
  HopK k;
  k.out = a.out;
  k.in = a.in;
  k.self = a.self;
  k.links = a.links;
  k.rlinks = a.rlinks;
  k.clover = a.clover;
  k.T = lat->T;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.p = a.out_parity;
  k.mode = a.mode;
  k.nch = lat->nch_link;
  k.Vh = lat->Vh;
  k.stride = a.field_stride;
  k.sgn = a.dagger ? -1.0 : 1.0;
  k.coef = a.coef;
  k.diag = a.diag;
  k.nrhs = a.nrhs;
  k.tmask = a.tmask;
  return k;
}

// launch one site-kernel instance; pdl: programmatic stream serialisation (the
// kernel may start while the previous one on the stream finishes)
template <typename Kern>
static void launch_pdl(Kern kern, const HopK &k, SkipK sk, dim3 grid, int bs, cudaStream_t st, int pdl) {
  if (!pdl) {
    kern<<<grid, bs, 0, st>>>(k, sk);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(bs);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, k, sk);
}

// Grid of a PERSIST launch for `nwork` items: the fewest full waves of
// resident blocks, spread so that every block gets the same number of items
// (within one).  Resident blocks per SM are looked up once per kernel, block
// size and device.
template <typename Kern>
static dim3 persist_grid(Kern kern, int bs, unsigned nwork) {
  static int cache[8][9] = {};  // [device][bs / 32], bs = 32 ... 256
  static int sms_of[8] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int b = bs / 32;
  int per_sm = 1, sms = 1;
  if (dev >= 0 && dev < 8 && b >= 1 && b <= 8) {
    if (!cache[dev][b]) {
      int n = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, bs, 0) != cudaSuccess || n < 1) n = 1;
      cache[dev][b] = n;
    }
    if (!sms_of[dev]) {
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
      sms_of[dev] = n;
    }
    per_sm = cache[dev][b];
    sms = sms_of[dev];
  }
  const unsigned cap = (unsigned)(per_sm * sms);
  const unsigned waves = (nwork + cap - 1) / cap;
  return dim3(waves ? (nwork + waves - 1) / waves : 1u);
}

template <int D, bool REAL, int P>
static void launch_site(const HopK &k, SkipK sk, dim3 grid, int bs, int variant, cudaStream_t st, int pdl) {
  if (k.tmask) launch_pdl(hop_kernel<D, REAL, P, 256, 1, true>, k, sk, grid, bs, st, pdl);  // time-slab bulk pass
  else if (variant == 1) launch_pdl(hop_kernel<D, REAL, P, 128, 3>, k, sk, grid, bs, st, pdl);
  else if (variant == 2) launch_pdl(hop_kernel<D, REAL, P, 64, 12>, k, sk, grid, bs, st, pdl);
  else if (variant == 3) launch_pdl(hop_kernel<D, REAL, P, 128, 4>, k, sk, grid, bs, st, pdl);
  else if (variant == 4) {
    // one wave of resident blocks at the budget of variant 1 (FP32 only: on
    // FP16 fields it measured 5-20 % slower than the ordinary grid)
    if constexpr (P == 1) {
      auto kern = hop_kernel<D, REAL, P, 128, 3, false, true>;
      launch_pdl(kern, k, sk, persist_grid(kern, bs, grid.x), bs, st, pdl);
    }
  } else launch_pdl(hop_kernel<D, REAL, P, 256, 1>, k, sk, grid, bs, st, pdl);
}

// Launch the site-per-thread kernel for (D, REAL) of precision P with `bs`
// threads per block and register-budget variant 0 ... 4 (the autotuner picks).
template <int P>
int hop_dispatch(const hr_lattice *lat, const HopArgs &a, cudaStream_t st, int bs, int variant) {
  const HopK k = make_hopk(lat, a);
  const SkipK sk = make_skipk(a);
  dim3 grid((unsigned)(((lat->Vh + bs - 1) / bs) * a.nrhs));
  const int d = lat->d;
  if (lat->is_real) {
    switch (d) {
      case 3: launch_site<3, true, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 8: launch_site<8, true, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      default: return HR_ERR_UNSUPPORTED;
    }
  } else {
    switch (d) {
      case 2: launch_site<2, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 3: launch_site<3, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 4: launch_site<4, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 5: launch_site<5, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 6: launch_site<6, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 7: launch_site<7, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      case 8: launch_site<8, false, P>(k, sk, grid, bs, variant, st, a.pdl); break;
      default: return HR_ERR_UNSUPPORTED;
    }
  }
  return hr_check_launch("hop_kernel");
}
