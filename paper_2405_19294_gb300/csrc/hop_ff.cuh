// Float-float hopping stencil: one site per thread, every real a pair of
// FP32 numbers (cplx.cuh), for d_R <= 8.  Each hop_ff_*.cu translation unit
// instantiates some of the (d_R, real) classes (compiled in parallel).
//
// The eight hops run as a loop with the direction a run-time value, unlike the
// fully unrolled FP32 / FP16 / FP64 stencil (hop.cuh): a float-float stencil
// is about ten times the instructions of an FP32 one, and unrolled over the
// eight hops it no longer fits the instruction caches (measured: warps stalled
// about 8 cycles per issued instruction waiting for instructions).  The
// projection and reconstruction of hop.cuh's compile-time forms become
// selects on the direction: for direction mu, with sig = -+1 the sign of the
// hop,
//   h0 = psi0 - sig X psi_a,   h1 = psi1 + f1 sig X psi_b,
// a = 2 for mu in {t, z} else 3, b the other of {2, 3}, f1 = -1 for mu in
// {t, x} else +1, and X = 1 for mu in {t, y}, i for mu in {x, z}; and
//   acc0 += r0, acc1 += r1, acc2 += g2 sig X r_m, acc3 += g3 sig X r_n,
// with (m, n) = (0, 1) for mu in {t, z} else (1, 0), g2 = -1 for t else +1,
// g3 = +1 for x else -1.
#pragma once

#include "hop.cuh"

// b scaled by f = +-1 (exact), times i when odd
__device__ __forceinline__ cx<ff> ff_rot(cx<ff> b, float f, bool odd) {
  const ff bx = odd ? -b.y : b.x, by = odd ? b.x : b.y;
  return mk(mkff(f * bx.h, f * bx.l), mkff(f * by.h, f * by.l));
}

// The D x 4 complex float-float accumulator of one site: in registers, or
// (SMEM, complex d_R >= 5) in shared memory at [a * 4 + q][thread], so that
// the loop over the output rows a can stay rolled as well.  Unrolled over the
// rows, the d_R = 6 stencil with its clover epilogue again outgrew the
// instruction caches (stalled about 3 cycles per issued instruction waiting
// for instructions, 31 % issue).
template <int D, bool SMEM>
struct FfAcc;
template <int D>
struct FfAcc<D, false> {
  cx<ff> v[D][4];
  __device__ __forceinline__ cx<ff> &operator()(int a, int q) { return v[a][q]; }
};
template <int D>
struct FfAcc<D, true> {
  cx<ff> *base;  // this thread's element (0, 0); element (a, q) is stride * (4 a + q) further
  int stride;
  __device__ __forceinline__ cx<ff> &operator()(int a, int q) { return base[(a * 4 + q) * stride]; }
};
// complex d_R >= 5 keeps its accumulator in shared memory
template <int D, bool REAL>
__host__ __device__ constexpr bool ff_smem_acc() {
  return !REAL && D >= 5;
}
// dynamic shared memory of a block of bs threads
template <int D, bool REAL>
__host__ __device__ constexpr size_t ff_smem_bytes(int bs) {
  return ff_smem_acc<D, REAL>() ? (size_t)bs * D * 4 * sizeof(cx<ff>) : 0;
}

// acc = B acc for the two packed Hermitian chiral blocks of the clover field
// at site i (A or A^{-1}), one block at a time in a loop (one copy of the
// block product's code)
template <int D, typename AccT>
__device__ __forceinline__ void ff_clover_inplace(const void *cl, int64_t Vh, int64_t i, AccT &acc) {
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    cx<ff> v[2 * D], w[2 * D];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
      for (int c = 0; c < D; ++c) v[s2 * D + c] = b ? acc(c, 2 + s2) : acc(c, s2);
    herm_apply<D, 3>(cl, Vh, i, b * 2 * D * D, v, w);
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (b) acc(c, 2 + s2) = w[s2 * D + c];
        else acc(c, s2) = w[s2 * D + c];
      }
  }
}

// w = B v as herm_apply does (one packed Hermitian 2d x 2d block), for even
// d_R with the matrix cut into 4 x 4 blocks and the loops over the blocks kept
// rolled: one copy of a diagonal block's and of an off-diagonal block's code
// instead of every entry unrolled.  The blocks of v and w are picked by selects
// (no run-time register indexing).  Sums run in another order than
// herm_apply's, so results differ by rounding only.
template <int D>
__device__ __forceinline__ void ff_herm_blocked(const void *cl, int64_t Vh, int64_t i, int off,
                                                const cx<ff> v[2 * D], cx<ff> w[2 * D]) {
  constexpr int n = 2 * D, NB = n / 4;
  static_assert(n % 4 == 0, "4 x 4 blocks");
  auto gather = [&](const cx<ff> *x, int J, cx<ff> out[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cx<ff> t = x[q];
#pragma unroll
      for (int b = 1; b < NB; ++b)
        if (J == b) t = x[4 * b + q];
      out[q] = t;
    }
  };
  auto add_block = [&](int I, const cx<ff> d[4]) {
    cx<ff> t[4];
    gather(w, I, t);
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = t[q] + d[q];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (I == b) w[4 * b + q] = t[q];
  };
  auto chunk = [&](int r, int c) { return (int64_t)(off + D + r * (r - 1) / 2 + c) * Vh + i; };
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const cx<ff> dg = ld2<3>(cl, (int64_t)(off + q) * Vh + i);
    w[2 * q] = scale(dg.x, v[2 * q]);
    w[2 * q + 1] = scale(dg.y, v[2 * q + 1]);
  }
  // the strictly lower part of the diagonal blocks (I, I)
#pragma unroll 1
  for (int I = 0; I < NB; ++I) {
    cx<ff> vI[4], dI[4];
    gather(v, I, vI);
#pragma unroll
    for (int q = 0; q < 4; ++q) dI[q] = mk(ff(0), ff(0));
#pragma unroll
    for (int r = 1; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < r; ++c) {
        const cx<ff> a = ld2<3>(cl, chunk(4 * I + r, 4 * I + c));
        dI[r] = cfma(a, vI[c], dI[r]);
        dI[c] = cfmac(a, vI[r], dI[c]);
      }
    add_block(I, dI);
  }
  // the blocks (I, J) below the diagonal: w_I += B_IJ v_J, w_J += B_IJ^+ v_I
#pragma unroll 1
  for (int I = 1; I < NB; ++I)
#pragma unroll 1
    for (int J = 0; J < I; ++J) {
      cx<ff> vI[4], vJ[4], dI[4], dJ[4];
      gather(v, I, vI);
      gather(v, J, vJ);
#pragma unroll
      for (int q = 0; q < 4; ++q) dI[q] = dJ[q] = mk(ff(0), ff(0));
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const cx<ff> a = ld2<3>(cl, chunk(4 * I + r, 4 * J + c));
          dI[r] = cfma(a, vJ[c], dI[r]);
          dJ[c] = cfmac(a, vI[r], dJ[c]);
        }
      add_block(I, dI);
      add_block(J, dJ);
    }
}

// The clover blocks applied in place to a shared-memory accumulator (base,
// stride as FfAcc<D, true>): not inlined, so that the two places a launch may
// need it share one copy of the code; even d_R uses the blocked product.
template <int D>
__device__ __noinline__ void ff_clover_smem(const void *cl, int64_t Vh, int64_t i, cx<ff> *base, int stride) {
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    cx<ff> v[2 * D], w[2 * D];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
      for (int c = 0; c < D; ++c) v[s2 * D + c] = base[(c * 4 + 2 * b + s2) * stride];
    if constexpr (D % 2 == 0) ff_herm_blocked<D>(cl, Vh, i, b * 2 * D * D, v, w);
    else herm_apply<D, 3>(cl, Vh, i, b * 2 * D * D, v, w);
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
      for (int c = 0; c < D; ++c) base[(c * 4 + 2 * b + s2) * stride] = w[s2 * D + c];
  }
}
// smem: the block's dynamic shared memory (used when ff_smem_acc<D, REAL>())
template <int D, bool REAL>
__device__ __forceinline__ void hop_site_ff(const HopK &k, int64_t i, int rhs, unsigned char *smem) {
  constexpr bool SM = ff_smem_acc<D, REAL>();
  const size_t roff = (size_t)rhs * k.stride;
  const char *in = reinterpret_cast<const char *>(k.in) + roff;
  char *out = reinterpret_cast<char *>(k.out) + roff;
  const int64_t Vh = k.Vh;
  const int L = k.L, Lh = k.Lh, T = k.T, p = k.p;
  const Site s = site_of(i, p, L, Lh);
  const float sg = (float)k.sgn;  // +-1
  const int64_t slab = (int64_t)k.nch * Vh;
  const int64_t LLh = (int64_t)L * Lh;

  FfAcc<D, SM> acc;
  if constexpr (SM) {
    acc.base = reinterpret_cast<cx<ff> *>(smem) + threadIdx.x;
    acc.stride = (int)blockDim.x;
  }
  // the self term of the second launch first, divided by coef (a power of two
  // in every Schur and full-operator launch, so exactly): the hops then add
  // into it and the epilogue's scaling by coef gives A self + coef H with no
  // second D x 4 array live (which made the d_R = 6 clover kernel spill)
  if (k.mode == HOP_SELF) {
    const char *self = reinterpret_cast<const char *>(k.self) + roff;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<ff> v4[4];
      ld_colour<3>(self, Vh, i, c, v4);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc(c, q) = v4[q];
    }
    if (k.clover) {
      if constexpr (SM) ff_clover_smem<D>(k.clover, Vh, i, acc.base, acc.stride);
      else ff_clover_inplace<D>(k.clover, Vh, i, acc);
    }
    const ff f(k.clover ? 1.0 / k.coef : k.diag / k.coef);
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc(c, q) = scale(f, acc(c, q));
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc(c, q) = mk(ff(0), ff(0));
  }

#pragma unroll 1
  for (int n = 0; n < 8; ++n) {
    const int mu = n >> 1;
    const bool back = (n & 1) != 0;
    // neighbour j of site i along -+mu (as in hop.cuh)
    const int cc = mu == 0 ? s.t : (mu == 1 ? s.x : (mu == 2 ? s.y : s.z));
    const int E = mu == 0 ? T : L;
    const int cn = back ? (cc == 0 ? E - 1 : cc - 1) : (cc + 1 == E ? 0 : cc + 1);
    const int64_t st = mu == 0 ? (int64_t)L * LLh : (mu == 2 ? (int64_t)Lh : LLh);
    const int64_t j = mu == 1 ? i - (cc >> 1) + (cn >> 1) : i + (int64_t)(cn - cc) * st;
    // forward: U_mu(x) from the slot of parity p at i; backward: U_mu(x - mu)^+ at j
    const char *lk = reinterpret_cast<const char *>(k.links) + (size_t)(((back ? 1 - p : p) * 4 + mu) * slab) * 16u;
    const int64_t li = back ? j : i;
    const float sig = back ? sg : -sg;
    const bool odd = (mu & 1) != 0;
    const bool tz = mu == 0 || mu == 3;
    const float f1 = mu < 2 ? -sig : sig;
    const float g2 = mu == 0 ? -sig : sig, g3 = mu == 1 ? sig : -sig;

    cx<ff> h0[D], h1[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<ff> psi[4];
      ld_colour<3>(in, Vh, j, c, psi);
      const cx<ff> pa = tz ? psi[2] : psi[3], pb = tz ? psi[3] : psi[2];
      h0[c] = psi[0] + ff_rot(pa, -sig, odd);
      h1[c] = psi[1] + ff_rot(pb, f1, odd);
    }
    // row a of the link product, added to the accumulator as its 4 spins
    auto rebuild = [&](int a, const cx<ff> &r0, const cx<ff> &r1) {
      const cx<ff> rm = tz ? r0 : r1, rn = tz ? r1 : r0;
      acc(a, 0) = acc(a, 0) + r0;
      acc(a, 1) = acc(a, 1) + r1;
      acc(a, 2) = acc(a, 2) + ff_rot(rm, g2, odd);
      acc(a, 3) = acc(a, 3) + ff_rot(rn, g3, odd);
    };
    if constexpr (REAL) {
      // real links: chunk e >> 1, half e & 1 of entry e = a D + c (U^T backward)
      constexpr int NC = (D * D + 1) / 2;
      cx<ff> u[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) u[q] = ld2<3>(lk, (int64_t)q * Vh + li);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        cx<ff> r0 = mk(ff(0), ff(0)), r1 = mk(ff(0), ff(0));
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const int ef = a * D + c, eb = c * D + a;
          const ff uf = (ef & 1) ? u[ef >> 1].y : u[ef >> 1].x;
          const ff ub = (eb & 1) ? u[eb >> 1].y : u[eb >> 1].x;
          const ff ue = back ? ub : uf;
          r0 = rfma(ue, h0[c], r0);
          r1 = rfma(ue, h1[c], r1);
        }
        rebuild(a, r0, r1);
      }
    } else {
      // row a of U, or column a of U conjugated (U^+), loaded before the products
      auto row = [&](int a) {
        cx<ff> ur[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          ur[c] = ld2<3>(lk, (int64_t)(back ? c * D + a : a * D + c) * Vh + li);
          if (back) ur[c].y = -ur[c].y;
        }
        cx<ff> r0 = mk(ff(0), ff(0)), r1 = mk(ff(0), ff(0));
#pragma unroll
        for (int c = 0; c < D; ++c) {
          r0 = cfma(ur[c], h0[c], r0);
          r1 = cfma(ur[c], h1[c], r1);
        }
        rebuild(a, r0, r1);
      };
      if constexpr (SM) {
#pragma unroll 1
        for (int a = 0; a < D; ++a) row(a);
      } else {
#pragma unroll
        for (int a = 0; a < D; ++a) row(a);
      }
    }
  }

  // ---- epilogue: out = coef H (+ the self term folded in above), then
  // A^{-1} in place for the first launch of a Schur Dhat with clover ----
  const ff coef(k.coef);
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc(c, q) = scale(coef, acc(c, q));
  if (k.mode == HOP_SCALED && k.clover) {
    if constexpr (SM) ff_clover_smem<D>(k.clover, Vh, i, acc.base, acc.stride);
    else ff_clover_inplace<D>(k.clover, Vh, i, acc);
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    cx<ff> v4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v4[q] = acc(c, q);
    st_colour_ff(out, Vh, i, c, v4);
  }
}

template <int D, bool REAL, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) hop_ff_kernel(HopK k, SkipK sk) {
  extern __shared__ __align__(16) unsigned char ff_smem[];
  pdl_start();
  int64_t tile;
  int rhs;
  block_tile(k, tile, rhs);
  if (rhs_done(sk, rhs)) return;
  const int64_t i = tile * blockDim.x + threadIdx.x;
  if (i < k.Vh) hop_site_ff<D, REAL>(k, i, rhs, ff_smem);
}

// Persistent multi-lattice form (the batched solver's outer residuals): every
// block walks the work list of (lattice, tile) items with stride gridDim.x, as
// hop_multi_kernel does for the other precisions.
template <int D, bool REAL>
__global__ void __launch_bounds__(256, 1) hop_ff_multi_kernel(const HopK *descs, const int2 *items, int nitems,
                                                              const int *frozen) {
  extern __shared__ __align__(16) unsigned char ff_smem[];
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    if (frozen && frozen[it.x]) continue;
    const HopK k = descs[it.x];
    const int64_t i = (int64_t)it.y * blockDim.x + threadIdx.x;
    if (i < k.Vh) hop_site_ff<D, REAL>(k, i, 0, ff_smem);
  }
}

// (d_R, real links, launcher name) of every class built in float-float
#define HR_FF_CLASSES(X)                                                                               \
  X(2, false, hr_ff_c2) X(3, false, hr_ff_c3) X(3, true, hr_ff_r3) X(4, false, hr_ff_c4)             \
  X(5, false, hr_ff_c5) X(6, false, hr_ff_c6) X(7, false, hr_ff_c7) X(8, false, hr_ff_c8)             \
  X(8, true, hr_ff_r8)

// launch with the class's dynamic shared memory; pdl as in hop.cuh's launch_pdl
template <typename Kern>
static void launch_ff(Kern kern, const HopK &k, SkipK sk, dim3 grid, int bs, size_t smem, cudaStream_t st, int pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(bs);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, k, sk);
}

// register-budget variant 1 (128 threads x 3 blocks, about 168 registers)
// only where it does not spill: d_R <= 3
template <int D, bool REAL>
static void launch_site_ff(const HopK &k, SkipK sk, dim3 grid, int bs, int variant, cudaStream_t st, int pdl) {
  if constexpr (D <= 3) {
    if (variant == 1) {
      launch_ff(hop_ff_kernel<D, REAL, 128, 3>, k, sk, grid, bs, 0, st, pdl);
      return;
    }
  }
  launch_ff(hop_ff_kernel<D, REAL, 256, 1>, k, sk, grid, bs, ff_smem_bytes<D, REAL>(bs), st, pdl);
}

// NAME launches the class's site kernel; NAME##_multi returns its
// multi-lattice kernel
#define HR_FF_DEFINE(DD, RE, NAME)                                                                   \
  void NAME(const HopK &k, SkipK sk, dim3 grid, int bs, int variant, cudaStream_t st, int pdl) {   \
    launch_site_ff<DD, RE>(k, sk, grid, bs, variant, st, pdl);                                       \
  }                                                                                                  \
  const void *NAME##_multi() { return (const void *)hop_ff_multi_kernel<DD, RE>; }                  \
  size_t NAME##_smem(int bs) { return ff_smem_bytes<DD, RE>(bs); }
