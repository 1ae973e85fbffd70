// Tensor-core multi-right-hand-side hopping kernel for complex representations
// with d_R <= 8: the link products of all right-hand sides of a block run as
// warp-level MMA tiles.
//
// For one output site and one of its 8 hops the stencil needs Y = U H, with U
// the d x d link (U_R,mu(x), or U_R,mu(x-mu)^+ for the backward hop) and H the
// projected half-spinors of every right-hand side as columns (two per rhs:
// the rows h0, h1 of the projection of Sec. 2.2).  In the real embedding
//     [Re Y]   [Re U  -Im U] [Re H]
//     [Im Y] = [Im U   Re U] [Im H]
// this is a (2d x 2d) by (2d x 2 nrhs) real product: with 2d <= 16 one
// 16 x 16 x 8 MMA tile covers four right-hand sides.  The link is the shared
// operand of the tile, so one link read per site serves every rhs.
//   FP16 fields: mma.m16n8k16 with FP16 operands (link entries, and the
//   projected half-spinor formed in FP16 from the stored codes as the site
//   kernel does) and FP32 accumulation -- the same roundings as the site
//   kernel's FP16 x FP16 -> FP32 multiply-adds; the neighbour's site scale is
//   applied in the reconstruction.
//   FP32 fields: mma.m16n8k8 on TF32 operands with the three-term split
//   x = big + small, big = tf32(x), small = tf32(x - big), and
//   U H ~ U_s H_b + U_b H_s + U_b H_b (small terms first); the dropped U_s H_s
//   is below 2^-22 of |U||H|, which keeps the FP32 parity bound.
//
// Fragment layout (PTX mma, row.col, lane = 4 g + t):
//   A rows 0..7 = Re of output colour 0..7, rows 8..15 = Im;
//   A/B k index 0..7 = Re of input colour, 8..15 = Im;
//   B column n = 2 (rhs within the 4-rhs tile) + (half-spinor row);
//   C lane (g, t) = colour g, columns 2t, 2t+1 = rows h0, h1 of rhs t,
//   so each lane rebuilds the four spin rows of (colour g, rhs t) from its
//   own accumulator registers.
// Lane (g, t) loads the neighbour components its B fragment needs -- colours
// t and t+4 (TF32) or 2t and 2t+1 (FP16) of one rhs, the two spin components
// of its half-spinor row only -- straight from global memory.
//
// Work split.  A block covers S = 16 consecutive output sites x R <= 16 rhs.
//   1. The links of all 8 hops of the S sites (row-major per site, so a warp
//      reads one site's matrix from one shared-memory row) and, with clover,
//      the packed A or A^{-1} blocks are staged by cp.async.
//   2. Each warp takes the sites of the tile in turn and runs the 8 hops of
//      one site with its sums in registers (4 rhs tiles x 4 spin rows).
//   3. The sums go through shared memory to one thread per (site, rhs), which
//      runs the epilogue of the multi-rhs kernel (scaling, clover, self term,
//      store).
#pragma once

#include "hop_mrhs.cuh"

namespace tc {

constexpr int S = 16;        // output sites per block
constexpr int NT = 256;      // threads per block
constexpr int NW = NT / 32;  // warps per block
constexpr int RMAX = 16;     // right-hand sides per block
constexpr int RS = S + 1;    // sum staging: float2 stride between rhs (odd: conflict-free)

__device__ __forceinline__ unsigned f2tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = big + small with both parts TF32
__device__ __forceinline__ void split_tf32(float x, unsigned &big, unsigned &small) {
  big = f2tf32(x);
  small = f2tf32(x - __uint_as_float(big));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_f16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                        unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Half-spinor row hh of the projection (1 + sig g_mu) psi for one colour:
// h_hh = psi_hh + f psi_k, with partner spin k and factor f = +-1 (MU = 0, 2)
// or +-i (MU = 1, 3) as in the projection table of hop.cuh:
//   MU=0: k = 2+hh, f = -sig     MU=1: k = 3-hh, f = -i sig
//   MU=2: k = 3-hh, f = (hh ? sig : -sig)     MU=3: k = 2+hh, f = i (hh ? sig : -sig)
template <int MU>
__device__ __forceinline__ int partner_spin(int hh) { return (MU == 0 || MU == 3) ? 2 + hh : 3 - hh; }
template <int MU>
__device__ __forceinline__ float partner_sign(int hh, float sig) { return (MU <= 1 || hh == 0) ? -sig : sig; }

// FP32 field: spin s of colour c sits in chunk 2c + s/2, half s%2 (float2)
template <int MU>
__device__ __forceinline__ cx<float> proj_f32(const char *f, int64_t Vh, int64_t j, int c, int hh, float fs) {
  const int k = partner_spin<MU>(hh);
  const float2 a = __ldg(reinterpret_cast<const float2 *>(f + (((int64_t)(2 * c) * Vh + j) << 4)) + hh);
  const float2 b = __ldg(reinterpret_cast<const float2 *>(f + (((int64_t)(2 * c + 1) * Vh + j) << 4)) + (k & 1));
  if (MU == 0 || MU == 2) return mk(fmaf(fs, b.x, a.x), fmaf(fs, b.y, a.y));
  return mk(fmaf(-fs, b.y, a.x), fmaf(fs, b.x, a.y));  // a + i fs b
}

// FP16 field: colour c is one 16-byte chunk of the four spins (half2 each);
// the row is formed in half2 arithmetic (one rounding, as the site kernel)
template <int MU>
__device__ __forceinline__ __half2 proj_f16(const char *f, int64_t Vh, int64_t j, int c, int hh, float fs) {
  const uint4 v = __ldg(reinterpret_cast<const uint4 *>(f) + (int64_t)c * Vh + j);
  const int k = partner_spin<MU>(hh);
  const unsigned a = hh ? v.y : v.x;
  const unsigned b = (k == 2) ? v.z : v.w;
  if (MU == 0 || MU == 2) return __hfma2(__float2half2_rn(fs), u2h(b), u2h(a));
  return __hfma2(__floats2half2_rn(-fs, fs), __lowhigh2highlow(u2h(b)), u2h(a));
}

// One hop of one site for every rhs tile of the block, FP32 fields (3xTF32).
// lrow: the staged link matrix (row-major, d*d float2) of this hop;
// acc[k][r]: spin row r of (colour g, rhs 4k + t).
template <int D, int MU, bool ADJ>
__device__ __forceinline__ void hop_f32(cx<float> (&acc)[4][4], const char *in, size_t stride, int64_t Vh,
                                        int64_t j, const float2 *lrow, float sig, int g, int t, int ntile,
                                        int nr) {
  float2 u1 = make_float2(0.f, 0.f), u2 = u1;
  if (g < D) {
    if (t < D) u1 = lrow[ADJ ? t * D + g : g * D + t];
    if (t + 4 < D) u2 = lrow[ADJ ? (t + 4) * D + g : g * D + t + 4];
  }
  if (ADJ) {
    u1.y = -u1.y;
    u2.y = -u2.y;
  }
  // k-step 0 (Re h columns): (Re u1, Im u1, Re u2, Im u2); k-step 1 (Im h): (-Im u1, Re u1, -Im u2, Re u2)
  unsigned xb1, xs1, yb1, ys1, xb2, xs2, yb2, ys2;
  split_tf32(u1.x, xb1, xs1);
  split_tf32(u1.y, yb1, ys1);
  split_tf32(u2.x, xb2, xs2);
  split_tf32(u2.y, yb2, ys2);
  const unsigned SB = 0x80000000u;  // sign flip (exact on TF32)
  const int hh = g & 1;
  const float fs = partner_sign<MU>(hh, sig);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= ntile) break;
    const int rb = 4 * k + (g >> 1);
    cx<float> h1 = mk(0.f, 0.f), h2 = h1;
    if (rb < nr) {
      const char *f = in + (size_t)rb * stride;
      if (t < D) h1 = proj_f32<MU>(f, Vh, j, t, hh, fs);
      if (t + 4 < D) h2 = proj_f32<MU>(f, Vh, j, t + 4, hh, fs);
    }
    unsigned rb1, rs1, rb2, rs2, ib1, is1, ib2, is2;
    split_tf32(h1.x, rb1, rs1);
    split_tf32(h2.x, rb2, rs2);
    split_tf32(h1.y, ib1, is1);
    split_tf32(h2.y, ib2, is2);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tf32(c, xs1, ys1, xs2, ys2, rb1, rb2);
    mma_tf32(c, xb1, yb1, xb2, yb2, rs1, rs2);
    mma_tf32(c, ys1 ^ SB, xs1, ys2 ^ SB, xs2, ib1, ib2);
    mma_tf32(c, yb1 ^ SB, xb1, yb2 ^ SB, xb2, is1, is2);
    mma_tf32(c, xb1, yb1, xb2, yb2, rb1, rb2);
    mma_tf32(c, yb1 ^ SB, xb1, yb2 ^ SB, xb2, ib1, ib2);
    reconstruct<MU>(sig, mk(c[0], c[2]), mk(c[1], c[3]), acc[k]);
  }
}

// The same for FP16 fields (one m16n8k16 tile per 4 rhs).
template <int D, int MU, bool ADJ>
__device__ __forceinline__ void hop_f16(cx<float> (&acc)[4][4], const char *in, size_t stride, int64_t Vh,
                                        int64_t j, const __half2 *lrow, float sig, int g, int t, int ntile,
                                        int nr) {
  const __half2 z = __float2half2_rn(0.f);
  __half2 u1 = z, u2 = z;
  if (g < D) {
    if (2 * t < D) u1 = lrow[ADJ ? 2 * t * D + g : g * D + 2 * t];
    if (2 * t + 1 < D) u2 = lrow[ADJ ? (2 * t + 1) * D + g : g * D + 2 * t + 1];
  }
  // rows g (Re out) and g+8 (Im out) against columns 2t, 2t+1 (Re in) and 2t+8, 2t+9 (Im in)
  const unsigned ar = h2u(__lows2half2(u1, u2));
  __half2 ai = __highs2half2(u1, u2);
  if (ADJ) ai = __hneg2(ai);
  const unsigned aiu = h2u(ai), ain = h2u(__hneg2(ai));
  const int hh = g & 1;
  const float fs = partner_sign<MU>(hh, sig);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k >= ntile) break;
    const int rb = 4 * k + (g >> 1);
    __half2 h1 = z, h2 = z;
    if (rb < nr) {
      const char *f = in + (size_t)rb * stride;
      if (2 * t < D) h1 = proj_f16<MU>(f, Vh, j, 2 * t, hh, fs);
      if (2 * t + 1 < D) h2 = proj_f16<MU>(f, Vh, j, 2 * t + 1, hh, fs);
    }
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_f16(c, ar, aiu, ain, ar, h2u(__lows2half2(h1, h2)), h2u(__highs2half2(h1, h2)));
    const int rd = 4 * k + t;  // the rhs this lane's accumulator columns belong to
    const float w = (rd < nr) ? f16_scales(in + (size_t)rd * stride, Vh, D)[j] : 0.f;
    reconstruct_w<MU>(sig, w, mk(c[0], c[2]), mk(c[1], c[3]), acc[k]);
  }
}

// bytes of the dynamic shared memory of one block: staged links, staged sums
// (4D x es float2), clover blocks, neighbour indices
template <int D, int P, bool CLOVER>
struct Smem {
  static constexpr int NCH = D * D;
  static constexpr int ES = (P == 1) ? 8 : 4;  // staged link chunk (float2 / half2)
  static constexpr int LST = NCH | 1;          // chunks per staged link row (odd: conflict-free fill)
  static constexpr size_t LINKS = ((size_t)8 * S * LST * ES + 15) & ~(size_t)15;
  static constexpr size_t CLOV = CLOVER ? (size_t)4 * D * D * S * 8 : 0;
  static constexpr size_t NBI = (size_t)8 * S * sizeof(int64_t);
  static size_t bytes(int es) { return LINKS + (size_t)4 * D * es * 8 + CLOV + NBI; }
};

// float2 stride between the spin/colour rows of the staged sums: >= R * RS and
// 1 mod 4, so that the lanes of one accumulator store hit distinct banks
static inline int sum_stride(int R) {
  int es = R * RS;
  while ((es & 3) != 1) ++es;
  return es;
}

template <int D, int P, bool CLOVER>
__global__ void __launch_bounds__(NT, 2) hop_tc_kernel(HopK k, SkipK sk, int R, int es) {
  typedef Smem<D, P, CLOVER> M;
  extern __shared__ __align__(16) char smem[];
  char *lsm = smem;
  float2 *sums = reinterpret_cast<float2 *>(smem + M::LINKS);
  char *cbuf = smem + M::LINKS + (size_t)4 * D * es * 8;
  int64_t *nbi = reinterpret_cast<int64_t *>(cbuf + M::CLOV);  // [8][S]

  const int nrb = (k.nrhs + R - 1) / R;
  const int64_t tile = blockIdx.x / nrb;
  const int rbase = (int)(blockIdx.x % nrb) * R;
  const int nr = (k.nrhs - rbase < R) ? k.nrhs - rbase : R;  // rhs of this block
  if (sk.rr) {  // the whole block returns only when every rhs it covers has converged
    bool any = false;
    for (int q = 0; q < nr; ++q) any |= !rhs_done(sk, rbase + q);
    if (!any) return;
  }
  const int64_t Vh = k.Vh;
  const int64_t i0 = tile * S;
  const int L = k.L, Lh = k.Lh, T = k.T, p = k.p;
  if (threadIdx.x < S) {
    const int s = threadIdx.x;
    const int64_t ii = (i0 + s < Vh) ? i0 + s : 0;
    const Site st = site_of(ii, p, L, Lh);
    const int64_t LLh = (int64_t)L * Lh;
    const int tf = (st.t + 1 == T) ? 0 : st.t + 1, tb = (st.t == 0) ? T - 1 : st.t - 1;
    nbi[0 * S + s] = ii + (int64_t)(tf - st.t) * L * LLh;
    nbi[1 * S + s] = ii + (int64_t)(tb - st.t) * L * LLh;
    const int xf = (st.x + 1 == L) ? 0 : st.x + 1, xb = (st.x == 0) ? L - 1 : st.x - 1;
    nbi[2 * S + s] = ii - (st.x >> 1) + (xf >> 1);
    nbi[3 * S + s] = ii - (st.x >> 1) + (xb >> 1);
    const int yf = (st.y + 1 == L) ? 0 : st.y + 1, yb = (st.y == 0) ? L - 1 : st.y - 1;
    nbi[4 * S + s] = ii + (int64_t)(yf - st.y) * Lh;
    nbi[5 * S + s] = ii + (int64_t)(yb - st.y) * Lh;
    const int zf = (st.z + 1 == L) ? 0 : st.z + 1, zb = (st.z == 0) ? L - 1 : st.z - 1;
    nbi[6 * S + s] = ii + (int64_t)(zf - st.z) * LLh;
    nbi[7 * S + s] = ii + (int64_t)(zb - st.z) * LLh;
  }
  __syncthreads();
  // stage the links of the 8 hops: hop n = 2 mu + back; forward: slot [p][mu] at
  // the output site, backward: slot [1-p][mu] at the backward neighbour
  {
    const int64_t slab = (int64_t)k.nch * Vh;
    const char *lk = reinterpret_cast<const char *>(k.links);
    for (int e = threadIdx.x; e < 8 * M::NCH * S; e += NT) {
      const int ss = e % S, rest = e / S, ch = rest % M::NCH, n = rest / M::NCH;
      if (i0 + ss >= Vh) continue;
      const int mu = n >> 1, back = n & 1;
      const int64_t li = back ? nbi[n * S + ss] : i0 + ss;
      const char *src = lk + ((size_t)(((back ? 1 - p : p) * 4 + mu) * slab) + (size_t)ch * Vh + li) * M::ES;
      cp_async(lsm + ((size_t)(n * S + ss) * M::LST + ch) * M::ES, src, M::ES);
    }
    cp_async_commit();
    if (CLOVER) {
      const char *cl = reinterpret_cast<const char *>(k.clover);
      for (int e = threadIdx.x; e < 4 * D * D * S; e += NT) {
        const int ch = e / S, ss = e % S;
        if (i0 + ss < Vh) cp_async(cbuf + (size_t)(ch * S + ss) * 8, cl + ((size_t)ch * Vh + i0 + ss) * 8, 8);
      }
    }
    cp_async_commit();
  }
  cp_async_wait<1>();  // the links are in (the clover may still be streaming)
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int ntile = (nr + 3) >> 2;
  const char *in = reinterpret_cast<const char *>(k.in) + (size_t)rbase * k.stride;
  const float sg = (float)k.sgn;
  for (int s = warp; s < S; s += NW) {
    if (i0 + s >= Vh) break;  // warp-uniform
    cx<float> acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[q][r] = mk(0.f, 0.f);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int64_t j = nbi[n * S + s];
      const char *lrow = lsm + (size_t)(n * S + s) * M::LST * M::ES;
      const float sig = (n & 1) ? sg : -sg;
#define HR_TC_HOP(MU, ADJ)                                                                                    \
  if (P == 1)                                                                                                 \
    hop_f32<D, MU, ADJ>(acc, in, k.stride, Vh, j, reinterpret_cast<const float2 *>(lrow), sig, g, t, ntile, nr); \
  else                                                                                                        \
    hop_f16<D, MU, ADJ>(acc, in, k.stride, Vh, j, reinterpret_cast<const __half2 *>(lrow), sig, g, t, ntile, nr);
      switch (n) {
        case 0: HR_TC_HOP(0, false) break;
        case 1: HR_TC_HOP(0, true) break;
        case 2: HR_TC_HOP(1, false) break;
        case 3: HR_TC_HOP(1, true) break;
        case 4: HR_TC_HOP(2, false) break;
        case 5: HR_TC_HOP(2, true) break;
        case 6: HR_TC_HOP(3, false) break;
        default: HR_TC_HOP(3, true) break;
      }
#undef HR_TC_HOP
    }
    if (g < D) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 4 * q + t;
        if (q < ntile && r < nr)
#pragma unroll
          for (int sp = 0; sp < 4; ++sp)
            sums[(size_t)(g * 4 + sp) * es + r * RS + s] = make_float2(acc[q][sp].x, acc[q][sp].y);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // epilogue: one thread per (site, rhs)
  for (int e = threadIdx.x; e < S * nr; e += NT) {
    const int s = e % S, q = e / S;
    const int64_t i = i0 + s;
    if (i >= Vh) continue;
    cx<float> a[D][4];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int sp = 0; sp < 4; ++sp) {
        const float2 v = sums[(size_t)(c * 4 + sp) * es + q * RS + s];
        a[c][sp] = mk(v.x, v.y);
      }
    mrhs_epilogue<D, P, S, CLOVER>(k, a, cbuf, s, i, (size_t)(rbase + q) * k.stride);
  }
}

template <int D, int P, bool CLOVER>
int launch(const HopK &k, SkipK sk, cudaStream_t st) {
  const int R = k.nrhs < RMAX ? k.nrhs : RMAX;
  const int nrb = (k.nrhs + R - 1) / R;
  const int64_t tiles = (k.Vh + S - 1) / S;
  const int es = sum_stride(R);
  const size_t smem = Smem<D, P, CLOVER>::bytes(es);
  static bool attr = false;  // the largest block size is set once (R <= RMAX)
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(hop_tc_kernel<D, P, CLOVER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Smem<D, P, CLOVER>::bytes(sum_stride(RMAX)));
    if (e != cudaSuccess) {
      hr_note_cuda_error(e, "cudaFuncSetAttribute(hop_tc_kernel)", __FILE__, __LINE__);
      return HR_ERR_CUDA;
    }
    attr = true;
  }
  hop_tc_kernel<D, P, CLOVER><<<(unsigned)(tiles * nrb), NT, smem, st>>>(k, sk, R, es);
  return hr_check_launch("hop_tc_kernel");
}

template <int D, int P>
int launch_d(const HopK &k, SkipK sk, cudaStream_t st) {
  return k.clover ? launch<D, P, true>(k, sk, st) : launch<D, P, false>(k, sk, st);
}

}  // namespace tc

// Tensor-core multi-rhs launch for precision P (1: FP32, 2: FP16) on the
// complex classes it is built for (d_R = 3 ... 6).
template <int P>
int hop_tc_dispatch(const hr_lattice *lat, const HopArgs &a, cudaStream_t st) {
  const HopK k = make_hopk(lat, a);
  const SkipK sk = make_skipk(a);
  if (lat->is_real) return HR_ERR_UNSUPPORTED;
  switch (lat->d) {
    case 3: return tc::launch_d<3, P>(k, sk, st);
    case 4: return tc::launch_d<4, P>(k, sk, st);
    case 5: return tc::launch_d<5, P>(k, sk, st);
    case 6: return tc::launch_d<6, P>(k, sk, st);
  }
  return HR_ERR_UNSUPPORTED;
}
