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
//   FP32 fields: the same m16n8k16 FP16 tiles on FP16 pairs x = hi + lo
//   (about 22 significant bits): the half-spinor rows of each (site, rhs,
//   hop) are first scaled by a power of two into the FP16 range, the link
//   entries (|U_ij| <= 1) need none, and U H ~ U_lo H_hi + U_hi H_lo + U_hi H_hi
//   (small terms first; the dropped U_lo H_lo is below 2^-22 of |U||H|) with
//   FP32 accumulation, which keeps the FP32 parity bound.
//
// Fragment layout (PTX mma, row.col, lane = 4 g + t):
//   A rows 0..7 = Re of output colour 0..7, rows 8..15 = Im;
//   A/B k index 0..7 = Re of input colour, 8..15 = Im;
//   B column n = 2 (rhs within the 4-rhs tile) + (half-spinor row);
//   C lane (g, t) = colour g, columns 2t, 2t+1 = rows h0, h1 of rhs t,
//   so each lane rebuilds the four spin rows of (colour g, rhs t) from its
//   own accumulator registers.
//
// Work split.  A block covers S = 16 consecutive output sites x R <= 12 rhs.
//   0. With clover, the packed A or A^{-1} blocks are staged by cp.async; for
//      FP16 fields so are the links of all 8 hops of the S sites (row-major per
//      site, so a warp reads one site's matrix from one shared-memory row).
//      FP32 fields, whose B rows take twice the space, read each lane's two
//      link entries from global memory one hop ahead.
//   Then, hop by hop (double-buffered, one barrier per hop):
//   1. one thread per (site, rhs) loads the neighbour spinor of the next hop
//      (coalesced: consecutive threads read consecutive sites), projects it
//      and writes the two half-spinor rows to shared memory in B-fragment
//      order;
//   2. each warp runs the MMA tiles of its two sites (three 4-rhs tiles each)
//      for the current hop from shared memory and rebuilds the spin rows into
//      its accumulator registers.
//   3. After the last hop the sums go through shared memory to one thread per
//      (site, rhs), which runs the epilogue of the multi-rhs kernel (scaling,
//      clover, self term, store).
#pragma once

#include "hop_mrhs.cuh"

namespace tc {

constexpr int S = 16;        // output sites per block
constexpr int NT = 256;      // threads per block
constexpr int NW = NT / 32;  // warps per block
constexpr int RMAX = 12;     // right-hand sides per block (three 4-rhs MMA tiles)
constexpr int RS = S + 1;    // sum staging: float2 stride between rhs (odd: conflict-free)

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

// ------------------------------------------------------------------------
// Phase 1: one thread per (site, rhs) loads the neighbour spinor of one hop
// (coalesced: consecutive threads read consecutive sites), projects it to the
// two half-spinor rows and writes them to shared memory as MMA B operands.
// B row layout (one row per fragment column n = 2 rhs + half-spinor row, RW
// 32-bit words; RW = 12 = 4 mod 8 keeps the 8 rows x 4 words of one fragment
// load on distinct banks):
//   FP32: Re h_0 .. Re h_{D-1}, Im h_0 .. Im h_{D-1}            (floats)
//   FP16: (Re h_0, Re h_1), (Re h_2, Re h_3), ... in words 0..3,
//         (Im h_0, Im h_1), ... in words 4..7                   (half2)
// Rows of one site are NCOL = 32 apart plus a pad of 4 words, so the 16 sites
// written by one warp spread over the banks.  Colours >= D (and the rhs
// beyond the block's) stay zero from the initial clear.
constexpr int NCOL = 2 * RMAX;  // B rows (fragment columns) per site
template <int P>
struct Rows {
  static constexpr int RW = (P == 1) ? 20 : 12;   // words per B row (4 mod 8)
  static constexpr int SSTR = NCOL * RW + 4;      // words per site
  static constexpr int BBUF = S * SSTR;           // words per buffer
};

// The neighbour spinor of one (site, rhs) as loaded for phase 1: 2D float4
// chunks (FP32) or D uint4 chunks (FP16).  Loading is split from projecting so
// that the loads of the next hop are in flight while the warp runs the MMA
// tiles of the current one.
template <int D, int P>
struct Nb {
  uint4 v[P == 1 ? 2 * D : D];
};
template <int D, int P>
__device__ __forceinline__ void nb_load(Nb<D, P> &nb, const char *f, int64_t Vh, int64_t j) {
  const uint4 *b = reinterpret_cast<const uint4 *>(f);
#pragma unroll
  for (int c = 0; c < (P == 1 ? 2 * D : D); ++c) nb.v[c] = __ldg(b + (int64_t)c * Vh + j);
}
// FP32 fields: the two rows are scaled by a common power of two and stored as
// FP16 pairs hi + lo (words 0..7 hi, 8..15 lo, each Re pairs then Im pairs);
// w receives the inverse scale.  FP16 fields: the stored codes (w untouched).
template <int D, int P, int MU>
__device__ __forceinline__ void project_store(const Nb<D, P> &nb, float sig, uint32_t *row0, uint32_t *row1,
                                              float &w) {
  if constexpr (P == 1) {
    cx<float> h0[D], h1[D];
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const uint4 a = nb.v[2 * c], b = nb.v[2 * c + 1];
      cx<float> psi[4];
      psi[0] = mk(__uint_as_float(a.x), __uint_as_float(a.y));
      psi[1] = mk(__uint_as_float(a.z), __uint_as_float(a.w));
      psi[2] = mk(__uint_as_float(b.x), __uint_as_float(b.y));
      psi[3] = mk(__uint_as_float(b.z), __uint_as_float(b.w));
      project<MU>(sig, psi, h0[c], h1[c]);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(h0[c].x), fabsf(h0[c].y)), fmaxf(fabsf(h1[c].x), fabsf(h1[c].y))));
    }
    // power-of-two scale 2^-e with m 2^-e in [0.5, 1): exact, and it brings both
    // rows into the FP16 range; the sum is multiplied back by 2^e
    int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 126;
    e = (m > 0.f) ? max(-100, min(100, e)) : 0;
    const float sc = __uint_as_float((unsigned)(127 - e) << 23);
    w = __uint_as_float((unsigned)(127 + e) << 23);
    // each value -> hi + lo, both FP16: hi = fp16(v), lo = fp16(v - hi)
    auto split = [&](float a, float b, unsigned &hi, unsigned &lo) {
      const __half2 h = __floats2half2_rn(a * sc, b * sc);
      const float2 f = __half22float2(h);
      hi = h2u(h);
      lo = h2u(__floats2half2_rn(fmaf(a, sc, -f.x), fmaf(b, sc, -f.y)));
    };
    unsigned w0[16], w1[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 2 * q, c1 = (c + 1 < D) ? c + 1 : 0;
      const bool v0 = c < D, v1 = c + 1 < D;
      const cx<float> a0 = v0 ? h0[v0 ? c : 0] : mk(0.f, 0.f), b0 = v1 ? h0[c1] : mk(0.f, 0.f);
      const cx<float> a1 = v0 ? h1[v0 ? c : 0] : mk(0.f, 0.f), b1 = v1 ? h1[c1] : mk(0.f, 0.f);
      split(a0.x, b0.x, w0[q], w0[8 + q]);      // Re, hi / lo
      split(a0.y, b0.y, w0[4 + q], w0[12 + q]);  // Im
      split(a1.x, b1.x, w1[q], w1[8 + q]);
      split(a1.y, b1.y, w1[4 + q], w1[12 + q]);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      reinterpret_cast<uint4 *>(row0)[v] = make_uint4(w0[4 * v], w0[4 * v + 1], w0[4 * v + 2], w0[4 * v + 3]);
      reinterpret_cast<uint4 *>(row1)[v] = make_uint4(w1[4 * v], w1[4 * v + 1], w1[4 * v + 2], w1[4 * v + 3]);
    }
  } else {
    unsigned h0[D], h1[D];
#pragma unroll
    for (int c = 0; c < D; ++c) project_h2<MU>(sig, nb.v[c], h0[c], h1[c]);
    unsigned w0[8], w1[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 2 * q;
      const __half2 z = __float2half2_rn(0.f);
      const __half2 a0 = (c < D) ? u2h(h0[c < D ? c : 0]) : z, b0 = (c + 1 < D) ? u2h(h0[c + 1 < D ? c + 1 : 0]) : z;
      const __half2 a1 = (c < D) ? u2h(h1[c < D ? c : 0]) : z, b1 = (c + 1 < D) ? u2h(h1[c + 1 < D ? c + 1 : 0]) : z;
      w0[q] = h2u(__lows2half2(a0, b0));
      w0[4 + q] = h2u(__highs2half2(a0, b0));
      w1[q] = h2u(__lows2half2(a1, b1));
      w1[4 + q] = h2u(__highs2half2(a1, b1));
    }
    reinterpret_cast<uint4 *>(row0)[0] = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    reinterpret_cast<uint4 *>(row0)[1] = make_uint4(w0[4], w0[5], w0[6], w0[7]);
    reinterpret_cast<uint4 *>(row1)[0] = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    reinterpret_cast<uint4 *>(row1)[1] = make_uint4(w1[4], w1[5], w1[6], w1[7]);
  }
}

// Phase 2, FP32 fields: the link entries of lane (g, t) -- U(g, 2t), U(g, 2t+1),
// or conj U(2t, g), conj U(2t+1, g) for the backward hop -- are read from the
// link slot in global memory one hop ahead (a_fetch) and split into FP16 pairs
// hi + lo (|U_ij| <= 1, so no scale is needed); rows g (Re out) and g+8 (Im
// out) against columns 2t, 2t+1 (Re in) and 2t+8, 2t+9 (Im in) as in the FP16
// tile.
struct AF32P {
  unsigned rh, ih, nh, rl, il, nl;  // (Re, Im, -Im) x (hi, lo)
};
template <int D, bool ADJ>
__device__ __forceinline__ void a_fetch(float2 (&u)[2], const float2 *slot, int64_t Vh, int64_t li, int g, int t) {
  u[0] = u[1] = make_float2(0.f, 0.f);
  if (g < D) {
    if (2 * t < D) u[0] = __ldg(slot + (int64_t)(ADJ ? 2 * t * D + g : g * D + 2 * t) * Vh + li);
    if (2 * t + 1 < D) u[1] = __ldg(slot + (int64_t)(ADJ ? (2 * t + 1) * D + g : g * D + 2 * t + 1) * Vh + li);
  }
}
template <bool ADJ>
__device__ __forceinline__ AF32P a_f32p(float2 u1, float2 u2) {
  if (ADJ) {
    u1.y = -u1.y;
    u2.y = -u2.y;
  }
  AF32P a;
  const __half2 rh = __floats2half2_rn(u1.x, u2.x), ih = __floats2half2_rn(u1.y, u2.y);
  const float2 rf = __half22float2(rh), imf = __half22float2(ih);
  const __half2 rl = __floats2half2_rn(u1.x - rf.x, u2.x - rf.y), il = __floats2half2_rn(u1.y - imf.x, u2.y - imf.y);
  a.rh = h2u(rh);
  a.ih = h2u(ih);
  a.nh = h2u(__hneg2(ih));
  a.rl = h2u(rl);
  a.il = h2u(il);
  a.nl = h2u(__hneg2(il));
  return a;
}
// U H ~ U_lo H_hi + U_hi H_lo + U_hi H_hi (small terms first; the dropped
// U_lo H_lo is below 2^-22 of |U||H|), FP32 accumulation; w = 2^e undoes the
// row scale of phase 1
template <int MU>
__device__ __forceinline__ void tile_f32p(cx<float> (&acc)[4], const AF32P &a, const uint32_t *rows, float w,
                                          float sig, int g, int t) {
  const uint32_t *row = rows + g * Rows<1>::RW;
  const unsigned bh0 = row[t], bh1 = row[4 + t], bl0 = row[8 + t], bl1 = row[12 + t];
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  mma_f16(c, a.rl, a.il, a.nl, a.rl, bh0, bh1);
  mma_f16(c, a.rh, a.ih, a.nh, a.rh, bl0, bl1);
  mma_f16(c, a.rh, a.ih, a.nh, a.rh, bh0, bh1);
  reconstruct_w<MU>(sig, w, mk(c[0], c[2]), mk(c[1], c[3]), acc);
}

// FP16 fields: the link entries as stored (half2), from the staged links
struct AF16 {
  unsigned ar, ai, an;
};
template <int D, bool ADJ>
__device__ __forceinline__ AF16 a_f16(const __half2 *lrow, int g, int t) {
  const __half2 z = __float2half2_rn(0.f);
  __half2 u1 = z, u2 = z;
  if (g < D) {
    if (2 * t < D) u1 = lrow[ADJ ? 2 * t * D + g : g * D + 2 * t];
    if (2 * t + 1 < D) u2 = lrow[ADJ ? (2 * t + 1) * D + g : g * D + 2 * t + 1];
  }
  // rows g (Re out) and g+8 (Im out) against columns 2t, 2t+1 (Re in) and 2t+8, 2t+9 (Im in)
  __half2 ai = __highs2half2(u1, u2);
  if (ADJ) ai = __hneg2(ai);
  AF16 a;
  a.ar = h2u(__lows2half2(u1, u2));
  a.ai = h2u(ai);
  a.an = h2u(__hneg2(ai));
  return a;
}

// bytes of the dynamic shared memory of one block
template <int D, int P, bool CLOVER>
struct Smem {
  static constexpr int NCH = D * D;
  static constexpr int ES = 4;                 // staged link chunk (half2; FP16 fields only)
  static constexpr int LST = NCH | 1;          // chunks per staged link row (odd: conflict-free fill)
  // FP16 fields stage the links of the 8 hops; FP32 fields read them per lane
  // from global memory (their B rows take twice the space)
  static constexpr size_t LINKS = (P == 2) ? (((size_t)8 * S * LST * ES + 15) & ~(size_t)15) : 0;
  static constexpr size_t BROWS = (size_t)2 * Rows<P>::BBUF * 4;  // two B buffers
  static constexpr size_t WSC = (size_t)2 * S * RMAX * 4;    // per-rhs row scales per buffer
  static constexpr size_t CLOV = CLOVER ? (size_t)4 * D * D * S * 8 : 0;
  static constexpr size_t NBI = (size_t)8 * S * sizeof(int64_t);
  // the staged sums (4D x es float2) reuse the link and B-row space after the last hop
  __host__ __device__ static size_t bytes(int es) {
    const size_t sums = (size_t)4 * D * es * 8;
    const size_t work = LINKS + BROWS > sums ? LINKS + BROWS : sums;
    return work + WSC + CLOV + NBI;
  }
  __host__ __device__ static size_t work(int es) {
    const size_t sums = (size_t)4 * D * es * 8;
    return LINKS + BROWS > sums ? LINKS + BROWS : sums;
  }
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
  constexpr int RW = Rows<P>::RW, SSTR = Rows<P>::SSTR, BBUF = Rows<P>::BBUF;
  extern __shared__ __align__(16) char smem[];
  char *lsm = smem;
  uint32_t *brows = reinterpret_cast<uint32_t *>(smem + M::LINKS);
  float2 *sums = reinterpret_cast<float2 *>(smem);  // after the last hop
  float *wsc = reinterpret_cast<float *>(smem + M::work(es));
  char *cbuf = smem + M::work(es) + M::WSC;
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
  for (int w = threadIdx.x; w < 2 * BBUF; w += NT) brows[w] = 0u;  // pads and unused rhs stay zero
  for (int w = threadIdx.x; w < 2 * S * RMAX; w += NT) wsc[w] = 0.f;
  __syncthreads();
  // stage the links of the 8 hops: hop n = 2 mu + back; forward: slot [p][mu] at
  // the output site, backward: slot [1-p][mu] at the backward neighbour
  {
    const int64_t slab = (int64_t)k.nch * Vh;
    const char *lk = reinterpret_cast<const char *>(k.links);
    for (int e = threadIdx.x; e < (P == 2 ? 8 * M::NCH * S : 0); e += NT) {
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

  // phase 1 item of this thread: site ps, rhs pq of the block
  const int ps = threadIdx.x % S, pq = threadIdx.x / S;
  const bool p1 = (pq < nr) && (i0 + ps < Vh);
  const char *pin = reinterpret_cast<const char *>(k.in) + (size_t)(rbase + (pq < nr ? pq : 0)) * k.stride;
  const float sg = (float)k.sgn;
  Nb<D, P> nb;
  float nbw = 0.f;  // FP16: the neighbour's site scale; FP32: the rows' inverse scale
  auto p1_load = [&](int n) {
    if (!p1) return;
    const int64_t j = nbi[n * S + ps];
    nb_load<D, P>(nb, pin, Vh, j);
    if (P == 2) nbw = f16_scales(pin, Vh, D)[j];
  };
  auto p1_store = [&](int n, int buf) {
    if (!p1) return;
    const float sig = (n & 1) ? sg : -sg;
    uint32_t *r0 = brows + buf * BBUF + ps * SSTR + (2 * pq) * RW;
    switch (n >> 1) {
      case 0: project_store<D, P, 0>(nb, sig, r0, r0 + RW, nbw); break;
      case 1: project_store<D, P, 1>(nb, sig, r0, r0 + RW, nbw); break;
      case 2: project_store<D, P, 2>(nb, sig, r0, r0 + RW, nbw); break;
      default: project_store<D, P, 3>(nb, sig, r0, r0 + RW, nbw); break;
    }
    wsc[buf * S * RMAX + ps * RMAX + pq] = nbw;
  };

  // phase 2: warp w owns sites 2w, 2w+1 of the tile and all NTILE 4-rhs tiles of
  // each (tiles beyond the block's rhs multiply zero rows; sites beyond V/2
  // compute on the rows of site 0 and are never stored)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  constexpr int NTILE = RMAX / 4;
  constexpr int SPW = S / NW;  // sites per warp
  cx<float> acc[SPW][NTILE][4];
#pragma unroll
  for (int a = 0; a < SPW; ++a)
#pragma unroll
    for (int q = 0; q < NTILE; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[a][q][r] = mk(0.f, 0.f);

  // FP32: the link entries of hop n + 1, fetched while hop n computes
  float2 ua[SPW][2], un[SPW][2];
  auto a_next = [&](int n) {
    const int mu = n >> 1, back = n & 1;
    const float2 *slot = reinterpret_cast<const float2 *>(k.links) + (size_t)(((back ? 1 - p : p) * 4 + mu) * (int64_t)k.nch * Vh);
#pragma unroll
    for (int a = 0; a < SPW; ++a) {
      const int s = SPW * warp + a;
      const int64_t li = (i0 + s < Vh) ? (back ? nbi[n * S + s] : i0 + s) : 0;
      if (back) a_fetch<D, true>(un[a], slot, Vh, li, g, t);
      else a_fetch<D, false>(un[a], slot, Vh, li, g, t);
    }
  };
  if (P == 1) {
    a_next(0);
#pragma unroll
    for (int a = 0; a < SPW; ++a) ua[a][0] = un[a][0], ua[a][1] = un[a][1];
  }
  p1_load(0);
  p1_store(0, 0);
  cp_async_wait<1>();  // the links are in (the clover may still be streaming)
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    __syncthreads();  // hop n's B rows are written; hop n-1's are no longer read
    if (P == 1 && n < 7) a_next(n + 1);
    if (n < 7) {  // FP16: the loads stay in flight during the MMA tiles of hop n
      p1_load(n + 1);
      if (P == 1) p1_store(n + 1, (n + 1) & 1);  // FP32: too many registers to hold them
    }
    const uint32_t *bb = brows + (n & 1) * BBUF;
    const float sig = (n & 1) ? sg : -sg;
#pragma unroll
    for (int a = 0; a < SPW; ++a) {
      const int s = SPW * warp + a;
      const char *lrow = lsm + (size_t)(n * S + s) * M::LST * M::ES;
      const uint32_t *rows = bb + s * SSTR;
      const float *wr = wsc + (n & 1) * S * RMAX + s * RMAX + t;
#define HR_TC_SITE(MU, ADJ)                                                                               \
  if (P == 1) {                                                                                           \
    const AF32P af = a_f32p<ADJ>(ua[a][0], ua[a][1]);                                                     \
    _Pragma("unroll") for (int q = 0; q < NTILE; ++q)                                                     \
      tile_f32p<MU>(acc[a][q], af, rows + q * 8 * RW, wr[4 * q], sig, g, t);                              \
  } else {                                                                                                \
    const AF16 af = a_f16<D, ADJ>(reinterpret_cast<const __half2 *>(lrow), g, t);                         \
    float c[NTILE][4];                                                                                    \
    _Pragma("unroll") for (int q = 0; q < NTILE; ++q) {                                                   \
      const uint32_t *row = rows + (q * 8 + g) * RW;                                                      \
      c[q][0] = c[q][1] = c[q][2] = c[q][3] = 0.f;                                                        \
      mma_f16(c[q], af.ar, af.ai, af.an, af.ar, row[t], row[4 + t]);                                      \
    }                                                                                                     \
    _Pragma("unroll") for (int q = 0; q < NTILE; ++q)                                                     \
      reconstruct_w<MU>(sig, wr[4 * q], mk(c[q][0], c[q][2]), mk(c[q][1], c[q][3]), acc[a][q]);           \
  }
      switch (n) {
        case 0: HR_TC_SITE(0, false) break;
        case 1: HR_TC_SITE(0, true) break;
        case 2: HR_TC_SITE(1, false) break;
        case 3: HR_TC_SITE(1, true) break;
        case 4: HR_TC_SITE(2, false) break;
        case 5: HR_TC_SITE(2, true) break;
        case 6: HR_TC_SITE(3, false) break;
        default: HR_TC_SITE(3, true) break;
      }
#undef HR_TC_SITE
    }
    if (n < 7 && P == 2) p1_store(n + 1, (n + 1) & 1);
    if (P == 1 && n < 7)
#pragma unroll
      for (int a = 0; a < SPW; ++a) ua[a][0] = un[a][0], ua[a][1] = un[a][1];
  }
  __syncthreads();  // the link and B-row space becomes the sum staging
  if (g < D) {
#pragma unroll
    for (int a = 0; a < SPW; ++a) {
      const int s = SPW * warp + a;
#pragma unroll
      for (int q = 0; q < NTILE; ++q) {
        const int r = 4 * q + t;
        if (r < nr)
#pragma unroll
          for (int sp = 0; sp < 4; ++sp)
            sums[(size_t)(g * 4 + sp) * es + r * RS + s] = make_float2(acc[a][q][sp].x, acc[a][q][sp].y);
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
  // the largest block size (R = RMAX) is opted in once per device
  static unsigned long long attr = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev > 63) return HR_ERR_CUDA;
  if (!((attr >> dev) & 1ull)) {
    const cudaError_t e = cudaFuncSetAttribute(hop_tc_kernel<D, P, CLOVER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Smem<D, P, CLOVER>::bytes(sum_stride(RMAX)));
    if (e != cudaSuccess) {
      hr_note_cuda_error(e, "cudaFuncSetAttribute(hop_tc_kernel)", __FILE__, __LINE__);
      return HR_ERR_CUDA;
    }
    attr |= 1ull << dev;
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
