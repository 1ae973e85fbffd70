// Hopping kernel for large representations with the output colour rows of
// U_R x half-spinor spread over the warps of a block and 32 consecutive sites
// over the lanes of each warp.
//
// Sec. 3.1.2 of the paper parallelises the represented-link product in the
// representation dimension once a one-site-per-thread kernel runs out of
// registers.  Here every warp owns R consecutive output rows a = w R ...
// w R + R - 1 for the same 32 sites.  The links are read from the rows layout
// (hr_rows_nch): the 8 matrices an output site needs -- U_R(x) and
// U_R(x - mu)^+ -- stored at the output site, row-major, so every link load of
// a warp reads one chunk row of 32 consecutive sites (256 B in FP32, fully
// coalesced, both halves of a real chunk used).  For each of the 8 neighbours:
//   1. warp w loads colours c = w R ... of psi(j) for its 32 sites, projects
//      them (Sec. 2.2) and stores h0[c], h1[c] to shared memory laid out
//      [colour][lane] (double-buffered per neighbour; colours up to a multiple
//      of the column batch CB, the pad kept at zero).  FP16 fields with real
//      links stage h0, h1 as half2, and the products are f16 x f16 -> f32
//      FMAs on the FP16 link entries;
//   2. one block barrier; then each warp walks the colours in batches of CB:
//      it first issues all R x CB link loads of the batch (independent, so
//      they are in flight together), then multiplies them with the staged
//      half-spinors, and finally rebuilds the 4 spin components.
// Rows past d_R (when R does not divide it) are clamped to row d_R - 1: their
// loads stay in bounds and their results are dropped.  One barrier per
// neighbour suffices: a warp that writes the buffer of neighbour n+2 has
// passed the barrier of n+1, which every warp reaches only after it has
// finished reading neighbour n.  No clover epilogue (the clover term is built
// for d_R <= 8, where the site kernel is used).  Also built in float-float
// (P = 3) for the mixed solvers' outer residuals: the direction already is a
// run-time loop variable, so the code stays within the instruction caches.
#pragma once

#include "hop.cuh"

template <int D, bool REAL, int R>
struct RowsGeom {
  static constexpr int W = (D + R - 1) / R;  // warps per block
  static constexpr int NT = 32 * W;           // threads per block
  // colours per load batch: the whole (padded) row for small d_R, else 8-16 loads per batch
  static constexpr int CB = REAL ? (R * hr_rows_dp(D, true) / 2 <= 24 ? hr_rows_dp(D, true) : (R <= 2 ? 16 : 8))
                                 : (R * D <= 36 ? D : (R <= 2 ? 8 : 4));
  static constexpr int DC = (D + CB - 1) / CB * CB;                        // staged colours (padded)
  static constexpr int DP = hr_rows_dp(D, REAL);
  static constexpr int NCH = hr_rows_nch(D, REAL);
  // neighbour table: per warp for blocks of 8 warps or more (no block-wide wait
  // at the start of a tile, which idles an SM that holds a single block), else
  // one table per block written by warp 0 behind a barrier (fewer registers,
  // and several resident blocks hide the wait)
  static constexpr bool WARP_NB = W >= 8;
  static constexpr int NB_TABLES = WARP_NB ? W : 1;
};

// bytes of dynamic shared memory: the double-buffered half-spinors plus, for
// FP16 output, one float per (warp, lane) for the per-site maximum
// (and, per warp, the 8 neighbour indices of the tile's 32 sites)
template <int D, bool REAL, int R, int P>
constexpr size_t rows_smem_bytes() {
  return (size_t)2 * 2 * RowsGeom<D, REAL, R>::DC * 32 * sizeof(cx<typename PT<P>::A>) +
         (P == 2 ? (size_t)RowsGeom<D, REAL, R>::W * 32 * 4 : 0) + (size_t)RowsGeom<D, REAL, R>::NB_TABLES * 8 * 32 * 4;
}

// r0[r] += V[a_r][c] h0[c], r1[r] += V[a_r][c] h1[c] over all colours, for
// this warp's rows a_r; `lk` is the chunk-row base of V_n, li the site index.
template <int D, bool REAL, int P, int R>
__device__ __forceinline__ void rows_mul(const cx<typename PT<P>::A> *hs, int lane, const int ar[R],
                                         const void *lk, int64_t li, int64_t Vh, cx<typename PT<P>::A> r0[R],
                                         cx<typename PT<P>::A> r1[R]) {
  typedef typename PT<P>::A A;
  typedef RowsGeom<D, REAL, R> G;
  constexpr int CB = G::CB;
  // chunk rows of row a_r start at rp[r]; colours past the row (the pad up to
  // a multiple of CB) read on into the next row or, after the last matrix, into
  // the zeroed slack of the layout, and meet h = 0
  constexpr int ROWCH = REAL ? G::DP / 2 : D;
  const void *rp[R];
#pragma unroll
  for (int r = 0; r < R; ++r)
    rp[r] = reinterpret_cast<const char *>(lk) + (size_t)(ar[r] * ROWCH) * (size_t)Vh * sizeof(typename PT<P>::S2) +
            (size_t)li * sizeof(typename PT<P>::S2);
#pragma unroll 1
  for (int c0 = 0; c0 < G::DC; c0 += CB) {
    if (REAL) {
      A u[R][CB];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < CB / 2; ++q) {
          const cx<A> v = ld2<P>(rp[r], (int64_t)((c0 >> 1) + q) * Vh);
          u[r][2 * q] = v.x;
          u[r][2 * q + 1] = v.y;
        }
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        const cx<A> h0 = hs[(2 * (c0 + cc)) * 32 + lane], h1 = hs[(2 * (c0 + cc) + 1) * 32 + lane];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          r0[r] = rfma(u[r][cc], h0, r0[r]);
          r1[r] = rfma(u[r][cc], h1, r1[r]);
        }
      }
    } else {
      cx<A> u[R][CB];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) u[r][cc] = ld2<P>(rp[r], (int64_t)(c0 + cc) * Vh);
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        const cx<A> h0 = hs[(2 * (c0 + cc)) * 32 + lane], h1 = hs[(2 * (c0 + cc) + 1) * 32 + lane];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          r0[r] = cfma(u[r][cc], h0, r0[r]);
          r1[r] = cfma(u[r][cc], h1, r1[r]);
        }
      }
    }
  }
}

// FP16 form of rows_mul for real links: the staged half-spinors are
// [colour][lane] uint2 = (h0, h1) as half2; the link entries stay FP16, and
// every product is an f16 x f16 -> f32 FMA
template <int D, bool REAL, int R>
__device__ __forceinline__ void rows_mul_f16(const uint2 *hs, int lane, const int ar[R], const void *lk, int64_t li,
                                             int64_t Vh, cx<float> r0[R], cx<float> r1[R]) {
  static_assert(REAL, "complex links take rows_mul");
  typedef RowsGeom<D, REAL, R> G;
  constexpr int CB = G::CB;
  constexpr int ROWCH = G::DP / 2;
  const unsigned *rp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) rp[r] = reinterpret_cast<const unsigned *>(lk) + (size_t)(ar[r] * ROWCH) * (size_t)Vh + li;
#pragma unroll 1
  for (int c0 = 0; c0 < G::DC; c0 += CB) {
    unsigned u[R][CB / 2];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int q = 0; q < CB / 2; ++q) u[r][q] = __ldg(rp[r] + (int64_t)((c0 >> 1) + q) * Vh);
#pragma unroll
    for (int cc = 0; cc < CB; ++cc) {
      const uint2 h = hs[(c0 + cc) * 32 + lane];
      const bool hi = (cc & 1) != 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        r0[r].x = fma_f16(u[r][cc >> 1], h.x, r0[r].x, hi, false);
        r0[r].y = fma_f16(u[r][cc >> 1], h.x, r0[r].y, hi, true);
        r1[r].x = fma_f16(u[r][cc >> 1], h.y, r1[r].x, hi, false);
        r1[r].y = fma_f16(u[r][cc >> 1], h.y, r1[r].y, hi, true);
      }
    }
  }
}

// Zero the pad colours D ... DC-1 of both half-spinor buffers; called once at
// kernel start, before the first tile's first barrier.  No tile writes them.
template <int D, bool REAL, int P, int R>
__device__ __forceinline__ void rows_zero_pads(unsigned char *smem) {
  typedef typename PT<P>::A A;
  typedef RowsGeom<D, REAL, R> G;
  constexpr int DC = G::DC;
  if constexpr (DC > D && P == 2 && REAL) {
    // FP16 with real links stages [colour][lane] uint2 = (h0, h1): zero from
    // colour D to the end of each buffer
    uint2 *sh = reinterpret_cast<uint2 *>(smem);
    constexpr int PER = 2 * DC * 32 - D * 32;  // uint2 entries per buffer from colour D on
    for (int e = threadIdx.x; e < 2 * PER; e += G::NT) {
      const int buf = e / PER, rem = e % PER;
      sh[buf * (2 * DC * 32) + D * 32 + rem] = make_uint2(0u, 0u);
    }
  } else if constexpr (DC > D) {
    cx<A> *sh = reinterpret_cast<cx<A> *>(smem);
    for (int e = threadIdx.x; e < 2 * 2 * (DC - D) * 32; e += G::NT) {
      const int buf = e / (2 * (DC - D) * 32), rem = e % (2 * (DC - D) * 32);
      sh[buf * (2 * DC * 32) + 2 * D * 32 + rem] = mk(A(0), A(0));
    }
  }
}

// One tile of 32 output sites of right-hand side rhs.  Every thread of the
// block must call it (block barriers inside).  `smem` holds rows_smem_bytes.
template <int D, bool REAL, int P, int R>
__device__ __forceinline__ void hop_rows_tile(const HopK &k, int64_t tile, int rhs, unsigned char *smem) {
  typedef typename PT<P>::A A;
  typedef RowsGeom<D, REAL, R> G;
  constexpr int W = G::W;
  constexpr int DC = G::DC;
  cx<A> *sh = reinterpret_cast<cx<A> *>(smem);  // [2][2 DC][32]
  // FP16 with real links: half2 staging and f16 x f16 -> f32 FMAs (the adjoint
  // classes ran 7-76 % faster).  Complex links convert to FP32 on load: with
  // four mixed FMAs per complex entry the large sym classes ran 9-27 % slower.
  constexpr bool F16MIX = (P == 2) && REAL;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int a0 = w * R;
  const int64_t i = tile * 32 + lane;
  const bool active = i < k.Vh;
  const int64_t ii = active ? i : 0;  // inactive lanes still join the barriers
  const size_t roff = (size_t)rhs * k.stride;
  const void *in = reinterpret_cast<const char *>(k.in) + roff;
  void *out = reinterpret_cast<char *>(k.out) + roff;
  const int64_t Vh = k.Vh;
  const int L = k.L, Lh = k.Lh, T = k.T, p = k.p;
  const Site s = site_of(ii, p, L, Lh);
  const A sg = (A)k.sgn;
  const int64_t slab = (int64_t)G::NCH * Vh;  // chunks per [p][n] matrix slot
  const size_t es = (P == 0 || P == 3) ? 16 : (P == 1 ? 8 : 4);
  const float *isc = (P == 2) ? f16_scales(in, Vh, D) : nullptr;
  int ar[R];  // this warp's rows, clamped to the last one
#pragma unroll
  for (int r = 0; r < R; ++r) ar[r] = (a0 + r < D) ? a0 + r : D - 1;

  cx<A> acc[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = mk(A(0), A(0));

  // the 8 neighbour indices of this lane's site ([n][lane]) in shared memory,
  // rather than in a per-thread array, which the runtime direction index would
  // put in local memory.  WARP_NB: each warp fills its own table (warp barrier
  // only); otherwise warp 0 fills the block's table behind a block barrier, and
  // refills it for the next tile only after that tile's last barrier, by which
  // time every warp has read its last entry.
  int *nbs = reinterpret_cast<int *>(smem + rows_smem_bytes<D, REAL, R, P>() - (size_t)G::NB_TABLES * 8 * 32 * 4) +
             (G::WARP_NB ? w * 8 * 32 : 0);
  if (G::WARP_NB || w == 0) {
    const int64_t LLh = (int64_t)L * Lh;
    const int tf = (s.t + 1 == T) ? 0 : s.t + 1, tb = (s.t == 0) ? T - 1 : s.t - 1;
    nbs[0 * 32 + lane] = (int)(ii + (int64_t)(tf - s.t) * L * LLh);
    nbs[1 * 32 + lane] = (int)(ii + (int64_t)(tb - s.t) * L * LLh);
    const int xf = (s.x + 1 == L) ? 0 : s.x + 1, xb = (s.x == 0) ? L - 1 : s.x - 1;
    nbs[2 * 32 + lane] = (int)(ii - (s.x >> 1) + (xf >> 1));
    nbs[3 * 32 + lane] = (int)(ii - (s.x >> 1) + (xb >> 1));
    const int yf = (s.y + 1 == L) ? 0 : s.y + 1, yb = (s.y == 0) ? L - 1 : s.y - 1;
    nbs[4 * 32 + lane] = (int)(ii + (int64_t)(yf - s.y) * Lh);
    nbs[5 * 32 + lane] = (int)(ii + (int64_t)(yb - s.y) * Lh);
    const int zf = (s.z + 1 == L) ? 0 : s.z + 1, zb = (s.z == 0) ? L - 1 : s.z - 1;
    nbs[6 * 32 + lane] = (int)(ii + (int64_t)(zf - s.z) * LLh);
    nbs[7 * 32 + lane] = (int)(ii + (int64_t)(zb - s.z) * LLh);
  }
  if (G::WARP_NB) __syncwarp();
  else __syncthreads();

#pragma unroll 1
  for (int n = 0; n < 8; ++n) {
    const int mu = n >> 1;
    const bool bwd = n & 1;
    const int64_t j = nbs[n * 32 + lane];
    const A sig = bwd ? sg : -sg;
    const A scl = (P == 2) ? (A)isc[j] : A(1);
    cx<A> *hs = sh + (n & 1) * (2 * DC * 32);
    // 1. project this warp's colours of psi(j) (FP16 with real links: in half2,
    // unscaled; the neighbour's site scale joins the reconstruction)
    if constexpr (F16MIX) {
      uint2 *hu = reinterpret_cast<uint2 *>(hs);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = a0 + r;
        if (c < D) {
          const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in) + (int64_t)c * Vh + j);
          uint2 h;
          switch (mu) {
            case 0: project_h2<0>(sig, v, h.x, h.y); break;
            case 1: project_h2<1>(sig, v, h.x, h.y); break;
            case 2: project_h2<2>(sig, v, h.x, h.y); break;
            default: project_h2<3>(sig, v, h.x, h.y); break;
          }
          hu[c * 32 + lane] = h;
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = a0 + r;
        if (c < D) {
          cx<A> psi[4], h0, h1;
          ld_colour<P>(in, Vh, j, c, psi);
          switch (mu) {
            case 0: project<0>(sig, psi, h0, h1); break;
            case 1: project<1>(sig, psi, h0, h1); break;
            case 2: project<2>(sig, psi, h0, h1); break;
            default: project<3>(sig, psi, h0, h1); break;
          }
          if (P == 2) {
            h0 = scale(scl, h0);
            h1 = scale(scl, h1);
          }
          hs[(2 * c) * 32 + lane] = h0;
          hs[(2 * c + 1) * 32 + lane] = h1;
        }
      }
    }
    __syncthreads();
    // 2. this warp's rows of V_n h: V_n = U_R(x) (forward) or U_R(x - mu)^+
    // (backward), both stored at the output site in the rows layout
    const void *lk = reinterpret_cast<const char *>(k.rlinks) + (size_t)((p * 8 + n) * slab) * es;
    cx<A> r0[R], r1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) r0[r] = r1[r] = mk(A(0), A(0));
    if constexpr (F16MIX) rows_mul_f16<D, REAL, R>(reinterpret_cast<const uint2 *>(hs), lane, ar, lk, ii, Vh, r0, r1);
    else rows_mul<D, REAL, P, R>(hs, lane, ar, lk, ii, Vh, r0, r1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (a0 + r < D) {
        if constexpr (F16MIX) {
          switch (mu) {
            case 0: reconstruct_w<0>(sig, scl, r0[r], r1[r], acc[r]); break;
            case 1: reconstruct_w<1>(sig, scl, r0[r], r1[r], acc[r]); break;
            case 2: reconstruct_w<2>(sig, scl, r0[r], r1[r], acc[r]); break;
            default: reconstruct_w<3>(sig, scl, r0[r], r1[r], acc[r]); break;
          }
        } else {
          switch (mu) {
            case 0: reconstruct<0>(sig, r0[r], r1[r], acc[r]); break;
            case 1: reconstruct<1>(sig, r0[r], r1[r], acc[r]); break;
            case 2: reconstruct<2>(sig, r0[r], r1[r], acc[r]); break;
            default: reconstruct<3>(sig, r0[r], r1[r], acc[r]); break;
          }
        }
      }
    }
  }

  // ---- epilogue (no clover) ----
  const A coef = (A)k.coef;
  const void *self = (k.mode == HOP_SELF) ? reinterpret_cast<const char *>(k.self) + roff : nullptr;
  const A ssc = (P == 2 && self) ? (A)f16_scales(self, Vh, D)[ii] : A(1);
  const A dg = (A)k.diag;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int c = a0 + r;
    if (c < D) {
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][q] = scale(coef, acc[r][q]);
      if (self) {
        cx<A> sv[4];
        ld_colour<P>(self, Vh, ii, c, sv);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = axpy_r(dg * ssc, sv[q], acc[r][q]);
      }
    }
  }
  if constexpr (P == 2) {
    // per-site maximum over all D colours: this warp's rows, then across warps
    float *red = reinterpret_cast<float *>(smem + (size_t)2 * 2 * DC * 32 * sizeof(cx<A>));
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (a0 + r < D)
#pragma unroll
        for (int q = 0; q < 4; ++q) m = fmaxf(m, fmaxf(fabsf((float)acc[r][q].x), fabsf((float)acc[r][q].y)));
    red[w * 32 + lane] = m;
    __syncthreads();
    m = 0.f;
#pragma unroll
    for (int v = 0; v < W; ++v) m = fmaxf(m, red[v * 32 + lane]);
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    if (active) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = a0 + r;
        if (c < D) {
          cx<float> v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = mk((float)acc[r][q].x * inv, (float)acc[r][q].y * inv);
          st_colour16(out, Vh, i, c, v);
        }
      }
      if (w == 0) f16_scales_w(out, Vh, D)[i] = m;
    }
  } else if (active) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = a0 + r;
      if (c < D) {
        if constexpr (P == 0) st_colour64(out, Vh, i, c, reinterpret_cast<const cx<double> *>(acc[r]));
        else if constexpr (P == 3) st_colour_ff(out, Vh, i, c, acc[r]);
        else st_colour32(out, Vh, i, c, reinterpret_cast<const cx<float> *>(acc[r]));
      }
    }
  }
}

template <int D, bool REAL, int P, int R>
__global__ void __launch_bounds__(RowsGeom<D, REAL, R>::NT) hop_rows_kernel(HopK k, SkipK sk) {
  extern __shared__ __align__(16) unsigned char rows_smem[];
  int64_t tile;
  int rhs;
  block_tile(k, tile, rhs);
  if (rhs_done(sk, rhs)) return;  // block-uniform: before any barrier
  rows_zero_pads<D, REAL, P, R>(rows_smem);
  hop_rows_tile<D, REAL, P, R>(k, tile, rhs, rows_smem);
}

// Persistent multi-lattice form (work list of (lattice, tile of 32 sites)).
// Between items no extra barrier is needed: an item writes buffer 0 first,
// last read at the previous item's neighbour 6, and every warp has passed
// that item's neighbour-7 barrier; the FP16 reduction array is rewritten only
// after 8 more barriers, by which time every warp has read it.
template <int D, bool REAL, int P, int R>
__global__ void __launch_bounds__(RowsGeom<D, REAL, R>::NT) hop_rows_multi_kernel(const HopK *descs, const int2 *items,
                                                                            int nitems, const int *frozen) {
  extern __shared__ __align__(16) unsigned char rows_smem[];
  rows_zero_pads<D, REAL, P, R>(rows_smem);
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    if (frozen && frozen[it.x]) continue;
    const HopK k = descs[it.x];
    hop_rows_tile<D, REAL, P, R>(k, it.y, 0, rows_smem);
  }
}

// Opt the instantiation into its dynamic shared memory (above 48 KB for FP64
// at large d_R) once per process.
template <typename F>
static int rows_smem_optin(F *fn, size_t bytes) {
  if (bytes <= 48 * 1024) return HR_OK;
  HR_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return HR_OK;
}
// the opt-in once per device and kernel (the attribute is per device)
template <typename F>
static int rows_smem_optin_once(F *fn, size_t bytes, unsigned long long &done) {
  int dev = 0;
  HR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev > 63) return HR_ERR_UNSUPPORTED;
  if ((done >> dev) & 1ull) return HR_OK;
  HR_TRY(rows_smem_optin(fn, bytes));
  done |= 1ull << dev;
  return HR_OK;
}

template <int D, bool REAL, int P, int R>
int launch_rows(const HopK &k, SkipK sk, int nrhs, cudaStream_t st) {
  constexpr size_t sm = rows_smem_bytes<D, REAL, R, P>();
  static unsigned long long done = 0;
  HR_TRY(rows_smem_optin_once(hop_rows_kernel<D, REAL, P, R>, sm, done));
  dim3 grid((unsigned)(((k.Vh + 31) / 32) * nrhs));
  hop_rows_kernel<D, REAL, P, R><<<grid, RowsGeom<D, REAL, R>::NT, sm, st>>>(k, sk);
  return hr_check_launch("hop_rows_kernel");
}

template <int P>
int rows_dispatch(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, int rows) {
  if (a.clover) return HR_ERR_UNSUPPORTED;
  if (!a.rlinks) return HR_ERR_STATE;
  const HopK k = make_hopk(lat, a);
  const SkipK sk = make_skipk(a);
  const int d = lat->d;
  const bool real = lat->is_real != 0;
#define HR_ROWS_CASE(DD, RE, RR) \
  if (d == DD && real == RE && rows == RR) return launch_rows<DD, RE, P, RR>(k, sk, a.nrhs, s);
  HR_ROWS_SHAPES(HR_ROWS_CASE)
#undef HR_ROWS_CASE
  return HR_ERR_UNSUPPORTED;
}

template <int P>
static const void *rows_multi_ptr(int d, int is_real, int rows, int *block, size_t *smem) {
  const bool real = is_real != 0;
#define HR_ROWS_CASE(DD, RE, RR)                                                  \
  if (d == DD && real == RE && rows == RR) {                                      \
    *block = RowsGeom<DD, RE, RR>::NT;                                            \
    *smem = rows_smem_bytes<DD, RE, RR, P>();                                     \
    static unsigned long long done = 0;                                             \
    const int opt = rows_smem_optin_once(hop_rows_multi_kernel<DD, RE, P, RR>, *smem, done); \
    return opt == HR_OK ? (const void *)hop_rows_multi_kernel<DD, RE, P, RR> : nullptr; \
  }
  HR_ROWS_SHAPES(HR_ROWS_CASE)
#undef HR_ROWS_CASE
  return nullptr;
}
