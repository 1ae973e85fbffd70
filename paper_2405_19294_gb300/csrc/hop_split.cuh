// Hopping kernel with the colour dimension split across a group of G threads
// per output site, for larger representations (d_R = 6 ... 35).
//
// The paper notes (Sec. 3.1.2) that a one-site-per-thread kernel spills
// registers once the represented link no longer fits, and parallelises the
// U_R x half-spinor product in the representation dimension instead (its
// LARGE_N kernel).  Here thread g of a group owns the output colour rows
// a = g, g + G, g + 2G, ...; for every one of the 8 neighbours
//   1. each thread loads its colours c (same distribution) of the neighbour
//      spinor, projects them (Sec. 2.2) and writes h0[c], h1[c] to shared
//      memory (double-buffered per neighbour);
//   2. after one warp barrier every thread multiplies its rows of U_R (or
//      columns, for U_R^+) with the full half-spinor read back from shared
//      memory (a broadcast within the group; colour outer, rows inner, so each
//      staged value is read once per thread) and rebuilds its 4 spin rows.
// Groups are aligned inside a warp (G divides 32), so only __syncwarp is used.
// Global loads stay coalesced: one load instruction covers 32/G consecutive
// sites for each of G chunk arrays.  No clover epilogue (clover is built for
// d_R <= 8, where the one-site-per-thread kernel is used).
#pragma once

#include "hop.cuh"
#include "hop_rows.cuh"

// One tile of 128/G output sites of right-hand side rhs; `sh` is the block's
// double-buffered half-spinor staging area.  Every lane of the block must
// call it (warp barriers inside).
template <int D, bool REAL, int P, int G>
__device__ __forceinline__ void hop_split_tile(const HopK &k, int64_t tile, int rhs,
                                               cx<typename PT<P>::A> (*sh)[128 / G][2 * D]) {
  typedef typename PT<P>::A A;
  constexpr int R = (D + G - 1) / G;      // rows per thread
  constexpr int SPB = 128 / G;            // sites per block
  const int g = threadIdx.x % G;
  const int sl = threadIdx.x / G;
  const int64_t i = tile * SPB + sl;
  const bool active = i < k.Vh;
  const int64_t ii = active ? i : 0;      // inactive lanes still join the warp barriers
  const size_t roff = (size_t)rhs * k.stride;
  const void *in = reinterpret_cast<const char *>(k.in) + roff;
  void *out = reinterpret_cast<char *>(k.out) + roff;
  const int64_t Vh = k.Vh;
  const int L = k.L, Lh = k.Lh, T = k.T, p = k.p;
  const Site s = site_of(ii, p, L, Lh);
  const A sg = (A)k.sgn;
  const int64_t slab = (int64_t)k.nch * Vh;
  const size_t es = (P == 0) ? 16 : (P == 1 ? 8 : 4);
  const float *isc = (P == 2) ? f16_scales(in, Vh, D) : nullptr;

  cx<A> acc[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = mk(A(0), A(0));

  const int64_t LLh = (int64_t)L * Lh;
  int64_t nb[8];
  {
    const int tf = (s.t + 1 == T) ? 0 : s.t + 1, tb = (s.t == 0) ? T - 1 : s.t - 1;
    nb[0] = ii + (int64_t)(tf - s.t) * L * LLh;
    nb[1] = ii + (int64_t)(tb - s.t) * L * LLh;
    const int xf = (s.x + 1 == L) ? 0 : s.x + 1, xb = (s.x == 0) ? L - 1 : s.x - 1;
    nb[2] = ii - (s.x >> 1) + (xf >> 1);
    nb[3] = ii - (s.x >> 1) + (xb >> 1);
    const int yf = (s.y + 1 == L) ? 0 : s.y + 1, yb = (s.y == 0) ? L - 1 : s.y - 1;
    nb[4] = ii + (int64_t)(yf - s.y) * Lh;
    nb[5] = ii + (int64_t)(yb - s.y) * Lh;
    const int zf = (s.z + 1 == L) ? 0 : s.z + 1, zb = (s.z == 0) ? L - 1 : s.z - 1;
    nb[6] = ii + (int64_t)(zf - s.z) * LLh;
    nb[7] = ii + (int64_t)(zb - s.z) * LLh;
  }

#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int mu = n >> 1;
    const bool bwd = n & 1;
    const int64_t j = nb[n];
    const A sig = bwd ? sg : -sg;
    const A scl = (P == 2) ? (A)isc[j] : A(1);
    cx<A> *hs = sh[n & 1][sl];
    // 1. project this thread's colours of psi(j)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = g + r * G;
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
        hs[2 * c] = h0;
        hs[2 * c + 1] = h1;
      }
    }
    __syncwarp();
    // 2. this thread's rows of U h (forward) or U^+ h (backward)
    const void *lk = reinterpret_cast<const char *>(k.links) +
                     (size_t)(((bwd ? 1 - p : p) * 4 + mu) * slab) * es;
    const int64_t li = bwd ? j : ii;
    // colour outer, this thread's rows inner: each staged h[c] is read once
    cx<A> r0[R], r1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) r0[r] = r1[r] = mk(A(0), A(0));
#pragma unroll 5
    for (int c = 0; c < D; ++c) {
      const cx<A> h0 = hs[2 * c], h1 = hs[2 * c + 1];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int a = g + r * G;
        if (a < D) {
          if (REAL) {
            const int e = bwd ? (c * D + a) : (a * D + c);
            const cx<A> pr = ld2<P>(lk, (int64_t)(e >> 1) * Vh + li);
            const A ue = (e & 1) ? pr.y : pr.x;
            r0[r] = rfma(ue, h0, r0[r]);
            r1[r] = rfma(ue, h1, r1[r]);
          } else if (bwd) {
            const cx<A> ue = ld2<P>(lk, (int64_t)(c * D + a) * Vh + li);
            r0[r] = cfmac(ue, h0, r0[r]);
            r1[r] = cfmac(ue, h1, r1[r]);
          } else {
            const cx<A> ue = ld2<P>(lk, (int64_t)(a * D + c) * Vh + li);
            r0[r] = cfma(ue, h0, r0[r]);
            r1[r] = cfma(ue, h1, r1[r]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (g + r * G < D) {
        switch (mu) {
          case 0: reconstruct<0>(sig, r0[r], r1[r], acc[r]); break;
          case 1: reconstruct<1>(sig, r0[r], r1[r], acc[r]); break;
          case 2: reconstruct<2>(sig, r0[r], r1[r], acc[r]); break;
          default: reconstruct<3>(sig, r0[r], r1[r], acc[r]); break;
        }
      }
    }
    // no second barrier: neighbour n+2 rewrites this buffer only after every
    // thread has passed the barrier of neighbour n+1, i.e. finished reading it
  }

  // ---- epilogue (no clover) ----
  const A coef = (A)k.coef;
  const void *self = (k.mode == HOP_SELF) ? reinterpret_cast<const char *>(k.self) + roff : nullptr;
  const A ssc = (P == 2 && self) ? (A)f16_scales(self, Vh, D)[ii] : A(1);
  const A dg = (A)k.diag;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int c = g + r * G;
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
  if (P == 2) {
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (g + r * G < D)
#pragma unroll
        for (int q = 0; q < 4; ++q) m = fmaxf(m, fmaxf(fabsf((float)acc[r][q].x), fabsf((float)acc[r][q].y)));
#pragma unroll
    for (int o = 1; o < G; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    if (active) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = g + r * G;
        if (c < D) {
          cx<float> v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = mk((float)acc[r][q].x * inv, (float)acc[r][q].y * inv);
          st_colour16(out, Vh, i, c, v);
        }
      }
      if (g == 0) f16_scales_w(out, Vh, D)[i] = m;
    }
  } else if (active) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = g + r * G;
      if (c < D) {
        if (P == 0) st_colour64(out, Vh, i, c, reinterpret_cast<const cx<double> *>(acc[r]));
        else st_colour32(out, Vh, i, c, reinterpret_cast<const cx<float> *>(acc[r]));
      }
    }
  }
}

template <int D, bool REAL, int P, int G>
__global__ void __launch_bounds__(128) hop_split_kernel(HopK k, SkipK sk) {
  __shared__ cx<typename PT<P>::A> sh[2][128 / G][2 * D];  // half-spinor per site, double buffered
  int64_t tile;
  int rhs;
  block_tile(k, tile, rhs);
  if (rhs_done(sk, rhs)) return;
  hop_split_tile<D, REAL, P, G>(k, tile, rhs, sh);
}

// Persistent multi-lattice form (work list of (lattice, tile), see hop_multi_kernel).
template <int D, bool REAL, int P, int G>
__global__ void __launch_bounds__(128) hop_split_multi_kernel(const HopK *descs, const int2 *items, int nitems,
                                                              const int *frozen) {
  __shared__ cx<typename PT<P>::A> sh[2][128 / G][2 * D];
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    if (frozen && frozen[it.x]) continue;
    const HopK k = descs[it.x];
    hop_split_tile<D, REAL, P, G>(k, it.y, 0, sh);
    __syncwarp();  // the next item reuses the staging buffers
  }
}

template <int D, bool REAL, int P, int G>
int launch_split(const HopK &k, SkipK sk, int nrhs, cudaStream_t st) {
  constexpr int SPB = 128 / G;
  dim3 grid((unsigned)(((k.Vh + SPB - 1) / SPB) * nrhs));
  hop_split_kernel<D, REAL, P, G><<<grid, 128, 0, st>>>(k, sk);
  return hr_check_launch("hop_split_kernel");
}

// Kernel entry of the persistent multi-lattice hop for (D, REAL, shape), and
// its block size; null when the shape does not exist for that d_R.
template <int P>
static const void *multi_kernel_ptr(int d, int is_real, HopShape sh, int *block) {
  *block = sh.split_g ? 128 : sh.bs;
  if (sh.split_g == 0) {
    if (is_real) {
      if (d == 3) return (const void *)hop_multi_kernel<3, true, P>;
      if (d == 8) return (const void *)hop_multi_kernel<8, true, P>;
    } else {
      if (d == 2) return (const void *)hop_multi_kernel<2, false, P>;
      if (d == 3) return (const void *)hop_multi_kernel<3, false, P>;
      if (d == 4) return (const void *)hop_multi_kernel<4, false, P>;
      if (d == 5) return (const void *)hop_multi_kernel<5, false, P>;
      if (d == 6) return (const void *)hop_multi_kernel<6, false, P>;
      if (d == 7) return (const void *)hop_multi_kernel<7, false, P>;
      if (d == 8) return (const void *)hop_multi_kernel<8, false, P>;
    }
    return nullptr;
  }
  const int g = sh.split_g;
  const bool real = is_real != 0;
#define HR_SPLIT_PTR(DD, RE, GG) \
  if (d == DD && real == RE && g == GG) return (const void *)hop_split_multi_kernel<DD, RE, P, GG>;
  HR_SPLIT_SHAPES(HR_SPLIT_PTR)
#undef HR_SPLIT_PTR
  return nullptr;
}

// Persistent launch: grid = min(work items, SMs x resident blocks per SM).
template <int P>
int hop_multi_launch(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                     const int *frozen, cudaStream_t s) {
  int block = 0;
  size_t smem = 0;
  const void *fn = sh.rows ? rows_multi_ptr<P>(d, is_real, sh.rows, &block, &smem)
                           : multi_kernel_ptr<P>(d, is_real, sh, &block);
  if (!fn) return HR_ERR_UNSUPPORTED;
  if (nitems <= 0) return HR_OK;
  int dev = 0, sms = 0, per_sm = 0;
  HR_CUDA(cudaGetDevice(&dev));
  HR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem));
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > nitems) grid = nitems;
  void *args[] = {(void *)&descs, (void *)&items, (void *)&nitems, (void *)&frozen};
  HR_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s));
  return HR_OK;
}
