// Multi-right-hand-side hopping kernel: one read of each link per site for
// all right-hand sides of a block.
//
// A block covers S consecutive output sites x R right-hand sides (thread t:
// site t % S, rhs t / S, so each warp reads runs of consecutive sites of one
// rhs -- coalesced).  For each direction mu the forward links U_R,mu(x) and the
// backward links U_R,mu(x - mu) of the block's S sites are staged once in
// shared memory (entry-major, conflict-free) and then used by all R
// right-hand-side threads of that site; the neighbour spinors are per rhs.
// Link traffic from L2 / HBM therefore drops by R compared with running the
// right-hand sides as separate blocks.  The arithmetic per (site, rhs) is the
// one-site-per-thread stencil of hop.cuh (same projection table, epilogue).
#pragma once

#include "hop.cuh"

template <bool REAL, typename A>
struct LinkEl {
  typedef cx<A> T;
};
template <typename A>
struct LinkEl<true, A> {
  typedef A T;
};

template <int D, bool REAL, int P, int MU, bool ADJ, int S>
__device__ __forceinline__ void hop_dir_smem(cx<typename PT<P>::A> acc[D][4], const void *in, int64_t Vh, int64_t j,
                                             const typename LinkEl<REAL, typename PT<P>::A>::T (*U)[S], int s,
                                             typename PT<P>::A sig, typename PT<P>::A scl) {
  typedef typename PT<P>::A A;
  cx<A> h0[D], h1[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    cx<A> psi[4];
    ld_colour<P>(in, Vh, j, c, psi);
    project<MU>(sig, psi, h0[c], h1[c]);
    if (P == 2) {
      h0[c] = scale(scl, h0[c]);
      h1[c] = scale(scl, h1[c]);
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<A> r0 = mk(A(0), A(0)), r1 = mk(A(0), A(0));
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int e = ADJ ? (c * D + a) : (a * D + c);
      if constexpr (REAL) {
        const A ue = U[e][s];
        r0 = rfma(ue, h0[c], r0);
        r1 = rfma(ue, h1[c], r1);
      } else {
        const cx<A> ue = U[e][s];
        if (ADJ) {
          r0 = cfmac(ue, h0[c], r0);
          r1 = cfmac(ue, h1[c], r1);
        } else {
          r0 = cfma(ue, h0[c], r0);
          r1 = cfma(ue, h1[c], r1);
        }
      }
    }
    reconstruct<MU>(sig, r0, r1, acc[a]);
  }
}

template <int D, bool REAL, int P, int S>
__global__ void __launch_bounds__(256) hop_mrhs_kernel(HopK k, int R) {
  typedef typename PT<P>::A A;
  typedef typename LinkEl<REAL, A>::T LE;
  __shared__ LE su[2][D * D][S];  // forward / backward links of one direction
  __shared__ int64_t nbi[8][S];    // neighbour indices of the block's sites
  const int s = threadIdx.x % S, q = threadIdx.x / S;
  const int nrb = (k.nrhs + R - 1) / R;
  const int64_t tile = blockIdx.x / nrb;
  const int rhs = (int)(blockIdx.x % nrb) * R + q;
  const int64_t i0 = tile * S;
  const int64_t i = i0 + s;
  const int64_t Vh = k.Vh;
  const int L = k.L, Lh = k.Lh, T = k.T, p = k.p;
  const bool active = (i < Vh) && (q < R) && (rhs < k.nrhs);
  if (threadIdx.x < S) {
    const int64_t ii = (i < Vh) ? i : 0;
    const Site st = site_of(ii, p, L, Lh);
    const int64_t LLh = (int64_t)L * Lh;
    const int tf = (st.t + 1 == T) ? 0 : st.t + 1, tb = (st.t == 0) ? T - 1 : st.t - 1;
    nbi[0][s] = ii + (int64_t)(tf - st.t) * L * LLh;
    nbi[1][s] = ii + (int64_t)(tb - st.t) * L * LLh;
    const int xf = (st.x + 1 == L) ? 0 : st.x + 1, xb = (st.x == 0) ? L - 1 : st.x - 1;
    nbi[2][s] = ii - (st.x >> 1) + (xf >> 1);
    nbi[3][s] = ii - (st.x >> 1) + (xb >> 1);
    const int yf = (st.y + 1 == L) ? 0 : st.y + 1, yb = (st.y == 0) ? L - 1 : st.y - 1;
    nbi[4][s] = ii + (int64_t)(yf - st.y) * Lh;
    nbi[5][s] = ii + (int64_t)(yb - st.y) * Lh;
    const int zf = (st.z + 1 == L) ? 0 : st.z + 1, zb = (st.z == 0) ? L - 1 : st.z - 1;
    nbi[6][s] = ii + (int64_t)(zf - st.z) * LLh;
    nbi[7][s] = ii + (int64_t)(zb - st.z) * LLh;
  }
  const size_t roff = (size_t)(rhs < k.nrhs ? rhs : 0) * k.stride;
  const void *in = reinterpret_cast<const char *>(k.in) + roff;
  void *out = reinterpret_cast<char *>(k.out) + roff;
  const A sg = (A)k.sgn;
  const int64_t slab = (int64_t)k.nch * Vh;
  const size_t es = (P == 0) ? 16 : (P == 1 ? 8 : 4);
  const float *isc = (P == 2) ? f16_scales(in, Vh, D) : nullptr;
  cx<A> acc[D][4];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[c][r] = mk(A(0), A(0));

#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    __syncthreads();  // neighbour indices ready / previous direction's links consumed
    const char *lf = reinterpret_cast<const char *>(k.links) + (size_t)((p * 4 + mu) * slab) * es;
    const char *lb = reinterpret_cast<const char *>(k.links) + (size_t)(((1 - p) * 4 + mu) * slab) * es;
    for (int e = threadIdx.x; e < 2 * D * D * S; e += blockDim.x) {
      const int side = e / (D * D * S), rem = e % (D * D * S), ent = rem / S, ss = rem % S;
      if (i0 + ss < Vh) {
        const int64_t li = side == 0 ? i0 + ss : nbi[2 * mu + 1][ss];
        const char *lk = side == 0 ? lf : lb;
        if constexpr (REAL) {
          const cx<A> pr = ld2<P>(lk, (int64_t)(ent >> 1) * Vh + li);
          su[side][ent][ss] = (ent & 1) ? pr.y : pr.x;
        } else {
          su[side][ent][ss] = ld2<P>(lk, (int64_t)ent * Vh + li);
        }
      }
    }
    __syncthreads();
    if (active) {
      const int64_t jf = nbi[2 * mu][s], jb = nbi[2 * mu + 1][s];
      const A sf = (P == 2) ? (A)isc[jf] : A(1), sb = (P == 2) ? (A)isc[jb] : A(1);
      switch (mu) {
        case 0:
          hop_dir_smem<D, REAL, P, 0, false, S>(acc, in, Vh, jf, su[0], s, -sg, sf);
          hop_dir_smem<D, REAL, P, 0, true, S>(acc, in, Vh, jb, su[1], s, sg, sb);
          break;
        case 1:
          hop_dir_smem<D, REAL, P, 1, false, S>(acc, in, Vh, jf, su[0], s, -sg, sf);
          hop_dir_smem<D, REAL, P, 1, true, S>(acc, in, Vh, jb, su[1], s, sg, sb);
          break;
        case 2:
          hop_dir_smem<D, REAL, P, 2, false, S>(acc, in, Vh, jf, su[0], s, -sg, sf);
          hop_dir_smem<D, REAL, P, 2, true, S>(acc, in, Vh, jb, su[1], s, sg, sb);
          break;
        default:
          hop_dir_smem<D, REAL, P, 3, false, S>(acc, in, Vh, jf, su[0], s, -sg, sf);
          hop_dir_smem<D, REAL, P, 3, true, S>(acc, in, Vh, jb, su[1], s, sg, sb);
          break;
      }
    }
  }
  if (!active) return;
  // ---- epilogue (as hop_site) ----
  const A coef = (A)k.coef;
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[c][r] = scale(coef, acc[c][r]);
  if (k.mode == HOP_SCALED) {
    if (k.clover) clover_apply<D, P>(k.clover, Vh, i, acc);
  } else {
    const void *self = reinterpret_cast<const char *>(k.self) + roff;
    const A ssc = (P == 2) ? (A)f16_scales(self, Vh, D)[i] : A(1);
    cx<A> sv[D][4];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      ld_colour<P>(self, Vh, i, c, sv[c]);
      if (P == 2)
#pragma unroll
        for (int r = 0; r < 4; ++r) sv[c][r] = scale(ssc, sv[c][r]);
    }
    if (k.clover) {
      clover_apply<D, P>(k.clover, Vh, i, sv);
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = acc[c][r] + sv[c][r];
    } else {
      const A dg = (A)k.diag;
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = axpy_r(dg, sv[c][r], acc[c][r]);
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
      for (int r = 0; r < 4; ++r) m = fmaxf(m, fmaxf(fabsf((float)acc[c][r].x), fabsf((float)acc[c][r].y)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<float> v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = mk((float)acc[c][r].x * inv, (float)acc[c][r].y * inv);
      st_colour16(out, Vh, i, c, v);
    }
    f16_scales_w(out, Vh, D)[i] = m;
  }
}

template <int D, bool REAL, int P, int S>
int launch_mrhs_t(const HopK &k, cudaStream_t st) {
  const int R = (k.nrhs < 256 / S) ? k.nrhs : 256 / S;
  const int nrb = (k.nrhs + R - 1) / R;
  const int64_t tiles = (k.Vh + S - 1) / S;
  hop_mrhs_kernel<D, REAL, P, S><<<(unsigned)(tiles * nrb), S * R, 0, st>>>(k, R);
  return hr_check_launch("hop_mrhs_kernel");
}

// Multi-rhs launch for the one-site-per-thread classes (d_R <= 8), S sites per block.
template <int P>
int hop_mrhs_dispatch(const hr_lattice *lat, const HopArgs &a, cudaStream_t st, int S) {
  const HopK k = make_hopk(lat, a);
  const int d = lat->d;
#define MR(DD, RR)                                                  \
  return (S == 8) ? launch_mrhs_t<DD, RR, P, 8>(k, st)              \
                  : (S == 16 ? launch_mrhs_t<DD, RR, P, 16>(k, st)  \
                             : launch_mrhs_t<DD, RR, P, 32>(k, st))
  if (lat->is_real) {
    if (d == 3) MR(3, true);
    if (d == 8) MR(8, true);
  } else {
    if (d == 2) MR(2, false);
    if (d == 3) MR(3, false);
    if (d == 4) MR(4, false);
    if (d == 5) MR(5, false);
    if (d == 6) MR(6, false);
  }
#undef MR
  return HR_ERR_UNSUPPORTED;
}
