// Multi-right-hand-side hopping kernel: one read of each link (and clover
// block) per site for all right-hand sides of a block.
//
// A block covers S consecutive output sites x R right-hand sides (thread t:
// site t % S, rhs t / S, so each warp reads runs of consecutive sites of one
// rhs -- coalesced).  The links are staged in shared memory as raw storage
// chunks ([chunk][site], conflict-free) by asynchronous copies (cp.async),
// in a ring of three buffers by direction: while the block computes direction
// mu from one buffer, the forward and backward links of direction mu+1 (and,
// during the last direction, the clover blocks of the epilogue) stream into
// the next.  With three buffers the one being refilled was last read two
// directions earlier, before the barrier every thread passed at the start of
// the previous direction, so one barrier per direction suffices.
// Link and clover traffic from L2 / HBM therefore drops by R compared with
// running the right-hand sides as separate blocks, and the staging latency
// hides behind the arithmetic.  The arithmetic per (site, rhs) is the
// one-site-per-thread stencil of hop.cuh (same projection table, epilogue).
#pragma once

#include "hop.cuh"

__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
  else if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// chunk k of site s from a staged [chunk][S] array of storage type, converted
template <int P, int S>
__device__ __forceinline__ cx<typename PT<P>::A> sm2(const char *base, int k, int s) {
  if constexpr (P == 0) {
    const double2 v = reinterpret_cast<const double2 *>(base)[k * S + s];
    return mk(v.x, v.y);
  } else if constexpr (P == 1) {
    const float2 v = reinterpret_cast<const float2 *>(base)[k * S + s];
    return mk(v.x, v.y);
  } else {
    const float2 v = __half22float2(reinterpret_cast<const __half2 *>(base)[k * S + s]);
    return mk(v.x, v.y);
  }
}

template <int D, bool REAL, int P, int MU, bool ADJ, int S>
__device__ __forceinline__ void hop_dir_staged(cx<typename PT<P>::A> acc[D][4], const void *in, int64_t Vh, int64_t j,
                                               const char *U, int s, typename PT<P>::A sig,
                                               typename PT<P>::A scl) {
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
      if (REAL) {
        const cx<A> pr = sm2<P, S>(U, e >> 1, s);
        const A ue = (e & 1) ? pr.y : pr.x;
        r0 = rfma(ue, h0[c], r0);
        r1 = rfma(ue, h1[c], r1);
      } else {
        const cx<A> ue = sm2<P, S>(U, e, s);
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

// w = B_b v for chiral block b of the packed Hermitian blocks staged as
// [chunk][S] (FP64 chunks for FP64 fields, FP32 otherwise); v[sp * D + c] is
// spin 2b + sp, colour c
template <int D, int P, int S>
__device__ __forceinline__ void clover_block_staged(const char *cl, int s, int b, const cx<typename PT<P>::A> v[2 * D],
                                                    cx<typename PT<P>::A> w[2 * D]) {
  constexpr int PC = (P == 0) ? 0 : 1;
  const int off = b * 2 * D * D;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    const auto dg = sm2<PC, S>(cl, off + q, s);
    w[2 * q] = scale(dg.x, v[2 * q]);
    w[2 * q + 1] = scale(dg.y, v[2 * q + 1]);
  }
#pragma unroll
  for (int r = 1; r < 2 * D; ++r)
#pragma unroll
    for (int c = 0; c < r; ++c) {
      const auto a = sm2<PC, S>(cl, off + D + r * (r - 1) / 2 + c, s);
      w[r] = cfma(a, v[c], w[r]);
      w[c] = cfmac(a, v[r], w[c]);
    }
}

// acc <- B acc, one chiral block at a time
template <int D, int P, int S>
__device__ __forceinline__ void clover_apply_staged(const char *cl, int s, cx<typename PT<P>::A> acc[D][4]) {
  typedef typename PT<P>::A A;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    cx<A> v[2 * D], w[2 * D];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < D; ++c) v[sp * D + c] = acc[c][2 * b + sp];
    clover_block_staged<D, P, S>(cl, s, b, v, w);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < D; ++c) acc[c][2 * b + sp] = w[sp * D + c];
  }
}

// spins 2b, 2b+1 of colour c of site i of a spinor field
template <int P>
__device__ __forceinline__ void ld_half_colour(const void *f, int64_t Vh, int64_t i, int c, int b,
                                               cx<typename PT<P>::A> psi[2]) {
  if constexpr (P == 0) {
    const double2 *p = reinterpret_cast<const double2 *>(f);
    const double2 v0 = __ldg(p + (int64_t)(4 * c + 2 * b) * Vh + i);
    const double2 v1 = __ldg(p + (int64_t)(4 * c + 2 * b + 1) * Vh + i);
    psi[0] = mk(v0.x, v0.y);
    psi[1] = mk(v1.x, v1.y);
  } else if constexpr (P == 1) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(f) + (int64_t)(2 * c + b) * Vh + i);
    psi[0] = mk(a.x, a.y);
    psi[1] = mk(a.z, a.w);
  } else {
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(f) + ((int64_t)c * Vh + i) * 2 + b);
    const float2 f0 = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 f1 = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    psi[0] = mk(f0.x, f0.y);
    psi[1] = mk(f1.x, f1.y);
  }
}

// The epilogue of the multi-rhs kernels for output site i (tile slot s) of the
// right-hand side at byte offset roff: acc = coef * H, then HOP_SCALED
// (clover: A^{-1} acc) or HOP_SELF (acc + A self, or diag * self without
// clover), and the store; clover blocks staged in shared memory as
// [chunk][S] (as hop_site does from global memory).
template <int D, int P, int S, bool CLOVER>
__device__ __forceinline__ void mrhs_epilogue(const HopK &k, cx<typename PT<P>::A> (&acc)[D][4], const char *cbuf,
                                              int s, int64_t i, size_t roff) {
  typedef typename PT<P>::A A;
  const int64_t Vh = k.Vh;
  void *out = reinterpret_cast<char *>(k.out) + roff;
  const A coef = (A)k.coef;
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[c][r] = scale(coef, acc[c][r]);
  if (k.mode == HOP_SCALED) {
    if (CLOVER) clover_apply_staged<D, P, S>(cbuf, s, acc);
  } else {
    const void *self = reinterpret_cast<const char *>(k.self) + roff;
    const A ssc = (P == 2) ? (A)f16_scales(self, Vh, D)[i] : A(1);
    if (CLOVER) {
      // acc += A self, chiral block by block (the self field is read in halves so
      // that only one block's input and output are live next to acc)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        cx<A> v[2 * D], w[2 * D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          cx<A> h[2];
          ld_half_colour<P>(self, Vh, i, c, b, h);
          v[c] = (P == 2) ? scale(ssc, h[0]) : h[0];
          v[D + c] = (P == 2) ? scale(ssc, h[1]) : h[1];
        }
        clover_block_staged<D, P, S>(cbuf, s, b, v, w);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
          for (int c = 0; c < D; ++c) acc[c][2 * b + sp] = acc[c][2 * b + sp] + w[sp * D + c];
      }
    } else {
      const A dg = (A)k.diag;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        cx<A> sv[4];
        ld_colour<P>(self, Vh, i, c, sv);
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = axpy_r(dg, (P == 2) ? scale(ssc, sv[r]) : sv[r], acc[c][r]);
      }
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

// FP32 / FP16 kernels of d_R = 6 are held to 128 registers (two 256-thread
// blocks' worth per SM), which their clover epilogue otherwise exceeds.  For
// the other classes 0 leaves the minimum unspecified, which compiles as the
// one-argument form; an explicit 1 had raised their register counts.
template <int D, int P>
constexpr int mrhs_min_blocks() { return (P != 0 && D == 6) ? 2 : 0; }

template <int D, bool REAL, int P, int S, bool CLOVER>
__global__ void __launch_bounds__(256, mrhs_min_blocks<D, P>()) hop_mrhs_kernel(HopK k, SkipK sk, int R) {
  typedef typename PT<P>::A A;
  constexpr int NCH = REAL ? (D * D + 1) / 2 : D * D;  // link chunks
  constexpr int ES = (P == 0) ? 16 : (P == 1 ? 8 : 4);  // bytes per link chunk
  constexpr int CES = (P == 0) ? 16 : 8;                // bytes per clover chunk
  constexpr int CCH = CLOVER ? 4 * D * D : 1;           // clover chunks per site (both blocks)
  __shared__ __align__(16) char lbuf[3][2][NCH * S * ES];  // [buffer][forward/backward]
  __shared__ __align__(16) char cbuf[CCH * S * CES];
  __shared__ int64_t nbi[8][S];
  const int s = threadIdx.x % S, q = threadIdx.x / S;
  const int nrb = (k.nrhs + R - 1) / R;
  const int64_t tile = blockIdx.x / nrb;
  const int rhs = (int)(blockIdx.x % nrb) * R + q;
  if (sk.rr) {  // the whole block returns only when every rhs it covers has converged
    const int r0 = (int)(blockIdx.x % nrb) * R;
    bool any = false;
    for (int qq = 0; qq < R && r0 + qq < k.nrhs; ++qq) any |= !rhs_done(sk, r0 + qq);
    if (!any) return;
  }
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
  __syncthreads();
  const int64_t slab = (int64_t)k.nch * Vh;
  // issue the asynchronous copies of direction mu's forward and backward links
  auto stage_links = [&](int mu, int buf) {
    const char *lf = reinterpret_cast<const char *>(k.links) + (size_t)((p * 4 + mu) * slab) * ES;
    const char *lb = reinterpret_cast<const char *>(k.links) + (size_t)(((1 - p) * 4 + mu) * slab) * ES;
    for (int e = threadIdx.x; e < 2 * NCH * S; e += blockDim.x) {
      const int side = e / (NCH * S), rem = e % (NCH * S), ch = rem / S, ss = rem % S;
      if (i0 + ss < Vh) {
        const int64_t li = side == 0 ? i0 + ss : nbi[2 * mu + 1][ss];
        const char *src = (side == 0 ? lf : lb) + ((size_t)ch * Vh + li) * ES;
        cp_async(&lbuf[buf][side][(ch * S + ss) * ES], src, ES);
      }
    }
  };
  auto stage_clover = [&]() {
    if (!CLOVER) return;
    const char *cl = reinterpret_cast<const char *>(k.clover);
    for (int e = threadIdx.x; e < CCH * S; e += blockDim.x) {
      const int ch = e / S, ss = e % S;
      if (i0 + ss < Vh) cp_async(&cbuf[(ch * S + ss) * CES], cl + ((size_t)ch * Vh + i0 + ss) * CES, CES);
    }
  };
  const size_t roff = (size_t)(rhs < k.nrhs ? rhs : 0) * k.stride;
  const void *in = reinterpret_cast<const char *>(k.in) + roff;
  const A sg = (A)k.sgn;
  const float *isc = (P == 2) ? f16_scales(in, Vh, D) : nullptr;
  cx<A> acc[D][4];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[c][r] = mk(A(0), A(0));

  stage_links(0, 0);
  cp_async_commit();
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (mu < 3) stage_links(mu + 1, (mu + 1) % 3);
    else stage_clover();
    cp_async_commit();
    cp_async_wait<1>();  // all but the group just issued: direction mu is in
    __syncthreads();
    if (active) {
      const int64_t jf = nbi[2 * mu][s], jb = nbi[2 * mu + 1][s];
      const A sf = (P == 2) ? (A)isc[jf] : A(1), sb = (P == 2) ? (A)isc[jb] : A(1);
      const char *uf = lbuf[mu % 3][0], *ub = lbuf[mu % 3][1];
      switch (mu) {
        case 0:
          hop_dir_staged<D, REAL, P, 0, false, S>(acc, in, Vh, jf, uf, s, -sg, sf);
          hop_dir_staged<D, REAL, P, 0, true, S>(acc, in, Vh, jb, ub, s, sg, sb);
          break;
        case 1:
          hop_dir_staged<D, REAL, P, 1, false, S>(acc, in, Vh, jf, uf, s, -sg, sf);
          hop_dir_staged<D, REAL, P, 1, true, S>(acc, in, Vh, jb, ub, s, sg, sb);
          break;
        case 2:
          hop_dir_staged<D, REAL, P, 2, false, S>(acc, in, Vh, jf, uf, s, -sg, sf);
          hop_dir_staged<D, REAL, P, 2, true, S>(acc, in, Vh, jb, ub, s, sg, sb);
          break;
        default:
          hop_dir_staged<D, REAL, P, 3, false, S>(acc, in, Vh, jf, uf, s, -sg, sf);
          hop_dir_staged<D, REAL, P, 3, true, S>(acc, in, Vh, jb, ub, s, sg, sb);
          break;
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  if (!active) return;
  mrhs_epilogue<D, P, S, CLOVER>(k, acc, cbuf, s, i, roff);
}

template <int D, bool REAL, int P, int S>
int launch_mrhs_t(const HopK &k, SkipK sk, cudaStream_t st) {
  const int R = (k.nrhs < 256 / S) ? k.nrhs : 256 / S;
  const int nrb = (k.nrhs + R - 1) / R;
  const int64_t tiles = (k.Vh + S - 1) / S;
  if (k.clover) hop_mrhs_kernel<D, REAL, P, S, true><<<(unsigned)(tiles * nrb), S * R, 0, st>>>(k, sk, R);
  else hop_mrhs_kernel<D, REAL, P, S, false><<<(unsigned)(tiles * nrb), S * R, 0, st>>>(k, sk, R);
  return hr_check_launch("hop_mrhs_kernel");
}

// S sites per block: 16 (8 for FP64, whose chunks are twice as large), and
// half that for d_R = 8, whose staged links and clover blocks are larger.
template <int D, bool REAL, int P>
int mrhs_pick(const HopK &k, SkipK sk, cudaStream_t st, int S) {
  constexpr int SMAX = (D == 8) ? (P == 0 ? 4 : 8) : (P == 0 ? 8 : 16);
  if (S >= SMAX) return launch_mrhs_t<D, REAL, P, SMAX>(k, sk, st);
  return launch_mrhs_t<D, REAL, P, (SMAX >= 8 ? SMAX / 2 : SMAX)>(k, sk, st);
}

// Multi-rhs launch for the one-site-per-thread classes (d_R <= 8).
template <int P>
int hop_mrhs_dispatch(const hr_lattice *lat, const HopArgs &a, cudaStream_t st, int S) {
  const HopK k = make_hopk(lat, a);
  const SkipK sk = make_skipk(a);
  const int d = lat->d;
  if (lat->is_real) {
    if (d == 3) return mrhs_pick<3, true, P>(k, sk, st, S);
    if (d == 8) return mrhs_pick<8, true, P>(k, sk, st, S);
  } else {
    if (d == 2) return mrhs_pick<2, false, P>(k, sk, st, S);
    if (d == 3) return mrhs_pick<3, false, P>(k, sk, st, S);
    if (d == 4) return mrhs_pick<4, false, P>(k, sk, st, S);
    if (d == 5) return mrhs_pick<5, false, P>(k, sk, st, S);
    if (d == 6) return mrhs_pick<6, false, P>(k, sk, st, S);
  }
  return HR_ERR_UNSUPPORTED;
}
