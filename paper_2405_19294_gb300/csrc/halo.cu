// Time-slab domain decomposition of the even-odd operator: the halo-ready
// geometry of Sec. 2 (bulk sites plus receive buffers, masked directions,
// a send buffer filled from the boundary sites, half-spinors on the wire).
//
// A sub-domain lattice (hr_lattice_create_domain) holds the time slab
// [t0, t0 + T) of a T_global x L^3 lattice.  One hop of the even-odd
// operator on it runs in two parts:
//   begin: (1) fill the two send buffers from the input field's boundary
//          sites -- the bottom face (local t = 0) sends the projected
//          half-spinor (1 - g0 sign) psi, which the slab below multiplies by
//          its own U_0 for its forward hop; the top face (local t = T-1)
//          sends U_0^+ (1 + g0 sign) psi, already multiplied, which the slab
//          above only has to rebuild (the partial application before sending
//          that Sec. 2 describes);
//          (2) the bulk hop over every output site with the two t hops that
//          cross a face masked out (HopArgs::tmask in the site kernel);
//   end:   after the caller has exchanged the buffers (receive-up from the
//          slab above, receive-down from the slab below), add the masked
//          terms to the face sites of the output.
// The epilogues are linear (no clover on slabs), so adding the face terms
// afterwards gives the same operator.  Buffer layout: [rhs][2][d][L^3/2]
// complex (h0 then h1 per colour; face site f is the site of local
// checkerboard index t L^3/2 + f), FP64 for FP64 fields and FP32 otherwise.
#include <string.h>

#include "hop.cuh"

namespace {

struct HaloK {
  void *out;
  const void *in;
  const void *links;
  void *send_up, *send_down;
  const void *recv_up, *recv_down;
  int T, L, Lh, nrhs, q;  // q: parity of the field read (pack) or written (complete)
  int64_t Vh, Lf;
  size_t stride;           // bytes between rhs fields
  double sgn, coef;
};

template <int P>
struct HT {
  typedef float T;
};
template <>
struct HT<0> {
  typedef double T;
};

// halo element (rhs, half h, colour c, face site f)
template <int P>
__device__ __forceinline__ cx<typename HT<P>::T> *hel(void *b, const HaloK &k, int rhs, int h, int c, int64_t f,
                                                      int D) {
  return reinterpret_cast<cx<typename HT<P>::T> *>(b) + (((int64_t)rhs * 2 + h) * D + c) * k.Lf + f;
}

template <int D, bool REAL, int P>
__global__ void halo_pack_kernel(HaloK k) {
  typedef typename PT<P>::A A;
  typedef typename HT<P>::T H;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 2 * k.Lf * k.nrhs) return;
  const int64_t f = g % k.Lf;
  const int top = (int)((g / k.Lf) & 1);
  const int rhs = (int)(g / (2 * k.Lf));
  const void *in = reinterpret_cast<const char *>(k.in) + (size_t)rhs * k.stride;
  const int64_t i = (top ? (int64_t)(k.T - 1) * k.Lf : 0) + f;
  const A sg = (A)k.sgn;
  const A sig = top ? sg : -sg;  // the receiver's backward / forward t hop
  const A scl = (P == 2) ? (A)f16_scales(in, k.Vh, D)[i] : A(1);
  cx<A> h0[D], h1[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    cx<A> psi[4];
    ld_colour<P>(in, k.Vh, i, c, psi);
    project<0>(sig, psi, h0[c], h1[c]);
    if (P == 2) {
      h0[c] = scale(scl, h0[c]);
      h1[c] = scale(scl, h1[c]);
    }
  }
  if (!top) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      *hel<P>(k.send_down, k, rhs, 0, c, f, D) = mk((H)h0[c].x, (H)h0[c].y);
      *hel<P>(k.send_down, k, rhs, 1, c, f, D) = mk((H)h1[c].x, (H)h1[c].y);
    }
    return;
  }
  // U_0(y)^+ h at the top-face site y (its own link, parity q slot, mu = 0)
  const int64_t slab = (int64_t)(REAL ? (D * D + 1) / 2 : D * D) * k.Vh;
  const size_t es = (P == 0) ? 16 : (P == 1 ? 8 : 4);
  const void *lk = reinterpret_cast<const char *>(k.links) + (size_t)((k.q * 4 + 0) * slab) * es;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    cx<A> r0 = mk(A(0), A(0)), r1 = mk(A(0), A(0));
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (REAL) {
        const int e = c * D + a;
        const cx<A> pr = ld2<P>(lk, (int64_t)(e >> 1) * k.Vh + i);
        const A ue = (e & 1) ? pr.y : pr.x;
        r0 = rfma(ue, h0[c], r0);
        r1 = rfma(ue, h1[c], r1);
      } else {
        const cx<A> ue = ld2<P>(lk, (int64_t)(c * D + a) * k.Vh + i);
        r0 = cfmac(ue, h0[c], r0);
        r1 = cfmac(ue, h1[c], r1);
      }
    }
    *hel<P>(k.send_up, k, rhs, 0, a, f, D) = mk((H)r0.x, (H)r0.y);
    *hel<P>(k.send_up, k, rhs, 1, a, f, D) = mk((H)r1.x, (H)r1.y);
  }
}

template <int D, bool REAL, int P>
__global__ void halo_complete_kernel(HaloK k) {
  typedef typename PT<P>::A A;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 2 * k.Lf * k.nrhs) return;
  const int64_t f = g % k.Lf;
  const int top = (int)((g / k.Lf) & 1);
  const int rhs = (int)(g / (2 * k.Lf));
  void *out = reinterpret_cast<char *>(k.out) + (size_t)rhs * k.stride;
  const int64_t i = (top ? (int64_t)(k.T - 1) * k.Lf : 0) + f;
  const A sg = (A)k.sgn;
  cx<A> acc[D][4];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[c][s] = mk(A(0), A(0));
  if (top) {
    // forward t hop of the top face: U_0(x) times the half-spinor from the slab above
    cx<A> h0[D], h1[D];
    const void *rb = k.recv_up;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const auto v0 = *hel<P>(const_cast<void *>(rb), k, rhs, 0, c, f, D);
      const auto v1 = *hel<P>(const_cast<void *>(rb), k, rhs, 1, c, f, D);
      h0[c] = mk((A)v0.x, (A)v0.y);
      h1[c] = mk((A)v1.x, (A)v1.y);
    }
    const int64_t slab = (int64_t)(REAL ? (D * D + 1) / 2 : D * D) * k.Vh;
    const size_t es = (P == 0) ? 16 : (P == 1 ? 8 : 4);
    const void *lk = reinterpret_cast<const char *>(k.links) + (size_t)((k.q * 4 + 0) * slab) * es;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      cx<A> r0 = mk(A(0), A(0)), r1 = mk(A(0), A(0));
#pragma unroll
      for (int c = 0; c < D; ++c) {
        if (REAL) {
          const int e = a * D + c;
          const cx<A> pr = ld2<P>(lk, (int64_t)(e >> 1) * k.Vh + i);
          const A ue = (e & 1) ? pr.y : pr.x;
          r0 = rfma(ue, h0[c], r0);
          r1 = rfma(ue, h1[c], r1);
        } else {
          const cx<A> ue = ld2<P>(lk, (int64_t)(a * D + c) * k.Vh + i);
          r0 = cfma(ue, h0[c], r0);
          r1 = cfma(ue, h1[c], r1);
        }
      }
      reconstruct<0>(-sg, r0, r1, acc[a]);
    }
  } else {
    // backward t hop of the bottom face: already U_0^+ h from the slab below
    const void *rb = k.recv_down;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const auto v0 = *hel<P>(const_cast<void *>(rb), k, rhs, 0, a, f, D);
      const auto v1 = *hel<P>(const_cast<void *>(rb), k, rhs, 1, a, f, D);
      reconstruct<0>(sg, mk((A)v0.x, (A)v0.y), mk((A)v1.x, (A)v1.y), acc[a]);
    }
  }
  const A coef = (A)k.coef;
  if (P == 2) {
    // decode the site, add, re-encode with the new site scale
    const A osc = (A)f16_scales(out, k.Vh, D)[i];
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<A> v[4];
      ld_colour<P>(out, k.Vh, i, c, v);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        acc[c][s] = axpy_r(osc, v[s], scale(coef, acc[c][s]));
        m = fmaxf(m, fmaxf(fabsf((float)acc[c][s].x), fabsf((float)acc[c][s].y)));
      }
    }
    const float inv = m > 0.f ? 1.0f / m : 0.f;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<float> v[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) v[s] = mk((float)acc[c][s].x * inv, (float)acc[c][s].y * inv);
      st_colour16(out, k.Vh, i, c, v);
    }
    f16_scales_w(out, k.Vh, D)[i] = m;
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      cx<A> v[4];
      ld_colour<P>(out, k.Vh, i, c, v);
#pragma unroll
      for (int s = 0; s < 4; ++s) v[s] = v[s] + scale(coef, acc[c][s]);
      if (P == 0) st_colour64(out, k.Vh, i, c, reinterpret_cast<const cx<double> *>(v));
      else st_colour32(out, k.Vh, i, c, reinterpret_cast<const cx<float> *>(v));
    }
  }
}

template <int P>
int launch_halo(const hr_lattice *lat, const HaloK &k, bool pack, cudaStream_t s) {
  const int64_t n = 2 * k.Lf * k.nrhs;
  const unsigned grid = (unsigned)((n + 127) / 128);
  const int d = lat->d;
#define HR_HALO(DD, RE)                                                         \
  if (d == DD && (lat->is_real != 0) == RE) {                                   \
    if (pack) halo_pack_kernel<DD, RE, P><<<grid, 128, 0, s>>>(k);             \
    else halo_complete_kernel<DD, RE, P><<<grid, 128, 0, s>>>(k);              \
    return hr_check_launch(pack ? "halo_pack_kernel" : "halo_complete_kernel"); \
  }
  HR_HALO(3, true) HR_HALO(8, true) HR_HALO(2, false) HR_HALO(3, false) HR_HALO(4, false) HR_HALO(5, false)
  HR_HALO(6, false) HR_HALO(7, false) HR_HALO(8, false)
#undef HR_HALO
  return HR_ERR_UNSUPPORTED;
}

HaloK make_halok(const hr_lattice *lat, int q, int prec, int nrhs, int dagger) {
  HaloK k;
  memset(&k, 0, sizeof(k));
  k.links = lat->links[prec];
  k.T = lat->T;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.nrhs = nrhs;
  k.q = q;
  k.Vh = lat->Vh;
  k.Lf = (int64_t)lat->L * lat->L * (lat->L / 2);
  k.stride = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  k.sgn = dagger ? -1.0 : 1.0;
  return k;
}

int run_halo(const hr_lattice *lat, const HaloK &k, int prec, bool pack, cudaStream_t s) {
  switch (prec) {
    case HR_F64: return launch_halo<0>(lat, k, pack, s);
    case HR_F32: return launch_halo<1>(lat, k, pack, s);
    case HR_F16: return launch_halo<2>(lat, k, pack, s);
  }
  return HR_ERR_ARG;
}

int check_domain_call(const hr_lattice *lat, int out_parity, int prec, int nrhs, int stage) {
  if (!lat || (out_parity != HR_EVEN && out_parity != HR_ODD) || prec < HR_F64 || prec > HR_F16 || nrhs < 1 ||
      (stage != 0 && stage != 1))
    return HR_ERR_ARG;
  if (!lat->dom || !lat->have_links) return HR_ERR_STATE;
  if (lat->csw != 0.0) return HR_ERR_UNSUPPORTED;
  return HR_OK;
}

int begin_impl(hr_lattice *lat, void *out, const void *in_hop, const void *self, int out_parity, double m0, int prec,
               int nrhs, int dagger, int stage, void *send_up, void *send_down, cudaStream_t s) {
  HR_TRY(check_domain_call(lat, out_parity, prec, nrhs, stage));
  if (!out || !in_hop || !send_up || !send_down || (stage == 1 && !self) || out == in_hop) return HR_ERR_ARG;
  HaloK k = make_halok(lat, 1 - out_parity, prec, nrhs, dagger);
  k.in = in_hop;
  k.send_up = send_up;
  k.send_down = send_down;
  HR_TRY(run_halo(lat, k, prec, true, s));
  const double diag = 4.0 + m0;
  HopArgs a;
  memset(&a, 0, sizeof(a));
  a.links = lat->links[prec];
  a.rlinks = lat->rlinks[prec];
  a.dagger = dagger;
  a.nrhs = nrhs;
  a.out = out;
  a.in = in_hop;
  a.self = stage ? self : nullptr;
  a.out_parity = out_parity;
  a.mode = stage ? HOP_SELF : HOP_SCALED;
  a.coef = stage ? 0.5 : -0.5 / diag;
  a.diag = diag;
  a.field_stride = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  a.tmask = 1;
  HR_TRY(hr_launch_hop(lat, prec, a, s));
  lat->hop_launches += 1;
  return HR_OK;
}

int end_impl(hr_lattice *lat, void *out, int out_parity, double m0, int prec, int nrhs, int dagger, int stage,
             const void *recv_up, const void *recv_down, cudaStream_t s) {
  HR_TRY(check_domain_call(lat, out_parity, prec, nrhs, stage));
  if (!out || !recv_up || !recv_down) return HR_ERR_ARG;
  HaloK k = make_halok(lat, out_parity, prec, nrhs, dagger);
  k.out = out;
  k.recv_up = recv_up;
  k.recv_down = recv_down;
  k.coef = stage ? 0.5 : -0.5 / (4.0 + m0);
  return run_halo(lat, k, prec, false, s);
}

}  // namespace

extern "C" int hr_domain_halo_bytes(const hr_lattice *lat, int prec, int nrhs, size_t *bytes) {
  if (!lat || !bytes || prec < HR_F64 || prec > HR_F16 || nrhs < 1) return HR_ERR_ARG;
  const size_t el = prec == HR_F64 ? 16 : 8;
  *bytes = (size_t)nrhs * 2 * lat->d * ((size_t)lat->L * lat->L * (lat->L / 2)) * el;
  return HR_OK;
}

extern "C" int hr_domain_hop_begin(hr_lattice *lat, void *out, const void *in_hop, const void *self, int out_parity,
                                   double m0, int prec, int nrhs, int dagger, int stage, void *send_up,
                                   void *send_down) {
  if (!lat) return HR_ERR_ARG;
  return begin_impl(lat, out, in_hop, self, out_parity, m0, prec, nrhs, dagger, stage, send_up, send_down,
                    lat->stream);
}

extern "C" int hr_domain_hop_end(hr_lattice *lat, void *out, int out_parity, double m0, int prec, int nrhs,
                                 int dagger, int stage, const void *recv_up, const void *recv_down) {
  if (!lat) return HR_ERR_ARG;
  return end_impl(lat, out, out_parity, m0, prec, nrhs, dagger, stage, recv_up, recv_down, lat->stream);
}

// All slabs of one lattice in this process: the whole even-odd Dhat, with the
// exchange done as device-to-device copies between the slabs' own buffers.
extern "C" int hr_domains_dphi(int n, hr_lattice *const *lats, void *const *out, const void *const *in, int parity,
                               double m0, int prec, int nrhs, int dagger) {
  if (n < 1 || !lats || !out || !in || (parity != HR_EVEN && parity != HR_ODD) || prec < HR_F64 ||
      prec > HR_F16 || nrhs < 1)
    return HR_ERR_ARG;
  int tsum = 0;
  for (int k = 0; k < n; ++k) {
    const hr_lattice *l = lats[k];
    if (!l || !out[k] || !in[k]) return HR_ERR_ARG;
    if (!l->dom || !l->have_links) return HR_ERR_STATE;
    if (l->L != lats[0]->L || l->N != lats[0]->N || l->rep != lats[0]->rep || l->Tg != lats[0]->Tg ||
        l->t0 != tsum)
      return HR_ERR_ARG;  // slabs must be given in time order and cover [0, T_global)
    tsum += l->T;
  }
  if (tsum != lats[0]->Tg) return HR_ERR_ARG;
  cudaStream_t s = lats[0]->stream;
  size_t hb = 0;
  HR_TRY(hr_domain_halo_bytes(lats[0], prec, nrhs, &hb));
  for (int k = 0; k < n; ++k) {
    hr_lattice *l = lats[k];
    if (l->halo_bytes < hb) {
      HR_CUDA(cudaStreamSynchronize(s));
      for (int b = 0; b < 4; ++b) {
        hr_dev_free(l->halo[b]);
        l->halo[b] = nullptr;
      }
      l->halo_bytes = 0;
      for (int b = 0; b < 4; ++b) HR_TRY(hr_dev_alloc(&l->halo[b], hb));
      l->halo_bytes = hb;
    }
    HR_TRY(hr_ensure_tmp(l, hr_spinor_field_bytes(l->Vh, l->d, prec) * (size_t)nrhs));
  }
  const int p = parity, q = 1 - parity;
  for (int stage = 0; stage < 2; ++stage) {
    for (int k = 0; k < n; ++k) {
      hr_lattice *l = lats[k];
      void *o = stage ? out[k] : l->tmp;
      const void *ih = stage ? (const void *)l->tmp : in[k];
      HR_TRY(begin_impl(l, o, ih, stage ? in[k] : nullptr, stage ? p : q, m0, prec, nrhs, dagger, stage,
                        l->halo[0], l->halo[1], s));
    }
    // receive-up of slab k <- send-down of slab k+1; receive-down of k <- send-up of k-1
    for (int k = 0; k < n; ++k) {
      HR_CUDA(cudaMemcpyAsync(lats[k]->halo[2], lats[(k + 1) % n]->halo[1], hb, cudaMemcpyDeviceToDevice, s));
      HR_CUDA(cudaMemcpyAsync(lats[k]->halo[3], lats[(k + n - 1) % n]->halo[0], hb, cudaMemcpyDeviceToDevice, s));
    }
    for (int k = 0; k < n; ++k) {
      hr_lattice *l = lats[k];
      HR_TRY(end_impl(l, stage ? out[k] : l->tmp, stage ? p : q, m0, prec, nrhs, dagger, stage, l->halo[2],
                      l->halo[3], s));
    }
  }
  return HR_OK;
}
