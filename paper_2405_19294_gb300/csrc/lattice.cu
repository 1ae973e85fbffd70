// Lattice handle, status strings, stream handling and the canonical <->
// internal spinor conversions (pack / unpack, including the FP16 per-site code).
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>

#include "cplx.cuh"

#include "hr_internal.h"

// detail of the last CUDA error seen by the calling host thread (hr_status_string)
static thread_local char g_last_error[512];

void hr_note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

// ---------------------------------------------------- device allocations ----
// Large library-owned buffers (links, clover, workspaces) go through an
// optional caller-supplied allocator (e.g. PyTorch's caching allocator); each
// allocation remembers the release function it came with, so changing the
// allocator later never frees a block through the wrong one.
namespace {
struct AllocRec {
  hr_free_fn fn;
  void *ctx;
  size_t bytes;
};
std::mutex g_amu;
hr_alloc_fn g_alloc = nullptr;
hr_free_fn g_free = nullptr;
void *g_actx = nullptr;
std::map<void *, AllocRec> g_arec;
}  // namespace

extern "C" int hr_set_allocator(hr_alloc_fn alloc, hr_free_fn release, void *ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return HR_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_amu);
  g_alloc = alloc;
  g_free = release;
  g_actx = ctx;
  return HR_OK;
}

int hr_dev_alloc(void **p, size_t bytes) {
  *p = nullptr;
  hr_alloc_fn a;
  hr_free_fn f;
  void *c;
  {
    std::lock_guard<std::mutex> lk(g_amu);
    a = g_alloc;
    f = g_free;
    c = g_actx;
  }
  if (!a) {
    HR_CUDA(cudaMalloc(p, bytes));
    return HR_OK;
  }
  void *q = a(bytes, c);  // outside the lock: the allocator may call back into anything
  if (!q) return HR_ERR_NOMEM;
  if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
    f(q, bytes, c);
    return HR_ERR_ARG;  // the library's vector loads need 256-byte alignment
  }
  {
    std::lock_guard<std::mutex> lk(g_amu);
    g_arec[q] = AllocRec{f, c, bytes};
  }
  *p = q;
  return HR_OK;
}

void hr_dev_free(void *p) {
  if (!p) return;
  AllocRec r;
  bool mine = false;
  {
    std::lock_guard<std::mutex> lk(g_amu);
    auto it = g_arec.find(p);
    if (it != g_arec.end()) {
      r = it->second;
      g_arec.erase(it);
      mine = true;
    }
  }
  if (mine) r.fn(p, r.bytes, r.ctx);
  else cudaFree(p);
}

int hr_check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    hr_note_cuda_error(e, what, __FILE__, __LINE__);
    return HR_ERR_CUDA;
  }
  return HR_OK;
}

extern "C" const char *hr_status_string(int status) {
  switch (status) {
    case HR_OK: return "ok";
    case HR_ERR_ARG: return "invalid argument";
    case HR_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case HR_ERR_NOMEM: return "device allocation failed";
    case HR_ERR_STATE: return "call out of order (links not loaded?)";
    case HR_ERR_BREAKDOWN: return "solver breakdown";
    case HR_ERR_NOT_CONVERGED: return "solver did not converge";
    case HR_ERR_UNSUPPORTED: return "unsupported combination";
    case HR_ERR_DEVICE: return "device-side guard latched an error";
    default: return "unknown status";
  }
}

static int rep_dim(int N, int rep) {
  switch (rep) {
    case HR_FUND: return N;
    case HR_ADJ: return N * N - 1;
    case HR_SYM: return N * (N + 1) / 2;
    case HR_ASYM: return N * (N - 1) / 2;
  }
  return -1;
}

extern "C" int hr_lattice_create(int T, int L, int N, int rep, hr_lattice **out) {
  if (!out) return HR_ERR_ARG;
  *out = nullptr;
  if (T < 2 || L < 2 || (T & 1) || (L & 1)) return HR_ERR_ARG;
  if (N < 2 || N > HR_MAX_NC || rep < HR_FUND || rep > HR_ASYM) return HR_ERR_ARG;
  if (N > 6 && rep != HR_FUND) return HR_ERR_ARG;
  if (N == 2 && rep == HR_ASYM) return HR_ERR_ARG;
  const int64_t V = (int64_t)T * L * L * L;
  if (V > ((int64_t)1 << 30)) return HR_ERR_ARG;
  hr_lattice *lat = (hr_lattice *)calloc(1, sizeof(hr_lattice));
  if (!lat) return HR_ERR_NOMEM;
  lat->T = T;
  lat->L = L;
  lat->N = N;
  lat->rep = rep;
  lat->d = rep_dim(N, rep);
  lat->is_real = rep == HR_ADJ;
  lat->V = V;
  lat->Vh = V / 2;
  lat->stream = 0;
  lat->nch_link = lat->is_real ? (lat->d * lat->d + 1) / 2 : lat->d * lat->d;
  cudaError_t e = cudaGetDevice(&lat->device);
  if (e != cudaSuccess) {
    free(lat);
    hr_note_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    return HR_ERR_CUDA;
  }
  e = cudaMalloc(&lat->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(lat->dev_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    free(lat);
    hr_note_cuda_error(e, "cudaMalloc(dev_err)", __FILE__, __LINE__);
    return HR_ERR_CUDA;
  }
  lat->t0 = 0;
  lat->Tg = T;
  *out = lat;
  return HR_OK;
}

extern "C" int hr_lattice_create_domain(int T_loc, int L, int N, int rep, int t0, int T_global, hr_lattice **out) {
  if (!out) return HR_ERR_ARG;
  *out = nullptr;
  if (T_loc < 2 || (T_loc & 1) || t0 < 0 || (t0 & 1) || (T_global & 1) || t0 + T_loc > T_global) return HR_ERR_ARG;
  HR_TRY(hr_lattice_create(T_loc, L, N, rep, out));
  (*out)->dom = 1;
  (*out)->t0 = t0;
  (*out)->Tg = T_global;
  return HR_OK;
}

void hr_cg_free(hr_lattice *lat);
void hr_bicgstab_forget(const hr_lattice *lat);

extern "C" int hr_lattice_destroy(hr_lattice *lat) {
  if (!lat) return HR_ERR_ARG;
  cudaDeviceSynchronize();  // the solver streams too: nothing may still use what is freed below
  hr_bicgstab_forget(lat);
  for (int p = 0; p < 4; ++p) {
    hr_dev_free(lat->links[p]);
    hr_dev_free(lat->rlinks[p]);
  }
  for (int b = 0; b < 4; ++b) hr_dev_free(lat->halo[b]);
  hr_dev_free(lat->clover_term);
  for (int p = 0; p < 3; ++p) {
    hr_dev_free(lat->clover_A[p]);
    hr_dev_free(lat->clover_Ainv[p]);
  }
  hr_dev_free(lat->tmp);
  cudaFree(lat->dev_err);
  cudaFree(lat->red_partials);
  cudaFree(lat->red_count);
  cudaFree(lat->red_out);
  cudaFreeHost(lat->red_out_host);
  hr_cg_free(lat);
  free(lat);
  return HR_OK;
}

extern "C" int hr_set_stream(hr_lattice *lat, void *cuda_stream) {
  if (!lat) return HR_ERR_ARG;
  lat->stream = (cudaStream_t)cuda_stream;
  return HR_OK;
}

extern "C" int hr_lattice_info(const hr_lattice *lat, hr_info *info) {
  if (!lat || !info) return HR_ERR_ARG;
  info->T = lat->T;
  info->L = lat->L;
  info->N = lat->N;
  info->rep = lat->rep;
  info->d = lat->d;
  info->is_real = lat->is_real;
  info->volume = lat->V;
  info->half_volume = lat->Vh;
  const double d = lat->d;
  // per output site: 8 matrix x (2 colour vectors) products, projections,
  // reconstructions and accumulation (complex: 8 x 2 x d^2 complex FMA = 128 d^2;
  // real links: 64 d^2), plus 56 d for projection / reconstruction / sums.
  info->flops_hop_site = (lat->is_real ? 64.0 : 128.0) * d * d + 56.0 * d;
  const double link_reals = lat->is_real ? d * d : 2.0 * d * d;
  const double spin_reals = 8.0 * d;
  const double w[3] = {8.0, 4.0, 2.0};
  for (int p = 0; p < 3; ++p) {
    // 8 links + one input spinor (ideal reuse) + one output spinor
    info->bytes_hop_site[p] = 8.0 * link_reals * w[p] + 2.0 * spin_reals * w[p] + (p == 2 ? 8.0 : 0.0);
  }
  return HR_OK;
}

extern "C" int hr_field_bytes(const hr_lattice *lat, int parity, int prec, int nrhs, size_t *bytes) {
  if (!lat || !bytes || nrhs < 1 || prec < HR_F64 || prec > HR_FF || parity < HR_EVEN || parity > HR_FULL)
    return HR_ERR_ARG;
  const size_t fb = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  *bytes = fb * (parity == HR_FULL ? 2u : 1u) * (size_t)nrhs;
  return HR_OK;
}

extern "C" int hr_synchronize(hr_lattice *lat) {
  if (!lat) return HR_ERR_ARG;
  HR_CUDA(cudaStreamSynchronize(lat->stream));
  int err = 0;
  HR_CUDA(cudaMemcpy(&err, lat->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    HR_CUDA(cudaMemset(lat->dev_err, 0, sizeof(int)));
    return HR_ERR_DEVICE;
  }
  return HR_OK;
}

// ------------------------------------------------------------ pack/unpack ----
struct PackK {
  int T, L, Lh, d, p;
  int64_t V, Vh;
  size_t fstride;   // bytes between rhs fields
  size_t poff;      // byte offset of this parity inside a rhs field (FULL)
};

template <int P>
__global__ void pack_kernel(void *internal, const double *canon, PackK k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k.Vh) return;
  const int r = blockIdx.y;
  const Site s = site_of(i, k.p, k.L, k.Lh);
  const int64_t x = lex_index(s.t, s.x, s.y, s.z, k.L);
  const int d = k.d;
  const double *src = canon + ((int64_t)r * k.V + x) * 8 * d;  // [4][d] complex
  char *f = reinterpret_cast<char *>(internal) + (size_t)r * k.fstride + k.poff;
  const int64_t Vh = k.Vh;
  if (P == 0) {
    double2 *q = reinterpret_cast<double2 *>(f);
    for (int c = 0; c < d; ++c)
      for (int sp = 0; sp < 4; ++sp)
        q[(int64_t)(4 * c + sp) * Vh + i] = make_double2(src[2 * (sp * d + c)], src[2 * (sp * d + c) + 1]);
  } else if (P == 3) {
    float4 *q = reinterpret_cast<float4 *>(f);
    for (int c = 0; c < d; ++c)
      for (int sp = 0; sp < 4; ++sp) {
        const ff re(src[2 * (sp * d + c)]), im(src[2 * (sp * d + c) + 1]);
        q[(int64_t)(4 * c + sp) * Vh + i] = make_float4(re.h, re.l, im.h, im.l);
      }
  } else if (P == 1) {
    float4 *q = reinterpret_cast<float4 *>(f);
    for (int c = 0; c < d; ++c)
      for (int h = 0; h < 2; ++h) {
        const double *a = src + 2 * ((2 * h) * d + c);
        const double *b = src + 2 * ((2 * h + 1) * d + c);
        q[(int64_t)(2 * c + h) * Vh + i] = make_float4((float)a[0], (float)a[1], (float)b[0], (float)b[1]);
      }
  } else {
    float m = 0.f;
    for (int e = 0; e < 8 * d; ++e) m = fmaxf(m, fabsf((float)src[e]));
    uint4 *q = reinterpret_cast<uint4 *>(f);
    for (int c = 0; c < d; ++c) {
      unsigned w[4];
      for (int sp = 0; sp < 4; ++sp) {
        const float re = (float)src[2 * (sp * d + c)], im = (float)src[2 * (sp * d + c) + 1];
        __half2 h = (m > 0.f) ? __halves2half2(__float2half_rn(__fdiv_rn(re, m)), __float2half_rn(__fdiv_rn(im, m)))
                              : __halves2half2(__float2half_rn(0.f), __float2half_rn(0.f));
        w[sp] = *reinterpret_cast<unsigned *>(&h);
      }
      q[(int64_t)c * Vh + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    f16_scales_w(f, Vh, d)[i] = m;
  }
}

template <int P>
__global__ void unpack_kernel(double *canon, const void *internal, PackK k) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k.Vh) return;
  const int r = blockIdx.y;
  const Site s = site_of(i, k.p, k.L, k.Lh);
  const int64_t x = lex_index(s.t, s.x, s.y, s.z, k.L);
  const int d = k.d;
  double *dst = canon + ((int64_t)r * k.V + x) * 8 * d;
  const char *f = reinterpret_cast<const char *>(internal) + (size_t)r * k.fstride + k.poff;
  const int64_t Vh = k.Vh;
  if (P == 0) {
    const double2 *q = reinterpret_cast<const double2 *>(f);
    for (int c = 0; c < d; ++c)
      for (int sp = 0; sp < 4; ++sp) {
        double2 v = q[(int64_t)(4 * c + sp) * Vh + i];
        dst[2 * (sp * d + c)] = v.x;
        dst[2 * (sp * d + c) + 1] = v.y;
      }
  } else if (P == 3) {
    const float4 *q = reinterpret_cast<const float4 *>(f);
    for (int c = 0; c < d; ++c)
      for (int sp = 0; sp < 4; ++sp) {
        float4 v = q[(int64_t)(4 * c + sp) * Vh + i];
        dst[2 * (sp * d + c)] = (double)v.x + (double)v.y;
        dst[2 * (sp * d + c) + 1] = (double)v.z + (double)v.w;
      }
  } else if (P == 1) {
    const float4 *q = reinterpret_cast<const float4 *>(f);
    for (int c = 0; c < d; ++c)
      for (int h = 0; h < 2; ++h) {
        float4 v = q[(int64_t)(2 * c + h) * Vh + i];
        dst[2 * ((2 * h) * d + c)] = v.x;
        dst[2 * ((2 * h) * d + c) + 1] = v.y;
        dst[2 * ((2 * h + 1) * d + c)] = v.z;
        dst[2 * ((2 * h + 1) * d + c) + 1] = v.w;
      }
  } else {
    const uint4 *q = reinterpret_cast<const uint4 *>(f);
    const double m = (double)f16_scales(f, Vh, d)[i];
    for (int c = 0; c < d; ++c) {
      uint4 u = q[(int64_t)c * Vh + i];
      unsigned w[4] = {u.x, u.y, u.z, u.w};
      for (int sp = 0; sp < 4; ++sp) {
        __half2 h = *reinterpret_cast<__half2 *>(&w[sp]);
        dst[2 * (sp * d + c)] = (double)__low2float(h) * m;
        dst[2 * (sp * d + c) + 1] = (double)__high2float(h) * m;
      }
    }
  }
}

// A canonical buffer may be device memory or page-locked (registered or
// cudaHostAlloc'd) host memory; for the latter the kernels access it through
// its mapped device address, so only the requested parity's sites cross the
// host link (NVLink-C2C on GB300) and no staging copy is needed.  Pageable,
// unregistered host memory is rejected (HR_ERR_ARG).
static int resolve_canonical(const void *p, const void **dev) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HR_ERR_ARG;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *dev = p;
    return HR_OK;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dev = at.devicePointer;
    return HR_OK;
  }
  return HR_ERR_ARG;
}

static int pack_common(hr_lattice *lat, void *internal, double *canon_w, const double *canon_r, int parity,
                       int prec, int nrhs, bool pack) {
  if (!lat || !internal || !(pack ? (const void *)canon_r : (const void *)canon_w) || nrhs < 1 ||
      prec < HR_F64 || prec > HR_FF || parity < HR_EVEN || parity > HR_FULL)
    return HR_ERR_ARG;
  {
    const void *dev = nullptr;
    HR_TRY(resolve_canonical(pack ? (const void *)canon_r : (const void *)canon_w, &dev));
    if (pack) canon_r = (const double *)dev;
    else canon_w = (double *)dev;
  }
  const size_t fb = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  PackK k;
  k.T = lat->T;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.d = lat->d;
  k.V = lat->V;
  k.Vh = lat->Vh;
  k.fstride = fb * (parity == HR_FULL ? 2 : 1);
  dim3 grid((unsigned)((lat->Vh + 127) / 128), (unsigned)nrhs);
  for (int p = 0; p < 2; ++p) {
    if (parity != HR_FULL && parity != p) continue;
    k.p = p;
    k.poff = (parity == HR_FULL && p == 1) ? fb : 0;
    if (pack) {
      if (prec == HR_F64) pack_kernel<0><<<grid, 128, 0, lat->stream>>>(internal, canon_r, k);
      else if (prec == HR_FF) pack_kernel<3><<<grid, 128, 0, lat->stream>>>(internal, canon_r, k);
      else if (prec == HR_F32) pack_kernel<1><<<grid, 128, 0, lat->stream>>>(internal, canon_r, k);
      else pack_kernel<2><<<grid, 128, 0, lat->stream>>>(internal, canon_r, k);
    } else {
      if (prec == HR_F64) unpack_kernel<0><<<grid, 128, 0, lat->stream>>>(canon_w, internal, k);
      else if (prec == HR_FF) unpack_kernel<3><<<grid, 128, 0, lat->stream>>>(canon_w, internal, k);
      else if (prec == HR_F32) unpack_kernel<1><<<grid, 128, 0, lat->stream>>>(canon_w, internal, k);
      else unpack_kernel<2><<<grid, 128, 0, lat->stream>>>(canon_w, internal, k);
    }
    HR_TRY(hr_check_launch(pack ? "pack_kernel" : "unpack_kernel"));
  }
  return HR_OK;
}

extern "C" int hr_pack_spinor(hr_lattice *lat, void *internal, const double *canonical, int parity, int prec,
                              int nrhs) {
  return pack_common(lat, internal, nullptr, canonical, parity, prec, nrhs, true);
}

extern "C" int hr_unpack_spinor(hr_lattice *lat, double *canonical, const void *internal, int parity, int prec,
                                int nrhs) {
  return pack_common(lat, const_cast<void *>(internal), canonical, nullptr, parity, prec, nrhs, false);
}
