// Many independent lattices (uneven volume, N and representation) solved
// together: the batched operator and CG (for example 64 small lattices of
// 8^4 to 16^3 x 32; the paper notes that at small volumes kernel-call overhead
// dominates, Sec. 3.1.1 and Sec. 3.2).
//
// Lattices are grouped into classes of equal (d_R, real links); each class
// runs one persistent multi-lattice hop launch per hopping stage over a work
// list of (lattice, tile) items, each lattice bringing its own descriptor.
// So one batched Dhat is 2 x (number of classes) launches whatever the number
// of lattices.  The CG vector updates and reductions are single launches over
// all lattices too, with one reduction slot (alpha, beta, |r|^2) per lattice.
// The whole inner iteration (4 x classes hop launches + 3 BLAS launches) is
// captured once into a CUDA graph and replayed in chunks; a lattice whose CG
// has converged sets its frozen flag and its tiles are skipped by the hop and
// update kernels while the others continue.  The outer defect correction
// (true residual, rescaling, x update) runs between chunks, batched over the
// lattices, in FP64 or (outer_prec = HR_FF) in float-float.
#include <algorithm>
#include <chrono>
#include <map>
#include <math.h>
#include <string.h>
#include <vector>

#include "blas_dev.cuh"
#include "hop.cuh"

namespace {

struct BLat {         // per-lattice view for the batched vector kernels
  char *x, *r;        // inner solution and residual (FP32)
  char *p, *Ap, *t;   // operator fields (inner precision)
  int64_t Vh;
  int d, nblk;
};

struct BClass {
  int d, is_real;
  HopShape sh[4];        // launch shape per precision (hr_prec, HR_FF included)
  std::vector<int> members;
  int2 *items[4];        // device work list (lattice index, tile) per precision
  int nitems[4];
  int tuned[4];
};

struct BPair {          // per-lattice (x, y) of a batched y = a x + b y
  const char *x;
  char *y;
  int64_t Vh;
  int d, nblk;
};

enum { B_RR0 = 0, B_RR1, B_PAP, B_ALPHA, B_BETA, B_STOP, B_A, B_B, B_OUT, B_NS };
// batched axpby operand pairs of the outer loop
// (P_B_BO, P_XO_X: b into and x out of the float-float outer iterate)
enum { P_B_R = 0, P_AP_R, P_R_RL, P_RL_PL, P_XL_X, P_XL_XL, P_B_BO, P_XO_X, B_NPAIRS };

int launch_multi(int prec, const BClass &c, const HopK *descs, const int *frozen, cudaStream_t s) {
  const HopShape sh = c.sh[prec];
  switch (prec) {
    case HR_F64: return hr_launch_hop_multi_f64(c.d, c.is_real, sh, descs, c.items[prec], c.nitems[prec], frozen, s);
    case HR_F32: return hr_launch_hop_multi_f32(c.d, c.is_real, sh, descs, c.items[prec], c.nitems[prec], frozen, s);
    case HR_F16: return hr_launch_hop_multi_f16(c.d, c.is_real, sh, descs, c.items[prec], c.nitems[prec], frozen, s);
    case HR_FF: return hr_launch_hop_multi_ff(c.d, c.is_real, sh, descs, c.items[prec], c.nitems[prec], frozen, s);
  }
  return HR_ERR_ARG;
}

// y = a x + b y per lattice (a, b, skip indexed by lattice), optional |y|^2 per lattice
template <int PX, int PY>
__global__ void baxpby_kernel(const BPair *pr, const int2 *items, const double *a, const double *b, RedArgs red,
                              int want_norm, const int *skip) {
  typedef typename PT<PY>::A AY;
  const int2 it = items[blockIdx.x];
  const BPair P = pr[it.x];
  double acc = 0.0;
  if (!(skip && skip[it.x]))
    acc = axpby_sites<PX, PY>(P.x, P.y, P.Vh, P.d, (AY)a[it.x], (AY)b[it.x],
                              (int64_t)it.y * blockDim.x + threadIdx.x, (int64_t)P.nblk * blockDim.x);
  if (want_norm) reduce_publish(acc, red, RED_PLAIN, it.x, it.y, P.nblk);
}

template <int P>
__global__ void bnorm2_kernel(const BLat *bl, const int2 *items, RedArgs red, int finish, const int *frozen) {
  const int2 it = items[blockIdx.x];
  const BLat L = bl[it.x];
  double acc = 0.0;
  if (!(frozen && frozen[it.x]))
    acc = norm2_sites<P>(L.t, L.Vh, L.d, (int64_t)it.y * blockDim.x + threadIdx.x, (int64_t)L.nblk * blockDim.x);
  reduce_publish(acc, red, finish, it.x, it.y, L.nblk);
}

template <int PR, int PP>
__global__ void bcg_xr_kernel(const BLat *bl, const int2 *items, RedArgs red) {
  typedef typename PT<PR>::A AR;
  const int2 it = items[blockIdx.x];
  const BLat L = bl[it.x];
  const AR al = (AR)red.alpha[it.x];
  double acc = 0.0;
  if (al != (AR)0)
    acc = cg_xr_sites<PR, PP>(L.x, L.r, L.p, L.Ap, L.Vh, L.d, al, (int64_t)it.y * blockDim.x + threadIdx.x,
                              (int64_t)L.nblk * blockDim.x);
  reduce_publish(acc, red, RED_BETA, it.x, it.y, L.nblk);
}

template <int PR, int PP>
__global__ void bcg_p_kernel(const BLat *bl, const int2 *items, const double *beta, const double *alpha) {
  const int2 it = items[blockIdx.x];
  if (alpha[it.x] == 0.0) return;
  const BLat L = bl[it.x];
  cg_p_sites<PR, PP>(L.r, L.p, L.Vh, L.d, (typename PT<PP>::A)beta[it.x], (int64_t)it.y * blockDim.x + threadIdx.x,
                     (int64_t)L.nblk * blockDim.x);
}

}  // namespace

struct hr_batch {
  int n;
  std::vector<hr_lattice *> lats;
  std::vector<BClass> cls;
  cudaStream_t stream;  // caller's stream
  cudaStream_t s;       // internal stream (capturable)
  std::vector<cudaStream_t> cs;  // one per class: the classes of a hopping stage run concurrently
  std::vector<cudaEvent_t> cev;  // per class: its launch of the stage is done
  cudaEvent_t fork;              // the stage may start
  HopK *d_desc;         // [8 stages][n]: inner Dhat, inner Dhat^+, FP64 Dhat, FP64 Dhat^+
  HopK *h_desc;         // pinned staging
  BPair *d_pairs;       // [B_NPAIRS][n] operand pairs of the batched axpby
  BPair *h_pairs;
  BLat *d_blat;
  BLat *h_blat;
  int2 *d_bitems;
  int nbitems;
  double *scal;         // [B_NS][n]
  double *host;         // pinned mirror
  int *iters, *frozen, *err;
  double *partials;
  unsigned *count;
};

static double *BS(hr_batch *b, int k) { return b->scal + (size_t)k * b->n; }

static int build_items(BClass &c, const std::vector<hr_lattice *> &lats, int prec) {
  const HopShape sh = c.sh[prec];
  const int tile = hr_shape_tile(sh);
  std::vector<int2> items;
  for (int li : c.members) {
    const int64_t nt = (lats[li]->Vh + tile - 1) / tile;
    for (int64_t t = 0; t < nt; ++t) items.push_back(make_int2(li, (int)t));
  }
  cudaFree(c.items[prec]);
  c.items[prec] = nullptr;
  c.nitems[prec] = (int)items.size();
  HR_CUDA(cudaMalloc(&c.items[prec], sizeof(int2) * std::max<size_t>(1, items.size())));
  HR_CUDA(cudaMemcpy(c.items[prec], items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  return HR_OK;
}

extern "C" int hr_batch_create(int n, hr_lattice *const *lats, hr_batch **out) {
  if (!out || !lats || n < 1 || n > 4096) return HR_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!lats[i]) return HR_ERR_ARG;
    if (!lats[i]->have_links) return HR_ERR_STATE;
    if (lats[i]->csw != 0.0 || lats[i]->dom) return HR_ERR_UNSUPPORTED;
    // the rows kernel reads the rows link layout, built with the links when csw = 0
    if (hr_has_rows_shapes(lats[i]->d, lats[i]->is_real) && !lats[i]->rlinks[HR_F16]) return HR_ERR_STATE;
  }
  hr_batch *b = new hr_batch();
  b->n = n;
  b->lats.assign(lats, lats + n);
  b->stream = lats[0]->stream;
  std::map<int, int> cidx;
  for (int i = 0; i < n; ++i) {
    const int key = lats[i]->d * 2 + lats[i]->is_real;
    auto it = cidx.find(key);
    if (it == cidx.end()) {
      BClass c;
      c.d = lats[i]->d;
      c.is_real = lats[i]->is_real;
      for (int q = 0; q < 4; ++q) {
        HopShape shapes[HR_MAX_SHAPES];
        if (hr_hop_shapes(c.d, c.is_real, q, 0, 0, shapes) < 1) {
          delete b;
          return HR_ERR_UNSUPPORTED;
        }
        c.sh[q] = shapes[0];
        c.items[q] = nullptr;
        c.nitems[q] = 0;
        c.tuned[q] = 0;
      }
      cidx[key] = (int)b->cls.size();
      b->cls.push_back(c);
      it = cidx.find(key);
    }
    b->cls[it->second].members.push_back(i);
  }
  int rc = HR_OK;
  for (auto &c : b->cls)
    for (int q = 0; q < 4; ++q)
      if (rc == HR_OK) rc = build_items(c, b->lats, q);
  std::vector<int2> bitems;
  for (int i = 0; i < n; ++i) {
    const int nblk = hr_blas_blocks(lats[i]->Vh);
    for (int k = 0; k < nblk; ++k) bitems.push_back(make_int2(i, k));
  }
  b->nbitems = (int)bitems.size();
  auto A = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == HR_OK) {
      hr_note_cuda_error(e, "hr_batch_create", __FILE__, __LINE__);
      rc = HR_ERR_CUDA;
    }
  };
  A(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
  // the classes run largest first (by even sites x link reals), each on its own stream
  std::sort(b->cls.begin(), b->cls.end(), [&](const BClass &x, const BClass &y) {
    auto work = [&](const BClass &c) {
      double w = 0.0;
      for (int li : c.members) w += (double)lats[li]->Vh;
      return w * (c.is_real ? 1.0 : 2.0) * c.d * c.d;
    };
    return work(x) > work(y);
  });
  b->cs.assign(b->cls.size(), nullptr);
  b->cev.assign(b->cls.size(), nullptr);
  for (size_t c = 0; c < b->cls.size(); ++c) {
    A(cudaStreamCreateWithFlags(&b->cs[c], cudaStreamNonBlocking));
    A(cudaEventCreateWithFlags(&b->cev[c], cudaEventDisableTiming));
  }
  A(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  A(cudaMalloc(&b->d_desc, sizeof(HopK) * 8 * n));
  A(cudaMallocHost(&b->h_desc, sizeof(HopK) * 8 * n));
  A(cudaMalloc(&b->d_pairs, sizeof(BPair) * B_NPAIRS * n));
  A(cudaMallocHost(&b->h_pairs, sizeof(BPair) * B_NPAIRS * n));
  A(cudaMalloc(&b->d_blat, sizeof(BLat) * n));
  A(cudaMallocHost(&b->h_blat, sizeof(BLat) * n));
  A(cudaMalloc(&b->d_bitems, sizeof(int2) * bitems.size()));
  if (rc == HR_OK) A(cudaMemcpy(b->d_bitems, bitems.data(), sizeof(int2) * bitems.size(), cudaMemcpyHostToDevice));
  A(cudaMalloc(&b->scal, sizeof(double) * B_NS * n));
  A(cudaMallocHost(&b->host, sizeof(double) * B_NS * n));
  A(cudaMalloc(&b->iters, sizeof(int) * n));
  A(cudaMalloc(&b->frozen, sizeof(int) * n));
  A(cudaMalloc(&b->err, sizeof(int)));
  A(cudaMalloc(&b->partials, sizeof(double) * 2 * HR_RED_MAXBLK * n));
  A(cudaMalloc(&b->count, sizeof(unsigned) * n));
  if (rc == HR_OK) {
    A(cudaMemset(b->count, 0, sizeof(unsigned) * n));
    A(cudaMemset(b->err, 0, sizeof(int)));
    A(cudaMemset(b->frozen, 0, sizeof(int) * n));
    A(cudaMemset(b->scal, 0, sizeof(double) * B_NS * n));
  }
  if (rc != HR_OK) {
    hr_batch_destroy(b);
    return rc;
  }
  *out = b;
  return HR_OK;
}

extern "C" int hr_batch_destroy(hr_batch *b) {
  if (!b) return HR_ERR_ARG;
  if (b->s) {
    cudaStreamSynchronize(b->s);
    cudaStreamDestroy(b->s);
  }
  for (auto st : b->cs)
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (auto e : b->cev)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto &c : b->cls)
    for (int q = 0; q < 4; ++q) cudaFree(c.items[q]);
  cudaFree(b->d_desc);
  cudaFreeHost(b->h_desc);
  cudaFree(b->d_pairs);
  cudaFreeHost(b->h_pairs);
  cudaFree(b->d_blat);
  cudaFreeHost(b->h_blat);
  cudaFree(b->d_bitems);
  cudaFree(b->scal);
  cudaFreeHost(b->host);
  cudaFree(b->iters);
  cudaFree(b->frozen);
  cudaFree(b->err);
  cudaFree(b->partials);
  cudaFree(b->count);
  delete b;
  return HR_OK;
}

extern "C" int hr_batch_set_stream(hr_batch *b, void *stream) {
  if (!b) return HR_ERR_ARG;
  b->stream = (cudaStream_t)stream;
  return HR_OK;
}

// Descriptors of the two hopping stages of Dhat_p (or its adjoint) for every
// lattice: stage 0: tmp_q = coef0 H in (A_qq^{-1} = 1/(4+m0)); stage 1:
// out = (4+m0) in + 1/2 H tmp_q.  Written to h_desc[slot * n + lattice].
static int fill_desc(hr_batch *b, int slot0, int prec, void *const *out, const void *const *in, int parity,
                     const double *m0, int dagger) {
  for (int i = 0; i < b->n; ++i) {
    hr_lattice *lat = b->lats[i];
    const size_t fb = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
    HR_TRY(hr_ensure_tmp(lat, fb));
    const double diag = 4.0 + m0[i];
    HopArgs a;
    memset(&a, 0, sizeof(a));
    a.links = lat->links[prec];
    a.rlinks = lat->rlinks[prec];
    a.dagger = dagger;
    a.nrhs = 1;
    a.field_stride = fb;
    a.out = lat->tmp;
    a.in = in[i];
    a.out_parity = 1 - parity;
    a.mode = HOP_SCALED;
    a.coef = -0.5 / diag;
    b->h_desc[(size_t)slot0 * b->n + i] = make_hopk(lat, a);
    a.out = out[i];
    a.in = lat->tmp;
    a.self = in[i];
    a.out_parity = parity;
    a.mode = HOP_SELF;
    a.coef = 0.5;
    a.diag = diag;
    b->h_desc[(size_t)(slot0 + 1) * b->n + i] = make_hopk(lat, a);
  }
  return HR_OK;
}

// Pick each class's launch shape by timing its candidates on stage 0 of the
// uploaded descriptors (persistent multi-lattice launches).
static int tune_classes(hr_batch *b, int prec, int slot0, cudaStream_t s) {
  HrEvent e0_owner, e1_owner;
  HR_CUDA(cudaEventCreate(&e0_owner.e));
  HR_CUDA(cudaEventCreate(&e1_owner.e));
  cudaEvent_t e0 = e0_owner.e, e1 = e1_owner.e;
  for (auto &c : b->cls) {
    if (c.tuned[prec]) continue;
    HopShape shapes[HR_MAX_SHAPES];
    const int ns = hr_hop_shapes(c.d, c.is_real, prec, 0, 0, shapes);
    float best = 1e30f;
    HopShape bs = shapes[0];
    const HopK *descs = b->d_desc + (size_t)slot0 * b->n;
    for (int k = 0; k < ns; ++k) {
      c.sh[prec] = shapes[k];
      HR_TRY(build_items(c, b->lats, prec));
      HR_TRY(launch_multi(prec, c, descs, nullptr, s));
      HR_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) HR_TRY(launch_multi(prec, c, descs, nullptr, s));
      HR_CUDA(cudaEventRecord(e1, s));
      HR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      HR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bs = shapes[k];
      }
    }
    c.sh[prec] = bs;
    c.tuned[prec] = 1;
    HR_TRY(build_items(c, b->lats, prec));
  }
  return HR_OK;
}

// Pin the launch shape of the class (d, is_real) at precision prec instead of
// timing its candidates; the shape must be one of them.
extern "C" int hr_batch_set_shape(hr_batch *b, int d, int is_real, int prec, int shape) {
  if (!b || prec < HR_F64 || prec > HR_FF) return HR_ERR_ARG;
  for (auto &c : b->cls) {
    if (c.d != d || c.is_real != (is_real != 0)) continue;
    HopShape shapes[HR_MAX_SHAPES];
    const int ns = hr_hop_shapes(c.d, c.is_real, prec, 0, 0, shapes);
    for (int k = 0; k < ns; ++k)
      if (hr_shape_code(shapes[k]) == shape) {
        c.sh[prec] = shapes[k];
        c.tuned[prec] = 1;
        return build_items(c, b->lats, prec);
      }
    return HR_ERR_ARG;
  }
  return HR_ERR_ARG;
}

// One hopping stage (descriptor slot `slot`) of every class: the class
// launches fork from `s` onto the classes' own streams and join back, so the
// small classes run beside the large ones instead of after them (inside a
// captured graph these become parallel branches).
static int batch_stage(hr_batch *b, int prec, int slot, const int *frozen, cudaStream_t s) {
  const HopK *descs = b->d_desc + (size_t)slot * b->n;
  if (b->cls.size() == 1) return launch_multi(prec, b->cls[0], descs, frozen, s);
  HR_CUDA(cudaEventRecord(b->fork, s));
  for (size_t c = 0; c < b->cls.size(); ++c) {
    HR_CUDA(cudaStreamWaitEvent(b->cs[c], b->fork, 0));
    HR_TRY(launch_multi(prec, b->cls[c], descs, frozen, b->cs[c]));
    HR_CUDA(cudaEventRecord(b->cev[c], b->cs[c]));
  }
  for (size_t c = 0; c < b->cls.size(); ++c) HR_CUDA(cudaStreamWaitEvent(s, b->cev[c], 0));
  return HR_OK;
}

// launches of one batched Dhat (stages slot0, slot0+1 of d_desc)
static int batch_dhat(hr_batch *b, int prec, int slot0, const int *frozen, cudaStream_t s) {
  HR_TRY(batch_stage(b, prec, slot0, frozen, s));
  return batch_stage(b, prec, slot0 + 1, frozen, s);
}

extern "C" int hr_batch_dphi(hr_batch *b, void *const *out, const void *const *in, int parity, const double *m0,
                             int prec, int dagger) {
  if (!b || !out || !in || !m0 || (parity != HR_EVEN && parity != HR_ODD) || prec < HR_F64 || prec > HR_FF)
    return HR_ERR_ARG;
  for (int i = 0; i < b->n; ++i)
    if (!out[i] || !in[i] || out[i] == in[i]) return HR_ERR_ARG;
  if (prec == HR_FF)
    for (auto *lat : b->lats) HR_TRY(hr_ff_prepare(lat, 0, 0.0, b->stream));
  HR_TRY(fill_desc(b, 0, prec, out, in, parity, m0, dagger));
  HR_CUDA(cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(HopK) * 2 * b->n, cudaMemcpyHostToDevice, b->stream));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HR_CUDA(cudaStreamIsCapturing(b->stream, &cap));
  if (cap == cudaStreamCaptureStatusNone) HR_TRY(tune_classes(b, prec, 0, b->stream));
  HR_TRY(batch_dhat(b, prec, 0, nullptr, b->stream));
  for (auto *lat : b->lats) lat->hop_launches += 2;
  return HR_OK;
}

// --------------------------------------------------------------- batched CG
extern "C" int hr_batch_cg_solve(hr_batch *b, void *const *x, const void *const *bsrc, int parity, const double *m0,
                                 const hr_cg_params *prm, hr_cg_stats *stats) {
  if (!b || !x || !bsrc || !m0 || !prm || (parity != HR_EVEN && parity != HR_ODD)) return HR_ERR_ARG;
  if (prm->tol <= 0.0 || prm->inner_prec < HR_F32 || prm->inner_prec > HR_F16) return HR_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  const int n = b->n, lo = prm->inner_prec;
  const int check_every = std::max(2, (prm->check_every > 0 ? prm->check_every : 10) & ~1);
  const int maxit = prm->maxit > 0 ? prm->maxit : 100000;
  const double inner_tol = prm->inner_tol > 0.0 ? prm->inner_tol : (lo == HR_F32 ? 1e-5 : 3e-3);
  cudaStream_t s = b->s;
  // order after the caller's stream
  HrEvent ev_owner;
  HR_CUDA(cudaEventCreateWithFlags(&ev_owner.e, cudaEventDisableTiming));
  cudaEvent_t ev = ev_owner.e;
  HR_CUDA(cudaEventRecord(ev, b->stream));
  HR_CUDA(cudaStreamWaitEvent(s, ev, 0));
  // workspaces and per-lattice descriptors
  std::vector<void *> pl(n), Apl(n), tl(n);
  for (int i = 0; i < n; ++i) {
    hr_lattice *lat = b->lats[i];
    HR_TRY(hr_cg_workspace(lat, HR_F64, hr_spinor_field_bytes(lat->Vh, lat->d, HR_F64)));
    HR_TRY(hr_cg_workspace(lat, HR_F32, hr_spinor_field_bytes(lat->Vh, lat->d, HR_F32)));
    if (lo == HR_F16) HR_TRY(hr_cg_workspace(lat, HR_F16, hr_spinor_field_bytes(lat->Vh, lat->d, HR_F16)));
    HR_TRY(hr_red_scratch(lat, 1));
    HR_TRY(hr_ensure_tmp(lat, hr_spinor_field_bytes(lat->Vh, lat->d, HR_F64)));
    pl[i] = hr_cg_field(lat, lo, 1);
    Apl[i] = hr_cg_field(lat, lo, 2);
    tl[i] = hr_cg_field(lat, lo, 3);
    BLat &L = b->h_blat[i];
    L.x = (char *)hr_cg_field(lat, HR_F32, 4);
    L.r = (char *)hr_cg_field(lat, HR_F32, 0);
    L.p = (char *)pl[i];
    L.Ap = (char *)Apl[i];
    L.t = (char *)tl[i];
    L.Vh = lat->Vh;
    L.d = lat->d;
    L.nblk = hr_blas_blocks(lat->Vh);
  }
  HR_TRY(fill_desc(b, 0, lo, tl.data(), (const void *const *)pl.data(), parity, m0, 0));   // t = Dhat p
  HR_TRY(fill_desc(b, 2, lo, Apl.data(), (const void *const *)tl.data(), parity, m0, 1));  // Ap = Dhat^+ t
  HR_CUDA(cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(HopK) * 4 * n, cudaMemcpyHostToDevice, s));
  HR_CUDA(cudaMemcpyAsync(b->d_blat, b->h_blat, sizeof(BLat) * n, cudaMemcpyHostToDevice, s));
  HR_TRY(tune_classes(b, lo, 0, s));
  HR_CUDA(cudaMemsetAsync(b->iters, 0, sizeof(int) * n, s));

  RedArgs red;
  memset(&red, 0, sizeof(red));
  red.partials = b->partials;
  red.count = b->count;
  red.err = b->err;
  red.stop = BS(b, B_STOP);
  red.iters = b->iters;
  red.frozen = b->frozen;

  // capture one chunk of check_every inner iterations
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  HR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = HR_OK;
  const dim3 bgrid(b->nbitems);
  for (int k = 0; k < check_every && rc == HR_OK; ++k) {
    double *rr = BS(b, (k & 1) ? B_RR1 : B_RR0), *rr_next = BS(b, (k & 1) ? B_RR0 : B_RR1);
    rc = batch_dhat(b, lo, 0, b->frozen, s);
    if (rc != HR_OK) break;
    RedArgs ra = red;
    ra.out = BS(b, B_PAP);
    ra.rr = rr;
    ra.alpha = BS(b, B_ALPHA);
    if (lo == HR_F32) bnorm2_kernel<1><<<bgrid, 256, 0, s>>>(b->d_blat, b->d_bitems, ra, RED_ALPHA, b->frozen);
    else bnorm2_kernel<2><<<bgrid, 256, 0, s>>>(b->d_blat, b->d_bitems, ra, RED_ALPHA, b->frozen);
    rc = batch_dhat(b, lo, 2, b->frozen, s);
    if (rc != HR_OK) break;
    RedArgs rb = red;
    rb.out = BS(b, B_OUT);
    rb.rr = rr;
    rb.rr_next = rr_next;
    rb.alpha = BS(b, B_ALPHA);
    rb.beta = BS(b, B_BETA);
    if (lo == HR_F32) {
      bcg_xr_kernel<1, 1><<<bgrid, 256, 0, s>>>(b->d_blat, b->d_bitems, rb);
      bcg_p_kernel<1, 1><<<bgrid, 256, 0, s>>>(b->d_blat, b->d_bitems, BS(b, B_BETA), BS(b, B_ALPHA));
    } else {
      bcg_xr_kernel<1, 2><<<bgrid, 256, 0, s>>>(b->d_blat, b->d_bitems, rb);
      bcg_p_kernel<1, 2><<<bgrid, 256, 0, s>>>(b->d_blat, b->d_bitems, BS(b, B_BETA), BS(b, B_ALPHA));
    }
  }
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (rc != HR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  HR_CUDA(ce);
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  HR_CUDA(ce);

  // -------------------------------------------------------------- outer loop
  // Every outer-loop vector operation is one batched launch over all lattices
  // (per-lattice a, b and skip flags); the true residual uses the
  // multi-lattice hop of precision po (descriptor stages 4..7): FP64, or
  // float-float with the outer iterate xo and bo = b as float-float fields
  // (the FP64 workspace's otherwise unused p and x buffers).
  int use_ff = prm->outer_prec == HR_FF;
  for (int i = 0; i < n && use_ff; ++i) HR_TRY(hr_ff_outer_usable(b->lats[i], 0, m0[i], 1, s, &use_ff));
  const int po = use_ff ? HR_FF : HR_F64;
  std::vector<void *> t64(n), Ap64(n), r64(n), xo(n), bo(n);
  for (int i = 0; i < n; ++i) {
    t64[i] = hr_cg_field(b->lats[i], HR_F64, 3);
    Ap64[i] = hr_cg_field(b->lats[i], HR_F64, 2);
    r64[i] = hr_cg_field(b->lats[i], HR_F64, 0);
    xo[i] = po == HR_FF ? hr_cg_field(b->lats[i], HR_F64, 4) : x[i];
    bo[i] = po == HR_FF ? hr_cg_field(b->lats[i], HR_F64, 1) : const_cast<void *>(bsrc[i]);
  }
  HR_TRY(fill_desc(b, 4, po, t64.data(), (const void *const *)xo.data(), parity, m0, 0));     // t = Dhat x
  HR_TRY(fill_desc(b, 6, po, Ap64.data(), (const void *const *)t64.data(), parity, m0, 1));   // Ap = Dhat^+ t
  for (int i = 0; i < n; ++i) {
    hr_lattice *lat = b->lats[i];
    const int nblk = hr_blas_blocks(lat->Vh);
    auto pair = [&](int which, const void *px, void *py) {
      b->h_pairs[(size_t)which * n + i] = BPair{(const char *)px, (char *)py, lat->Vh, lat->d, nblk};
    };
    pair(P_B_R, bo[i], r64[i]);
    pair(P_AP_R, Ap64[i], r64[i]);
    pair(P_R_RL, r64[i], b->h_blat[i].r);
    pair(P_RL_PL, b->h_blat[i].r, pl[i]);
    pair(P_XL_X, b->h_blat[i].x, xo[i]);
    pair(P_XL_XL, b->h_blat[i].x, b->h_blat[i].x);
    pair(P_B_BO, bsrc[i], bo[i]);
    pair(P_XO_X, xo[i], x[i]);
  }
  HR_CUDA(cudaMemcpyAsync(b->d_desc + (size_t)4 * n, b->h_desc + (size_t)4 * n, sizeof(HopK) * 4 * n,
                          cudaMemcpyHostToDevice, s));
  HR_CUDA(cudaMemcpyAsync(b->d_pairs, b->h_pairs, sizeof(BPair) * B_NPAIRS * n, cudaMemcpyHostToDevice, s));
  HR_TRY(tune_classes(b, po, 4, s));
  int *skip = b->frozen;  // reused between phases: 1 = lattice done (outer) / frozen (inner)
  std::vector<double> bn2(n), rn2(n);
  std::vector<int> active(n, 1), skipv(n);
  auto set = [&](int which, const std::vector<double> &v) -> int {
    HR_CUDA(cudaMemcpyAsync(BS(b, which), v.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    HR_CUDA(cudaStreamSynchronize(s));
    return HR_OK;
  };
  auto set_skip = [&]() -> int {
    for (int i = 0; i < n; ++i) skipv[i] = active[i] ? 0 : 1;
    HR_CUDA(cudaMemcpyAsync(skip, skipv.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    HR_CUDA(cudaStreamSynchronize(s));
    return HR_OK;
  };
  RedArgs rn = red;
  rn.out = BS(b, B_OUT);
  rn.frozen = nullptr;
  const dim3 agrid(b->nbitems);
  auto axpby = [&](int which, int px, int py, int norm) -> int {
    const BPair *pp = b->d_pairs + (size_t)which * n;
#define BAX(X, Y) baxpby_kernel<X, Y><<<agrid, 256, 0, s>>>(pp, b->d_bitems, BS(b, B_A), BS(b, B_B), rn, norm, skip)
    if (px == 0 && py == 0) BAX(0, 0);
    else if (px == 0 && py == 1) BAX(0, 1);
    else if (px == 1 && py == 0) BAX(1, 0);
    else if (px == 1 && py == 1) BAX(1, 1);
    else if (px == 1 && py == 2) BAX(1, 2);
    else if (px == 0 && py == 3) BAX(0, 3);
    else if (px == 3 && py == 3) BAX(3, 3);
    else if (px == 3 && py == 1) BAX(3, 1);
    else if (px == 1 && py == 3) BAX(1, 3);
    else if (px == 3 && py == 0) BAX(3, 0);
    else return HR_ERR_UNSUPPORTED;
#undef BAX
    return hr_check_launch("baxpby_kernel");
  };
  auto fetch_norms = [&](std::vector<double> &v) -> int {
    HR_CUDA(cudaMemcpyAsync(b->host, BS(b, B_OUT), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    HR_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; ++i)
      if (active[i]) v[i] = b->host[i];
    return HR_OK;
  };
  std::vector<double> one(n, 1.0), zero(n, 0.0), mone(n, -1.0), va(n);
  // x = 0; r = b; |b|^2
  for (int i = 0; i < n; ++i) {
    const size_t fb = hr_spinor_field_bytes(b->lats[i]->Vh, b->lats[i]->d, HR_F64);
    HR_CUDA(cudaMemsetAsync(x[i], 0, fb, s));
    if (po == HR_FF) HR_CUDA(cudaMemsetAsync(xo[i], 0, fb, s));
  }
  HR_TRY(set_skip());
  HR_TRY(set(B_A, one));
  HR_TRY(set(B_B, zero));
  if (po == HR_FF) HR_TRY(axpby(P_B_BO, HR_F64, HR_FF, 0));
  HR_TRY(axpby(P_B_R, po, po, 1));
  HR_TRY(fetch_norms(bn2));
  for (int i = 0; i < n; ++i) rn2[i] = bn2[i];

  int status = HR_OK, iters = 0, outer = 0;
  const double tol2 = prm->tol * prm->tol;
  while (true) {
    int nact = 0;
    for (int i = 0; i < n; ++i) {
      active[i] = !(rn2[i] <= tol2 * bn2[i]);
      nact += active[i];
    }
    if (nact == 0) break;
    if (iters >= maxit || outer >= 200) {
      status = HR_ERR_NOT_CONVERGED;
      break;
    }
    // rl = r / |r|, pl = rl, xl = 0 on active lattices; stop and rr per lattice
    std::vector<double> stop(n), rr(n);
    std::vector<int> frz(n);
    for (int i = 0; i < n; ++i) {
      const double rnv = sqrt(rn2[i]);
      va[i] = (active[i] && rnv > 0.0) ? 1.0 / rnv : 0.0;
      double tgt = prm->tol * sqrt(bn2[i]) / (2.0 * (rnv > 0.0 ? rnv : 1.0));
      if (tgt < inner_tol) tgt = inner_tol;
      stop[i] = active[i] ? tgt * tgt : 1e300;
      rr[i] = active[i] ? 1.0 : 0.0;
      frz[i] = active[i] ? 0 : 1;
    }
    HR_TRY(set_skip());
    HR_TRY(set(B_A, va));
    HR_TRY(set(B_B, zero));
    HR_TRY(axpby(P_R_RL, po, HR_F32, 0));
    HR_TRY(set(B_A, one));
    HR_TRY(axpby(P_RL_PL, HR_F32, lo, 0));
    HR_TRY(set(B_A, zero));
    HR_TRY(axpby(P_XL_XL, HR_F32, HR_F32, 0));  // xl = 0 x + 0 xl
    HR_TRY(set(B_STOP, stop));
    HR_TRY(set(B_RR0, rr));
    HR_CUDA(cudaMemcpyAsync(b->frozen, frz.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    HR_CUDA(cudaStreamSynchronize(s));
    // inner chunks (the graph's kernels read b->frozen, maintained on the device)
    int done = 0;
    while (iters + done < maxit) {
      HR_CUDA(cudaGraphLaunch(exec, s));
      done += check_every;
      HR_CUDA(cudaMemcpyAsync(frz.data(), b->frozen, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
      HR_CUDA(cudaStreamSynchronize(s));
      bool all = true;
      for (int i = 0; i < n; ++i) all = all && frz[i];
      if (all) break;
    }
    iters += done;
    ++outer;
    int herr = 0;
    HR_CUDA(cudaMemcpy(&herr, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
      HR_CUDA(cudaMemset(b->err, 0, sizeof(int)));
      status = HR_ERR_BREAKDOWN;
      break;
    }
    // x += |r| xl (active lattices), then r = b - M x (precision po)
    HR_TRY(set_skip());
    for (int i = 0; i < n; ++i) va[i] = sqrt(rn2[i]);
    HR_TRY(set(B_A, va));
    HR_TRY(set(B_B, one));
    HR_TRY(axpby(P_XL_X, HR_F32, po, 0));
    HR_TRY(batch_dhat(b, po, 4, skip, s));
    HR_TRY(batch_dhat(b, po, 6, skip, s));
    HR_TRY(set(B_A, one));
    HR_TRY(set(B_B, zero));
    HR_TRY(axpby(P_B_R, po, po, 0));
    HR_TRY(set(B_A, mone));
    HR_TRY(set(B_B, one));
    HR_TRY(axpby(P_AP_R, po, po, 1));
    HR_TRY(fetch_norms(rn2));
  }
  if (po == HR_FF) {  // x = the FP64 value of every lattice's float-float iterate
    std::fill(active.begin(), active.end(), 1);
    HR_TRY(set_skip());
    HR_TRY(set(B_A, one));
    HR_TRY(set(B_B, zero));
    HR_TRY(axpby(P_XO_X, HR_FF, HR_F64, 0));
  }
  cudaGraphExecDestroy(exec);
  HR_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    std::vector<int> it(n);
    HR_CUDA(cudaMemcpy(it.data(), b->iters, sizeof(int) * n, cudaMemcpyDeviceToHost));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < n; ++i) {
      stats[i].iterations = it[i];
      stats[i].outer_steps = outer;
      stats[i].true_residual = bn2[i] > 0.0 ? sqrt(rn2[i] / bn2[i]) : 0.0;
      stats[i].seconds = secs;
      stats[i].hop_launches = 0.0;
    }
  }
  return status;
}
