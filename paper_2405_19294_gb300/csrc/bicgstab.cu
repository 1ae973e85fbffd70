// Stabilised bi-conjugate gradient on the operator itself (Sec. 3.3 lists
// BiCGstab among the GPU-ported inverters; van der Vorst 1992), for Dhat_p
// (or D on the full lattice), one or many right-hand sides, FP64 or mixed
// precision.
//
// Per iteration: rho = <r^, r>; beta = (rho / rho_old)(alpha / omega);
// p = r + beta (p - omega v); v = A p; alpha = rho / <r^, v>; s = r - alpha v;
// t = A s; omega = <t, s> / <t, t>; x += alpha p + omega s; r = s - omega t.
// That is 4 hopping launches and 5 fused vector launches; every inner
// product is a deterministic FP64 block reduction whose last block computes
// the next scalar on the device, so an iteration has no host round trip and
// chunks of iterations are replayed from a CUDA graph.  A right-hand side
// whose |r| reached its stop value is frozen (alpha = omega = beta = 0 keeps
// x and r unchanged).  Mixed precision is FP64 defect correction around an
// FP32 inner BiCGstab, with the FP64 true residual b - A x.
#include <algorithm>
#include <chrono>
#include <math.h>
#include <string.h>

#include "blas_dev.cuh"

namespace {

#define BI_MAXRHS HR_MAX_RHS
// device scalars, [field][rhs]; complex values use two doubles
enum { Q_RHO = 0, Q_RHO_OLD = 2, Q_ALPHA = 4, Q_OMEGA = 6, Q_BETA = 8, Q_RR = 10, Q_STOP = 11, Q_FROZEN = 12,
       Q_BNORM = 13, Q_NS = 14 };

struct BiScal {
  double *q;          // [Q_NS][BI_MAXRHS]
  double *partials;   // [BI_MAXRHS][2*HR_RED_MAXBLK][4]
  unsigned *count;    // [BI_MAXRHS]
  int *err;
  int *iters;
};

__device__ __forceinline__ double *QS(const BiScal &b, int f, int rhs) { return b.q + (size_t)f * BI_MAXRHS + rhs; }

// K-value version of the deterministic block reduction; returns true in thread
// 0 of the last block of `slot`, with the sums in tot.
template <int K>
__device__ bool reduce_k(const double (&v)[K], const BiScal &b, int slot, int part, int nparts, double (&tot)[K]) {
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = block_sum(v[k]);
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) b.partials[((size_t)slot * 2 * HR_RED_MAXBLK + part) * 4 + k] = s[k];
    __threadfence();
    const unsigned prev = atomicAdd(&b.count[slot], 1u);
    last = (prev == (unsigned)nparts - 1u);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double t[K];
#pragma unroll
  for (int k = 0; k < K; ++k) t[k] = 0.0;
  if (threadIdx.x < 32) {
    for (int p = threadIdx.x; p < nparts; p += 32)
#pragma unroll
      for (int k = 0; k < K; ++k)
        t[k] += ((volatile double *)b.partials)[((size_t)slot * 2 * HR_RED_MAXBLK + p) * 4 + k];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
  }
  if (threadIdx.x != 0) return false;
  b.count[slot] = 0u;
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = t[k];
  return true;
}

__device__ __forceinline__ cx<double> cdiv(cx<double> a, cx<double> b) {
  const double den = b.x * b.x + b.y * b.y;
  return mk((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ cx<double> cmul(cx<double> a, cx<double> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ cx<double> ldq(const BiScal &b, int f, int rhs) { return mk(*QS(b, f, rhs), *QS(b, f + 1, rhs)); }
__device__ __forceinline__ void stq(const BiScal &b, int f, int rhs, cx<double> v) {
  *QS(b, f, rhs) = v.x;
  *QS(b, f + 1, rhs) = v.y;
}

#define SITES ((int64_t)blockIdx.x * blockDim.x + threadIdx.x), ((int64_t)gridDim.x * blockDim.x)
#define SLOT(f) (blockIdx.y / (f).nsub), ((blockIdx.y % (f).nsub) * gridDim.x + blockIdx.x), (gridDim.x * (f).nsub)

// complex <a, b> (and optionally |a|^2) over one sub-field
template <int P>
__device__ __forceinline__ void cdot_sites(const char *a, const char *b, int64_t Vh, int d, int64_t i0, int64_t st,
                                           double &re, double &im, double &aa) {
  typedef typename PT<P>::A A;
  for (int64_t i = i0; i < Vh; i += st) {
    A sr = 0, si = 0, sa = 0;
    for (int c = 0; c < d; ++c) {
      cx<A> av[4], bv[4];
      ldc<P>(a, Vh, d, i, c, av);
      ldc<P>(b, Vh, d, i, c, bv);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        sr += av[q].x * bv[q].x + av[q].y * bv[q].y;
        si += av[q].x * bv[q].y - av[q].y * bv[q].x;
        sa += av[q].x * av[q].x + av[q].y * av[q].y;
      }
    }
    re += (double)sr;
    im += (double)si;
    aa += (double)sa;
  }
}

// p = r + beta (p - omega v)
template <int P>
__global__ void bi_p_kernel(char *p, const char *r, const char *v, FieldDesc f, BiScal b) {
  typedef typename PT<P>::A A;
  const int rhs = blockIdx.y / f.nsub;
  if (*QS(b, Q_FROZEN, rhs) != 0.0) return;
  const cx<double> be = ldq(b, Q_BETA, rhs), om = ldq(b, Q_OMEGA, rhs);
  const cx<double> bo = cmul(be, om);
  const size_t off = (size_t)blockIdx.y * f.fb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f.Vh; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < f.d; ++c) {
      cx<A> pv[4], rv[4], vv[4];
      ldc<P>(p + off, f.Vh, f.d, i, c, pv);
      ldc<P>(r + off, f.Vh, f.d, i, c, rv);
      ldc<P>(v + off, f.Vh, f.d, i, c, vv);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // r + be p - (be om) v
        const A x = rv[q].x + (A)be.x * pv[q].x - (A)be.y * pv[q].y - (A)bo.x * vv[q].x + (A)bo.y * vv[q].y;
        const A y = rv[q].y + (A)be.x * pv[q].y + (A)be.y * pv[q].x - (A)bo.x * vv[q].y - (A)bo.y * vv[q].x;
        pv[q] = mk(x, y);
      }
      stc<P>(p + off, f.Vh, i, c, pv, 1.f);
    }
}

// alpha = rho / <r^, v>
template <int P>
__global__ void bi_alpha_kernel(const char *rh, const char *v, FieldDesc f, BiScal b) {
  const size_t off = (size_t)blockIdx.y * f.fb;
  double re = 0, im = 0, aa = 0;
  cdot_sites<P>(rh + off, v + off, f.Vh, f.d, SITES, re, im, aa);
  const double vv[2] = {re, im};
  double tot[2];
  const int rhs = blockIdx.y / f.nsub;
  if (reduce_k<2>(vv, b, SLOT(f), tot)) {
    if (*QS(b, Q_FROZEN, rhs) != 0.0) {
      stq(b, Q_ALPHA, rhs, mk(0.0, 0.0));
      return;
    }
    const cx<double> den = mk(tot[0], tot[1]);
    if (!(den.x != 0.0 || den.y != 0.0) || !isfinite(den.x) || !isfinite(den.y)) {
      atomicExch(b.err, 1);
      stq(b, Q_ALPHA, rhs, mk(0.0, 0.0));
      return;
    }
    stq(b, Q_ALPHA, rhs, cdiv(ldq(b, Q_RHO, rhs), den));
  }
}

// s = r - alpha v   (s may alias nothing)
template <int P>
__global__ void bi_s_kernel(char *s, const char *r, const char *v, FieldDesc f, BiScal b) {
  typedef typename PT<P>::A A;
  const int rhs = blockIdx.y / f.nsub;
  const cx<double> al = ldq(b, Q_ALPHA, rhs);
  const size_t off = (size_t)blockIdx.y * f.fb;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f.Vh; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < f.d; ++c) {
      cx<A> rv[4], vv[4];
      ldc<P>(r + off, f.Vh, f.d, i, c, rv);
      ldc<P>(v + off, f.Vh, f.d, i, c, vv);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        rv[q] = mk(rv[q].x - (A)al.x * vv[q].x + (A)al.y * vv[q].y, rv[q].y - (A)al.x * vv[q].y - (A)al.y * vv[q].x);
      stc<P>(s + off, f.Vh, i, c, rv, 1.f);
    }
}

// omega = <t, s> / <t, t>
template <int P>
__global__ void bi_omega_kernel(const char *t, const char *s, FieldDesc f, BiScal b) {
  const size_t off = (size_t)blockIdx.y * f.fb;
  double re = 0, im = 0, aa = 0;
  cdot_sites<P>(t + off, s + off, f.Vh, f.d, SITES, re, im, aa);
  const double vv[3] = {re, im, aa};
  double tot[3];
  const int rhs = blockIdx.y / f.nsub;
  if (reduce_k<3>(vv, b, SLOT(f), tot)) {
    if (*QS(b, Q_FROZEN, rhs) != 0.0) {
      stq(b, Q_OMEGA, rhs, mk(0.0, 0.0));
      return;
    }
    if (!(tot[2] > 0.0) || !isfinite(tot[2])) {
      atomicExch(b.err, 1);
      stq(b, Q_OMEGA, rhs, mk(0.0, 0.0));
      return;
    }
    stq(b, Q_OMEGA, rhs, mk(tot[0] / tot[2], tot[1] / tot[2]));
  }
}

// x += alpha p + omega s; r = s - omega t; rho' = <r^, r>, |r|^2; beta, freeze
template <int P>
__global__ void bi_xr_kernel(char *x, char *r, const char *p, const char *s, const char *t, const char *rh,
                             FieldDesc f, BiScal b) {
  typedef typename PT<P>::A A;
  const int rhs = blockIdx.y / f.nsub;
  const bool frozen = *QS(b, Q_FROZEN, rhs) != 0.0;
  const cx<double> al = ldq(b, Q_ALPHA, rhs), om = ldq(b, Q_OMEGA, rhs);
  const size_t off = (size_t)blockIdx.y * f.fb;
  double re = 0, im = 0, rr = 0;
  if (!frozen) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < f.Vh; i += (int64_t)gridDim.x * blockDim.x) {
      A sr = 0, si = 0, sa = 0;
      for (int c = 0; c < f.d; ++c) {
        cx<A> xv[4], pv[4], sv[4], tv[4], hv[4];
        ldc<P>(x + off, f.Vh, f.d, i, c, xv);
        ldc<P>(p + off, f.Vh, f.d, i, c, pv);
        ldc<P>(s + off, f.Vh, f.d, i, c, sv);
        ldc<P>(t + off, f.Vh, f.d, i, c, tv);
        ldc<P>(rh + off, f.Vh, f.d, i, c, hv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xv[q] = mk(xv[q].x + (A)al.x * pv[q].x - (A)al.y * pv[q].y + (A)om.x * sv[q].x - (A)om.y * sv[q].y,
                     xv[q].y + (A)al.x * pv[q].y + (A)al.y * pv[q].x + (A)om.x * sv[q].y + (A)om.y * sv[q].x);
          sv[q] = mk(sv[q].x - (A)om.x * tv[q].x + (A)om.y * tv[q].y, sv[q].y - (A)om.x * tv[q].y - (A)om.y * tv[q].x);
          sr += hv[q].x * sv[q].x + hv[q].y * sv[q].y;
          si += hv[q].x * sv[q].y - hv[q].y * sv[q].x;
          sa += sv[q].x * sv[q].x + sv[q].y * sv[q].y;
        }
        stc<P>(x + off, f.Vh, i, c, xv, 1.f);
        stc<P>(r + off, f.Vh, i, c, sv, 1.f);
      }
      re += (double)sr;
      im += (double)si;
      rr += (double)sa;
    }
  }
  const double vv[3] = {re, im, rr};
  double tot[3];
  if (reduce_k<3>(vv, b, SLOT(f), tot)) {
    if (frozen) return;
    if (b.iters) b.iters[rhs] += 1;
    const cx<double> rho = mk(tot[0], tot[1]);
    *QS(b, Q_RR, rhs) = tot[2];
    if (tot[2] <= *QS(b, Q_STOP, rhs)) {
      *QS(b, Q_FROZEN, rhs) = 1.0;
      stq(b, Q_BETA, rhs, mk(0.0, 0.0));
      return;
    }
    const cx<double> rho_old = ldq(b, Q_RHO, rhs);
    // beta = (rho / rho_old) (alpha / omega)
    const cx<double> be = cmul(cdiv(rho, rho_old), cdiv(al, om));
    if (!isfinite(be.x) || !isfinite(be.y)) atomicExch(b.err, 1);
    stq(b, Q_BETA, rhs, be);
    stq(b, Q_RHO, rhs, rho);
  }
}

}  // namespace

// --------------------------------------------------------------------- driver
// What an instantiated chunk graph depends on (lattice geometry and buffers,
// operator parameters, launch shape): replayed only while all of it matches.
struct BiGraphKey {
  const void *lat, *links, *rlinks, *tmp, *clover, *clover_inv;
  int T, L, d, prec, nrhs, parity, check_every, shape;
  const void *f;
  size_t fb;
  double m0, csw;
};

struct BiWork {
  size_t cap[3];
  void *f[3][8];  // per precision: x, r, rhat, p, v, s, t, spare
  double *q;
  double *partials;
  unsigned *count;
  int *err, *iters;
  double *host;
  cudaStream_t s;
  cudaGraphExec_t exec[2];  // last chunk graph per inner precision (FP64, FP32)
  BiGraphKey key[2];
};

static BiWork *g_bi = nullptr;  // one workspace per process, grown as needed (guarded by callers' serialisation)

static int bi_work(int prec, size_t bytes) {
  if (!g_bi) {
    g_bi = new BiWork;
    memset(g_bi, 0, sizeof(*g_bi));
    HR_CUDA(cudaMalloc(&g_bi->q, sizeof(double) * Q_NS * BI_MAXRHS));
    HR_CUDA(cudaMalloc(&g_bi->partials, sizeof(double) * BI_MAXRHS * 2 * HR_RED_MAXBLK * 4));
    HR_CUDA(cudaMalloc(&g_bi->count, sizeof(unsigned) * BI_MAXRHS));
    HR_CUDA(cudaMemset(g_bi->count, 0, sizeof(unsigned) * BI_MAXRHS));
    HR_CUDA(cudaMalloc(&g_bi->err, sizeof(int)));
    HR_CUDA(cudaMemset(g_bi->err, 0, sizeof(int)));
    HR_CUDA(cudaMalloc(&g_bi->iters, sizeof(int) * BI_MAXRHS));
    HR_CUDA(cudaMallocHost(&g_bi->host, sizeof(double) * Q_NS * BI_MAXRHS));
    HR_CUDA(cudaStreamCreateWithFlags(&g_bi->s, cudaStreamNonBlocking));
  }
  if (g_bi->cap[prec] < bytes) {
    HR_CUDA(cudaDeviceSynchronize());
    for (int k = 0; k < 2; ++k)  // the graphs refer to the buffers about to be replaced
      if (g_bi->exec[k]) {
        cudaGraphExecDestroy(g_bi->exec[k]);
        g_bi->exec[k] = nullptr;
      }
    for (int k = 0; k < 8; ++k) {
      hr_dev_free(g_bi->f[prec][k]);
      g_bi->f[prec][k] = nullptr;
    }
    g_bi->cap[prec] = 0;
    for (int k = 0; k < 8; ++k) HR_TRY(hr_dev_alloc(&g_bi->f[prec][k], bytes));
    g_bi->cap[prec] = bytes;
  }
  return HR_OK;
}

struct BiCtx {
  hr_lattice *lat;
  int parity, nrhs, prec;
  double m0, csw;
  FieldDesc f;
  BiScal sc;
  cudaStream_t s;
};

static int bi_iteration(BiCtx &c) {
  char **F = reinterpret_cast<char **>(g_bi->f[c.prec]);
  char *x = F[0], *r = F[1], *rh = F[2], *p = F[3], *v = F[4], *s = F[5], *t = F[6];
  const dim3 grid(hr_blas_blocks(c.f.Vh), c.nrhs * c.f.nsub);
#define L3(K, ...)                                                                  \
  do {                                                                              \
    if (c.prec == HR_F64) K<0><<<grid, 256, 0, c.s>>>(__VA_ARGS__);                 \
    else K<1><<<grid, 256, 0, c.s>>>(__VA_ARGS__);                                  \
    HR_TRY(hr_check_launch(#K));                                                    \
  } while (0)
  // hops of right-hand sides already frozen (|r|^2 <= stop) return at once
  const double *rr = g_bi->q + (size_t)Q_RR * BI_MAXRHS, *stop = g_bi->q + (size_t)Q_STOP * BI_MAXRHS;
  L3(bi_p_kernel, p, r, v, c.f, c.sc);
  HR_TRY(hr_dphi_impl_skip(c.lat, v, p, c.parity, c.m0, c.csw, c.prec, c.nrhs, 0, c.s, rr, stop));
  L3(bi_alpha_kernel, rh, v, c.f, c.sc);
  L3(bi_s_kernel, s, r, v, c.f, c.sc);
  HR_TRY(hr_dphi_impl_skip(c.lat, t, s, c.parity, c.m0, c.csw, c.prec, c.nrhs, 0, c.s, rr, stop));
  L3(bi_omega_kernel, t, s, c.f, c.sc);
  L3(bi_xr_kernel, x, r, p, s, t, rh, c.f, c.sc);
#undef L3
  return HR_OK;
}

// Inner BiCGstab on A e = r0 (fields in g_bi->f[prec]: r = r0 on entry, x = 0).
static int bi_loop(BiCtx &c, const double *stop, int check_every, int maxit, int *done_out) {
  const int nrhs = c.nrhs;
  char **F = reinterpret_cast<char **>(g_bi->f[c.prec]);
  const size_t bytes = c.f.fb * c.f.nsub * nrhs;
  // rhat = r, p = v = 0, rho = <r, r>, alpha = omega = rho_old = 1 -> beta = rho
  HR_CUDA(cudaMemcpyAsync(F[2], F[1], bytes, cudaMemcpyDeviceToDevice, c.s));
  HR_CUDA(cudaMemsetAsync(F[3], 0, bytes, c.s));
  HR_CUDA(cudaMemsetAsync(F[4], 0, bytes, c.s));
  double *q = g_bi->host;
  for (int k = 0; k < Q_NS * BI_MAXRHS; ++k) q[k] = 0.0;
  for (int r = 0; r < nrhs; ++r) {
    const double rr = stop[BI_MAXRHS + r];  // |r|^2 passed in
    q[Q_RHO * BI_MAXRHS + r] = rr;          // rho = <r^, r> = |r|^2
    q[Q_OMEGA * BI_MAXRHS + r] = 1.0;
    q[Q_ALPHA * BI_MAXRHS + r] = 1.0;
    q[Q_BETA * BI_MAXRHS + r] = 1.0;        // first p = r + 1 (0 - 1 0) = r
    q[Q_RR * BI_MAXRHS + r] = rr;
    q[Q_STOP * BI_MAXRHS + r] = stop[r];
    q[Q_FROZEN * BI_MAXRHS + r] = (rr <= stop[r]) ? 1.0 : 0.0;
  }
  HR_CUDA(cudaMemcpyAsync(g_bi->q, q, sizeof(double) * Q_NS * BI_MAXRHS, cudaMemcpyHostToDevice, c.s));
  // tune the operator outside capture (only while its shape is not known yet),
  // then capture a chunk of iterations -- or replay the last capture of the same key
  const int clover = c.csw != 0.0;
  if (hr_tuned_shape(c.lat, c.prec, nrhs, clover) < 0)
    HR_TRY(hr_dphi_impl(c.lat, F[6], F[5], c.parity, c.m0, c.csw, c.prec, nrhs, 0, c.s));
  if (c.parity != HR_FULL)
    HR_TRY(hr_ensure_tmp(c.lat, hr_spinor_field_bytes(c.lat->Vh, c.lat->d, c.prec) * nrhs));
  BiGraphKey key;
  memset(&key, 0, sizeof(key));
  key.lat = c.lat;
  key.links = c.lat->links[c.prec];
  key.rlinks = c.lat->rlinks[c.prec];
  key.tmp = c.lat->tmp;
  key.clover = clover ? c.lat->clover_A[c.prec == HR_F64 ? 0 : 1] : nullptr;
  key.clover_inv = clover ? c.lat->clover_Ainv[c.prec == HR_F64 ? 0 : 1] : nullptr;
  key.T = c.lat->T;
  key.L = c.lat->L;
  key.d = c.lat->d;
  key.prec = c.prec;
  key.nrhs = nrhs;
  key.parity = c.parity;
  key.check_every = check_every;
  key.shape = hr_tuned_shape(c.lat, c.prec, nrhs, clover);
  key.f = F[0];
  key.fb = c.f.fb;
  key.m0 = c.m0;
  key.csw = c.csw;
  const int slot = (c.prec == HR_F64) ? 0 : 1;
  cudaGraphExec_t exec = nullptr;
  double hops_per = 0.0;
  if (g_bi->exec[slot] && memcmp(&g_bi->key[slot], &key, sizeof(key)) == 0) {
    exec = g_bi->exec[slot];
    hops_per = 4.0 * check_every;  // two operator applications per iteration, two hops each
  } else {
    if (g_bi->exec[slot]) {
      cudaGraphExecDestroy(g_bi->exec[slot]);
      g_bi->exec[slot] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const double hops0 = c.lat->hop_launches;
    HR_CUDA(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
    int rc = HR_OK;
    for (int k = 0; k < check_every && rc == HR_OK; ++k) rc = bi_iteration(c);
    cudaError_t ce = cudaStreamEndCapture(c.s, &graph);
    hops_per = c.lat->hop_launches - hops0;
    c.lat->hop_launches = hops0;
    if (rc != HR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    HR_CUDA(ce);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    HR_CUDA(ce);
    g_bi->exec[slot] = exec;
    g_bi->key[slot] = key;
  }
  int done = 0, status = HR_OK;
  while (done < maxit) {
    HR_CUDA(cudaGraphLaunch(exec, c.s));
    c.lat->hop_launches += hops_per;
    done += check_every;
    HR_CUDA(cudaMemcpyAsync(q, g_bi->q, sizeof(double) * Q_NS * BI_MAXRHS, cudaMemcpyDeviceToHost, c.s));
    HR_CUDA(cudaStreamSynchronize(c.s));
    bool all = true;
    for (int r = 0; r < nrhs; ++r) {
      if (q[Q_FROZEN * BI_MAXRHS + r] == 0.0) all = false;
      if (!isfinite(q[Q_RR * BI_MAXRHS + r])) {
        status = HR_ERR_BREAKDOWN;
        all = true;
      }
    }
    int err = 0;
    HR_CUDA(cudaMemcpy(&err, g_bi->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      HR_CUDA(cudaMemset(g_bi->err, 0, sizeof(int)));
      status = HR_ERR_BREAKDOWN;
      all = true;
    }
    if (all) break;
  }
  *done_out = done;
  return status;
}

// Drop the cached chunk graphs captured on `lat`: called when the lattice is
// destroyed, so that a later lattice that happens to get the same host and
// device addresses never replays kernels bound to the freed buffers.
void hr_bicgstab_forget(const hr_lattice *lat) {
  if (!g_bi) return;
  for (int k = 0; k < 2; ++k)
    if (g_bi->exec[k] && g_bi->key[k].lat == lat) {
      cudaGraphExecDestroy(g_bi->exec[k]);
      g_bi->exec[k] = nullptr;
      memset(&g_bi->key[k], 0, sizeof(g_bi->key[k]));
    }
}

extern "C" int hr_bicgstab_solve(hr_lattice *lat, void *x, const void *b, int parity, double m0, double csw,
                                 const hr_cg_params *prm, hr_cg_stats *st) {
  if (!lat || !x || !b || !prm || parity < HR_EVEN || parity > HR_FULL) return HR_ERR_ARG;
  if (!lat->have_links) return HR_ERR_STATE;
  if (csw != lat->csw) return HR_ERR_ARG;
  const int nrhs = prm->nrhs < 1 ? 1 : prm->nrhs;
  if (nrhs > BI_MAXRHS || prm->tol <= 0.0 || (prm->inner_prec != HR_F64 && prm->inner_prec != HR_F32))
    return HR_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  const int lo = prm->inner_prec, nsub = parity == HR_FULL ? 2 : 1;
  const size_t fb64 = hr_spinor_field_bytes(lat->Vh, lat->d, HR_F64);
  const size_t fblo = hr_spinor_field_bytes(lat->Vh, lat->d, lo);
  HR_TRY(bi_work(HR_F64, fb64 * nsub * nrhs));
  if (lo != HR_F64) HR_TRY(bi_work(lo, fblo * nsub * nrhs));
  HR_TRY(hr_red_scratch(lat, nrhs));
  if (csw != 0.0) HR_TRY(hr_clover_prepare(lat, m0));
  if (parity != HR_FULL) HR_TRY(hr_ensure_tmp(lat, fb64 * nrhs));
  cudaStream_t s = g_bi->s;
  HrEvent ev_owner;
  HR_CUDA(cudaEventCreateWithFlags(&ev_owner.e, cudaEventDisableTiming));
  cudaEvent_t ev = ev_owner.e;
  HR_CUDA(cudaEventRecord(ev, lat->stream));
  HR_CUDA(cudaStreamWaitEvent(s, ev, 0));
  HR_CUDA(cudaMemsetAsync(g_bi->iters, 0, sizeof(int) * BI_MAXRHS, s));
  FieldDesc f64{lat->Vh, lat->d, fb64, nsub}, flo{lat->Vh, lat->d, fblo, nsub};
  BiCtx c;
  c.lat = lat;
  c.parity = parity;
  c.nrhs = nrhs;
  c.prec = lo;
  c.m0 = m0;
  c.csw = csw;
  c.f = flo;
  c.sc = BiScal{g_bi->q, g_bi->partials, g_bi->count, g_bi->err, g_bi->iters};
  c.s = s;
  // FP64 outer: R = b - A X (A = Dhat or D); lattice reduction scratch for norms
  RedArgs red;
  memset(&red, 0, sizeof(red));
  red.partials = lat->red_partials;
  red.count = lat->red_count;
  red.out = lat->red_out;
  red.err = lat->dev_err;
  double *sa = g_bi->q + (size_t)Q_BNORM * BI_MAXRHS;  // scratch scalars for axpby (a)
  double *sb = g_bi->q + (size_t)Q_STOP * BI_MAXRHS;   // (reused before the inner loop sets it)
  char *R = (char *)g_bi->f[HR_F64][7];                 // FP64 residual
  char *AX = (char *)g_bi->f[HR_F64][6];
  auto setv = [&](double *dev, const double *v) -> int {
    HR_CUDA(cudaMemcpyAsync(dev, v, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    HR_CUDA(cudaStreamSynchronize(s));
    return HR_OK;
  };
  auto norms = [&](double *out) -> int {
    HR_CUDA(cudaMemcpyAsync(out, lat->red_out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    HR_CUDA(cudaStreamSynchronize(s));
    return HR_OK;
  };
  double one[BI_MAXRHS], zero[BI_MAXRHS], mone[BI_MAXRHS], a[BI_MAXRHS], bn2[BI_MAXRHS], rn2[BI_MAXRHS],
      stop[2 * BI_MAXRHS];
  for (int k = 0; k < BI_MAXRHS; ++k) {
    one[k] = 1.0;
    zero[k] = 0.0;
    mone[k] = -1.0;
  }
  const size_t bytes64 = fb64 * nsub * nrhs;
  // outer residuals in float-float where that operator is built (mixed solves):
  // the iterate and b then live in the FP64 workspace's x and r buffers, which
  // the mixed solve does not otherwise use
  int use_ff = 0;
  if (lo != HR_F64 && prm->outer_prec == HR_FF) HR_TRY(hr_ff_outer_usable(lat, csw != 0.0, m0, nrhs, s, &use_ff));
  const int po = use_ff ? HR_FF : HR_F64;
  void *xo = po == HR_FF ? g_bi->f[HR_F64][0] : x;
  const void *bo = po == HR_FF ? g_bi->f[HR_F64][1] : b;
  HR_CUDA(cudaMemsetAsync(x, 0, bytes64, s));
  HR_TRY(setv(sa, one));
  HR_TRY(setv(sb, zero));
  HR_TRY(hr_blas_axpby(HR_F64, po, b, R, f64, f64, nrhs, sa, sb, red, 1, s));
  HR_TRY(norms(bn2));
  if (po == HR_FF) {
    HR_CUDA(cudaMemcpyAsync(g_bi->f[HR_F64][1], R, bytes64, cudaMemcpyDeviceToDevice, s));
    HR_CUDA(cudaMemsetAsync(xo, 0, bytes64, s));
  }
  for (int r = 0; r < nrhs; ++r) rn2[r] = bn2[r];
  const double inner_tol = prm->inner_tol > 0.0 ? prm->inner_tol : 1e-5;
  const int check_every = prm->check_every > 0 ? prm->check_every : 10;
  const int maxit = prm->maxit > 0 ? prm->maxit : 100000;
  int status = HR_OK, iters = 0, outer = 0;
  while (true) {
    bool ok = true;
    for (int r = 0; r < nrhs; ++r)
      if (!(rn2[r] <= prm->tol * prm->tol * bn2[r])) ok = false;
    if (ok) break;
    if (iters >= maxit || outer >= 200) {
      status = HR_ERR_NOT_CONVERGED;
      break;
    }
    // inner system A e = R / |R| in precision lo (FP64: R itself, target tol)
    for (int r = 0; r < nrhs; ++r) {
      const double rn = sqrt(rn2[r]);
      a[r] = rn > 0.0 ? 1.0 / rn : 0.0;
      double tg = prm->tol * sqrt(bn2[r]) / (2.0 * (rn > 0.0 ? rn : 1.0));
      if (lo != HR_F64 && tg < inner_tol) tg = inner_tol;
      stop[r] = rn > 0.0 ? tg * tg : 1e300;  // relative to the unit-norm inner residual
      stop[BI_MAXRHS + r] = rn > 0.0 ? 1.0 : 0.0;
    }
    HR_TRY(setv(sa, a));
    HR_TRY(setv(sb, zero));
    char **F = reinterpret_cast<char **>(g_bi->f[lo]);
    HR_TRY(hr_blas_axpby(po, lo, R, F[1], f64, flo, nrhs, sa, sb, red, 0, s));
    HR_CUDA(cudaMemsetAsync(F[0], 0, fblo * nsub * nrhs, s));
    int done = 0;
    status = bi_loop(c, stop, check_every, maxit - iters, &done);
    iters += done;
    ++outer;
    if (status != HR_OK) break;
    // x += |R| e; R = b - A x (in precision po)
    for (int r = 0; r < nrhs; ++r) a[r] = sqrt(rn2[r]);
    HR_TRY(setv(sa, a));
    HR_TRY(setv(sb, one));
    HR_TRY(hr_blas_axpby(lo, po, F[0], xo, flo, f64, nrhs, sa, sb, red, 0, s));
    HR_TRY(hr_dphi_impl(lat, AX, xo, parity, m0, csw, po, nrhs, 0, s));
    HR_TRY(setv(sa, one));
    HR_TRY(setv(sb, zero));
    HR_TRY(hr_blas_axpby(po, po, bo, R, f64, f64, nrhs, sa, sb, red, 0, s));
    HR_TRY(setv(sa, mone));
    HR_TRY(setv(sb, one));
    HR_TRY(hr_blas_axpby(po, po, AX, R, f64, f64, nrhs, sa, sb, red, 1, s));
    HR_TRY(norms(rn2));
  }
  if (po == HR_FF) {  // x = the FP64 value of the float-float iterate
    HR_TRY(setv(sa, one));
    HR_TRY(setv(sb, zero));
    HR_TRY(hr_blas_axpby(HR_FF, HR_F64, xo, x, f64, f64, nrhs, sa, sb, red, 0, s));
  }
  HR_CUDA(cudaStreamSynchronize(s));
  if (st) {
    int it[BI_MAXRHS];
    HR_CUDA(cudaMemcpy(it, g_bi->iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost));
    int mx = 0;
    double res = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      mx = std::max(mx, it[r]);
      res = std::max(res, bn2[r] > 0.0 ? sqrt(rn2[r] / bn2[r]) : 0.0);
    }
    st->iterations = mx;
    st->outer_steps = outer;
    st->true_residual = res;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st->hop_launches = 0.0;
  }
  return status;
}
