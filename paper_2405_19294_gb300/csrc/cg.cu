// Conjugate gradient on the normal equations (Sec. 3.3), plain FP64 or mixed
// precision, for one or many right-hand sides at once.
//
// One CG iteration is seven launches with no host round trip:
//   t = Dhat p, Ap = Dhat^+ t           (4 hopping launches)
//   pAp = |t|^2, alpha = rr / pAp       (reduction; scalars stay on the GPU)
//   x += alpha p, r -= alpha Ap, rr'    (fused update + reduction, beta = rr'/rr)
//   p = r + beta p
// A chunk of `check_every` iterations is captured once into a CUDA graph and
// replayed; after each chunk the host reads |r|^2 per right-hand side.  A
// right-hand side whose recursive residual reached its stop value is frozen
// on the device (alpha = 0) while the others continue.
//
// Mixed precision is defect correction: the FP64 residual r = b - M x is
// rescaled to unit norm, the inner CG (FP32, or FP16 operator fields with
// per-site scales and FP32 x, r) reduces it by inner_tol, x += |r| e in FP64,
// and r is recomputed exactly in FP64, until |r| <= tol |b|.  With
// outer_prec = HR_FF the outer iterate, b and r are float-float fields and r is
// recomputed by the float-float operator (about 48 bits, on the FP32 pipes);
// x is written back in FP64 at exit.  With an FP16
// inner solver a middle level sits in between: the FP16 CG restarts from FP32
// true residuals (r32 - M e32, FP32 operator) until the FP32 system has
// dropped by HR_MID_TOL, and only then is the (expensive on this part) FP64
// residual recomputed -- as many FP64 residuals as FP32-inner needs.
#define HR_MID_TOL 1e-5
#include <algorithm>
#include <chrono>
#include <math.h>
#include <string.h>

#include "blas.cuh"
#include "hr_internal.h"

// What an instantiated chunk graph depends on: replaying it is only valid for
// the same fields, scratch, shapes and operator parameters.
struct CgGraphKey {
  int pr, pp, check_every, nrhs, parity, shape;
  const void *x, *r, *p, *Ap, *t, *tmp;
  const void *links, *rlinks, *clover, *clover_inv;  // operator buffers the captured hops read
  size_t fbr, fbp;
  int64_t Vh;
  int nsub;
  double m0, csw;
};

struct hr_cg_work {
  size_t cap[3];        // bytes per buffer set, per precision
  void *f[3][6];        // per precision: r, p, Ap, t, x(low), spare
  double *scal;         // device scalars: [NS][HR_MAX_RHS]
  double *host;         // pinned mirror
  int *iters;           // [HR_MAX_RHS]
  cudaStream_t s;
  cudaGraphExec_t exec[2];  // the last chunk graphs (one per inner precision pair seen), reused while
  CgGraphKey key[2];        // their key matches: capture and instantiation cost ~1 ms each
};

enum { S_RR0 = 0, S_RR1, S_PAP, S_ALPHA, S_BETA, S_STOP, S_A, S_B, S_OUT, NS };

void hr_cg_free(hr_lattice *lat) {
  hr_cg_work *w = lat->cg;
  if (!w) return;
  for (int k = 0; k < 2; ++k)
    if (w->exec[k]) cudaGraphExecDestroy(w->exec[k]);
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 6; ++q) hr_dev_free(w->f[p][q]);
  cudaFree(w->scal);
  cudaFree(w->iters);
  cudaFreeHost(w->host);
  if (w->s) cudaStreamDestroy(w->s);
  delete w;
  lat->cg = nullptr;
}

static int cg_work(hr_lattice *lat, int prec, size_t bytes) {
  if (!lat->cg) {
    hr_cg_work *w = new hr_cg_work;
    memset(w, 0, sizeof(*w));
    lat->cg = w;
    HR_CUDA(cudaMalloc(&w->scal, sizeof(double) * NS * HR_MAX_RHS));
    HR_CUDA(cudaMemset(w->scal, 0, sizeof(double) * NS * HR_MAX_RHS));
    HR_CUDA(cudaMalloc(&w->iters, sizeof(int) * HR_MAX_RHS));
    HR_CUDA(cudaMallocHost(&w->host, sizeof(double) * NS * HR_MAX_RHS));
    HR_CUDA(cudaStreamCreateWithFlags(&w->s, cudaStreamNonBlocking));
  }
  hr_cg_work *w = lat->cg;
  if (w->cap[prec] < bytes) {
    for (int k = 0; k < 2; ++k)  // the graphs refer to the buffers about to be replaced
      if (w->exec[k]) {
        cudaGraphExecDestroy(w->exec[k]);
        w->exec[k] = nullptr;
      }
    for (int q = 0; q < 6; ++q) {
      hr_dev_free(w->f[prec][q]);
      w->f[prec][q] = nullptr;
    }
    w->cap[prec] = 0;
    for (int q = 0; q < 6; ++q) HR_TRY(hr_dev_alloc(&w->f[prec][q], bytes));
    w->cap[prec] = bytes;
  }
  return HR_OK;
}

static double *S(hr_cg_work *w, int k) { return w->scal + (size_t)k * HR_MAX_RHS; }

int hr_cg_workspace(hr_lattice *lat, int prec, size_t bytes) { return cg_work(lat, prec, bytes); }
void *hr_cg_field(hr_lattice *lat, int prec, int which) { return lat->cg ? lat->cg->f[prec][which] : nullptr; }

struct CgCtx {
  hr_lattice *lat;
  int parity, nrhs, dagger_unused;
  double m0, csw;
  cudaStream_t s;
  RedArgs red;
};

// Ap = M p = Dhat^+ Dhat p through t; fused |t|^2 -> pAp and alpha
// Inside a CG chunk (rr given) the hops of right-hand sides already at their
// stop value return at once: a chunk runs past convergence by up to
// check_every - 1 iterations, and those cost only launches, not the stencil.
static int apply_normal(CgCtx &c, int prec, void *Ap, const void *p, void *t, const FieldDesc &f, int finish,
                        const double *rr) {
  const double *stop = rr ? c.red.stop : nullptr;
  HR_TRY(hr_dphi_impl_skip(c.lat, t, p, c.parity, c.m0, c.csw, prec, c.nrhs, 0, c.s, rr, stop));
  RedArgs red = c.red;
  red.out = S(c.lat->cg, S_PAP);
  red.rr = rr;
  red.alpha = S(c.lat->cg, S_ALPHA);
  if (finish != RED_NONE_SKIP) HR_TRY(hr_blas_norm2(f, prec, t, c.nrhs, red, finish, c.s));
  HR_TRY(hr_dphi_impl_skip(c.lat, Ap, t, c.parity, c.m0, c.csw, prec, c.nrhs, 1, c.s, rr, stop));
  return HR_OK;
}

// one CG iteration on fields (x, r: prec pr; p, Ap, t: prec pp); rr buffers alternate
static int cg_iteration(CgCtx &c, int pr, int pp, void *x, void *r, void *p, void *Ap, void *t, const FieldDesc &fr,
                        const FieldDesc &fp, int odd) {
  hr_cg_work *w = c.lat->cg;
  double *rr = S(w, odd ? S_RR1 : S_RR0);
  double *rr_next = S(w, odd ? S_RR0 : S_RR1);
  HR_TRY(apply_normal(c, pp, Ap, p, t, fp, RED_ALPHA, rr));
  RedArgs red = c.red;
  red.out = S(w, S_OUT);
  red.rr = rr;
  red.rr_next = rr_next;
  red.alpha = S(w, S_ALPHA);
  red.beta = S(w, S_BETA);
  HR_TRY(hr_blas_cg_xr(pr, pp, x, r, p, Ap, fr, fp, c.nrhs, red, c.s));
  HR_TRY(hr_blas_cg_p(pr, pp, r, p, fr, fp, c.nrhs, S(w, S_BETA), S(w, S_ALPHA), c.s));
  return HR_OK;
}

// Run CG iterations until every rhs is frozen (rr <= stop) or maxit.  Fields
// must be initialised: r, p = r, x = 0, rr in S_RR0, stop in S_STOP.
static int cg_loop(CgCtx &c, int pr, int pp, void *x, void *r, void *p, void *Ap, void *t, const FieldDesc &fr,
                   const FieldDesc &fp, int check_every, int maxit, int *iters_done) {
  hr_cg_work *w = c.lat->cg;
  if (check_every < 2) check_every = 2;
  check_every &= ~1;  // even: the rr double buffer returns to S_RR0
  const int clover = c.csw != 0.0;
  // an uncaptured application first when the hop shape is not tuned yet: the
  // autotuner times candidates, which it cannot do while the stream is being
  // captured (t and Ap are scratch)
  if (hr_tuned_shape(c.lat, pp, c.nrhs, clover) < 0) {
    HR_TRY(hr_dphi_impl(c.lat, t, p, c.parity, c.m0, c.csw, pp, c.nrhs, 0, c.s));
    HR_TRY(hr_dphi_impl(c.lat, Ap, t, c.parity, c.m0, c.csw, pp, c.nrhs, 1, c.s));
  }
  if (c.parity != HR_FULL) HR_TRY(hr_ensure_tmp(c.lat, hr_spinor_field_bytes(c.lat->Vh, c.lat->d, pp) * c.nrhs));
  CgGraphKey key;
  memset(&key, 0, sizeof(key));
  key.pr = pr;
  key.pp = pp;
  key.check_every = check_every;
  key.nrhs = c.nrhs;
  key.parity = c.parity;
  key.shape = hr_tuned_shape(c.lat, pp, c.nrhs, clover);
  key.x = x;
  key.r = r;
  key.p = p;
  key.Ap = Ap;
  key.t = t;
  key.tmp = c.lat->tmp;
  key.links = c.lat->links[pp];
  key.rlinks = c.lat->rlinks[pp];
  key.clover = clover ? c.lat->clover_A[pp == HR_F64 ? 0 : 1] : nullptr;
  key.clover_inv = clover ? c.lat->clover_Ainv[pp == HR_F64 ? 0 : 1] : nullptr;
  key.fbr = fr.fb;
  key.fbp = fp.fb;
  key.Vh = fr.Vh;
  key.nsub = fr.nsub;
  key.m0 = c.m0;
  key.csw = c.csw;
  const int slot = (pp == HR_F16) ? 1 : 0;
  cudaGraphExec_t exec = nullptr;
  double hops_per_replay = 0.0;
  cudaError_t ce = cudaSuccess;
  if (w->exec[slot] && memcmp(&w->key[slot], &key, sizeof(key)) == 0) {
    exec = w->exec[slot];
    hops_per_replay = 4.0 * check_every;  // two Dhat per iteration, two hops each
  } else {
    if (w->exec[slot]) {
      cudaGraphExecDestroy(w->exec[slot]);
      w->exec[slot] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const double hops_before = c.lat->hop_launches;  // capture records launches, replays run them
    HR_CUDA(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
    int rc = HR_OK;
    for (int k = 0; k < check_every && rc == HR_OK; ++k)
      rc = cg_iteration(c, pr, pp, x, r, p, Ap, t, fr, fp, k & 1);
    ce = cudaStreamEndCapture(c.s, &graph);
    hops_per_replay = c.lat->hop_launches - hops_before;
    c.lat->hop_launches = hops_before;
    if (rc != HR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    HR_CUDA(ce);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    HR_CUDA(ce);
    w->exec[slot] = exec;
    w->key[slot] = key;
  }
  int done = 0;
  int status = HR_OK;
  while (done < maxit) {
    ce = cudaGraphLaunch(exec, c.s);
    if (ce != cudaSuccess) break;
    c.lat->hop_launches += hops_per_replay;
    done += check_every;
    ce = cudaMemcpyAsync(w->host, w->scal, sizeof(double) * NS * HR_MAX_RHS, cudaMemcpyDeviceToHost, c.s);
    if (ce != cudaSuccess) break;
    ce = cudaStreamSynchronize(c.s);
    if (ce != cudaSuccess) break;
    bool all = true;
    for (int q = 0; q < c.nrhs; ++q) {
      const double rrq = w->host[S_RR0 * HR_MAX_RHS + q];
      if (!(rrq <= w->host[S_STOP * HR_MAX_RHS + q])) all = false;
      if (!isfinite(rrq)) {
        status = HR_ERR_BREAKDOWN;
        all = true;
      }
    }
    if (all) break;
  }
  if (ce != cudaSuccess) {
    // a failed replay leaves the cached graph in doubt: drop it
    cudaGraphExecDestroy(exec);
    w->exec[slot] = nullptr;
    hr_note_cuda_error(ce, "cg_loop", __FILE__, __LINE__);
    return HR_ERR_CUDA;
  }
  int err = 0;
  HR_CUDA(cudaMemcpy(&err, c.lat->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    HR_CUDA(cudaMemset(c.lat->dev_err, 0, sizeof(int)));
    status = HR_ERR_BREAKDOWN;
  }
  *iters_done = done;
  return status;
}

// r = b - M x in precision po (HR_F64 or HR_FF; r, b, x, Ap and t all in it),
// returns |r|^2 per rhs on the host
static int true_residual(CgCtx &c, int po, void *r, const void *b, const void *x, void *Ap, void *t,
                         const FieldDesc &f, double *rn2) {
  hr_cg_work *w = c.lat->cg;
  HR_TRY(apply_normal(c, po, Ap, x, t, f, RED_NONE_SKIP, nullptr));
  double one[HR_MAX_RHS], zero[HR_MAX_RHS], mone[HR_MAX_RHS];
  for (int q = 0; q < HR_MAX_RHS; ++q) {
    one[q] = 1.0;
    zero[q] = 0.0;
    mone[q] = -1.0;
  }
  HR_CUDA(cudaMemcpyAsync(S(w, S_A), one, sizeof(one), cudaMemcpyHostToDevice, c.s));
  HR_CUDA(cudaMemcpyAsync(S(w, S_B), zero, sizeof(zero), cudaMemcpyHostToDevice, c.s));
  RedArgs red = c.red;
  red.out = S(w, S_OUT);
  HR_TRY(hr_blas_axpby(po, po, b, r, f, f, c.nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
  HR_CUDA(cudaMemcpyAsync(S(w, S_A), mone, sizeof(mone), cudaMemcpyHostToDevice, c.s));
  HR_CUDA(cudaMemcpyAsync(S(w, S_B), one, sizeof(one), cudaMemcpyHostToDevice, c.s));
  HR_TRY(hr_blas_axpby(po, po, Ap, r, f, f, c.nrhs, S(w, S_A), S(w, S_B), red, 1, c.s));
  HR_CUDA(cudaMemcpyAsync(rn2, S(w, S_OUT), sizeof(double) * c.nrhs, cudaMemcpyDeviceToHost, c.s));
  HR_CUDA(cudaStreamSynchronize(c.s));
  return HR_OK;
}

static int set_scalars(CgCtx &c, int which, const double *v) {
  HR_CUDA(cudaMemcpyAsync(S(c.lat->cg, which), v, sizeof(double) * c.nrhs, cudaMemcpyHostToDevice, c.s));
  return HR_OK;
}

extern "C" int hr_cg_solve(hr_lattice *lat, void *x, const void *b, int parity, double m0, double csw,
                           const hr_cg_params *prm, hr_cg_stats *st) {
  if (!lat || !x || !b || !prm || parity < HR_EVEN || parity > HR_FULL) return HR_ERR_ARG;
  if (!lat->have_links) return HR_ERR_STATE;
  if (csw != lat->csw) return HR_ERR_ARG;
  const int nrhs = prm->nrhs < 1 ? 1 : prm->nrhs;
  if (nrhs > HR_MAX_RHS || prm->tol <= 0.0 || prm->inner_prec < HR_F64 || prm->inner_prec > HR_F16)
    return HR_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  const double hop0 = lat->hop_launches;
  const int nsub = parity == HR_FULL ? 2 : 1;
  const int lo = prm->inner_prec;
  const size_t fb64 = hr_spinor_field_bytes(lat->Vh, lat->d, HR_F64);
  HR_TRY(cg_work(lat, HR_F64, fb64 * nsub * nrhs));
  if (lo != HR_F64) {
    HR_TRY(cg_work(lat, HR_F32, hr_spinor_field_bytes(lat->Vh, lat->d, HR_F32) * nsub * nrhs));
    if (lo == HR_F16) HR_TRY(cg_work(lat, HR_F16, hr_spinor_field_bytes(lat->Vh, lat->d, HR_F16) * nsub * nrhs));
  }
  HR_TRY(hr_red_scratch(lat, nrhs));
  if (csw != 0.0) HR_TRY(hr_clover_prepare(lat, m0));
  hr_cg_work *w = lat->cg;
  // the Schur intermediate must exist before graph capture
  if (parity != HR_FULL) {
    size_t mx = fb64;
    HR_TRY(hr_ensure_tmp(lat, mx * nrhs));
  }
  CgCtx c;
  memset(&c, 0, sizeof(c));
  c.lat = lat;
  c.parity = parity;
  c.nrhs = nrhs;
  c.m0 = m0;
  c.csw = csw;
  c.s = w->s;
  c.red.partials = lat->red_partials;
  c.red.count = lat->red_count;
  c.red.err = lat->dev_err;
  c.red.stop = S(w, S_STOP);
  c.red.iters = w->iters;
  // order after the caller's stream
  HrEvent ev_owner;
  HR_CUDA(cudaEventCreateWithFlags(&ev_owner.e, cudaEventDisableTiming));
  cudaEvent_t ev = ev_owner.e;
  HR_CUDA(cudaEventRecord(ev, lat->stream));
  HR_CUDA(cudaStreamWaitEvent(c.s, ev, 0));
  HR_CUDA(cudaMemsetAsync(w->iters, 0, sizeof(int) * HR_MAX_RHS, c.s));

  FieldDesc f64;
  f64.Vh = lat->Vh;
  f64.d = lat->d;
  f64.fb = fb64;
  f64.nsub = nsub;
  const size_t bytes64 = fb64 * nsub * nrhs;
  void *r = w->f[HR_F64][0], *p = w->f[HR_F64][1], *Ap = w->f[HR_F64][2], *t = w->f[HR_F64][3];

  double bn2[HR_MAX_RHS], rn2[HR_MAX_RHS], v[HR_MAX_RHS];
  int status = HR_OK, iters = 0, outer = 0;
  // outer residuals in float-float where that operator is built (mixed solves only)
  int use_ff = 0;
  if (lo != HR_F64 && prm->outer_prec == HR_FF) HR_TRY(hr_ff_outer_usable(lat, csw != 0.0, m0, nrhs, c.s, &use_ff));
  const int po = use_ff ? HR_FF : HR_F64;
  // the outer iterate and b in precision po: x and b themselves for FP64, else
  // the FP64 workspace's spare x and p buffers (p is unused by the mixed solve)
  void *xo = po == HR_FF ? w->f[HR_F64][4] : x;
  const void *bo = po == HR_FF ? w->f[HR_F64][1] : b;
  const int check_every = prm->check_every > 0 ? prm->check_every : 10;
  const int maxit = prm->maxit > 0 ? prm->maxit : 100000;
  // x = 0, r = b, |b|^2
  HR_CUDA(cudaMemsetAsync(x, 0, bytes64, c.s));
  {
    double one[HR_MAX_RHS], zero[HR_MAX_RHS];
    for (int q = 0; q < HR_MAX_RHS; ++q) {
      one[q] = 1.0;
      zero[q] = 0.0;
    }
    HR_TRY(set_scalars(c, S_A, one));
    HR_TRY(set_scalars(c, S_B, zero));
    RedArgs red = c.red;
    red.out = S(w, S_OUT);
    HR_TRY(hr_blas_axpby(HR_F64, po, b, r, f64, f64, nrhs, S(w, S_A), S(w, S_B), red, 1, c.s));
    HR_CUDA(cudaMemcpyAsync(bn2, S(w, S_OUT), sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c.s));
    if (po == HR_FF) {
      HR_CUDA(cudaMemcpyAsync(w->f[HR_F64][1], r, bytes64, cudaMemcpyDeviceToDevice, c.s));
      HR_CUDA(cudaMemsetAsync(xo, 0, bytes64, c.s));
    }
    HR_CUDA(cudaStreamSynchronize(c.s));
  }
  for (int q = 0; q < nrhs; ++q) rn2[q] = bn2[q];

  if (lo == HR_F64) {
    // ---------------------------------------------------------- plain FP64
    HR_CUDA(cudaMemcpyAsync(p, r, bytes64, cudaMemcpyDeviceToDevice, c.s));
    for (int q = 0; q < nrhs; ++q) v[q] = prm->tol * prm->tol * bn2[q];
    HR_TRY(set_scalars(c, S_STOP, v));
    while (true) {
      HR_TRY(set_scalars(c, S_RR0, rn2));
      int done = 0;
      status = cg_loop(c, HR_F64, HR_F64, x, r, p, Ap, t, f64, f64, check_every, maxit - iters, &done);
      iters += done;
      ++outer;
      if (status != HR_OK) break;
      HR_TRY(true_residual(c, HR_F64, r, b, x, Ap, t, f64, rn2));
      bool ok = true;
      for (int q = 0; q < nrhs; ++q)
        if (!(rn2[q] <= prm->tol * prm->tol * bn2[q])) ok = false;
      if (ok) break;
      if (iters >= maxit) {
        status = HR_ERR_NOT_CONVERGED;
        break;
      }
      // restart from the true residual
      HR_CUDA(cudaMemcpyAsync(p, r, bytes64, cudaMemcpyDeviceToDevice, c.s));
    }
  } else {
    // ------------------------------------------------- mixed precision
    const size_t fb32 = hr_spinor_field_bytes(lat->Vh, lat->d, HR_F32);
    const size_t fblo = hr_spinor_field_bytes(lat->Vh, lat->d, lo);
    FieldDesc f32, flo;
    f32 = f64;
    f32.fb = fb32;
    flo = f64;
    flo.fb = fblo;
    void *xl = w->f[HR_F32][4], *rl = w->f[HR_F32][0];
    void *pl = w->f[lo][1], *Apl = w->f[lo][2], *tl = w->f[lo][3];
    const double inner_tol = prm->inner_tol > 0.0 ? prm->inner_tol : (lo == HR_F32 ? 1e-5 : 3e-3);
    const int maxouter = 200;
    while (true) {
      bool ok = true;
      for (int q = 0; q < nrhs; ++q)
        if (!(rn2[q] <= prm->tol * prm->tol * bn2[q])) ok = false;
      if (ok) break;
      if (iters >= maxit || outer >= maxouter) {
        status = HR_ERR_NOT_CONVERGED;
        break;
      }
      // rl = r / |r|, pl = rl, xl = 0; stop = (max(inner_tol, tol |b| / (2 |r|)))^2
      double a[HR_MAX_RHS], zero[HR_MAX_RHS], one[HR_MAX_RHS], stop[HR_MAX_RHS], rr[HR_MAX_RHS];
      for (int q = 0; q < nrhs; ++q) {
        const double rn = sqrt(rn2[q]);
        a[q] = rn > 0.0 ? 1.0 / rn : 0.0;
        zero[q] = 0.0;
        one[q] = 1.0;
        double red_target = prm->tol * sqrt(bn2[q]) / (2.0 * (rn > 0.0 ? rn : 1.0));
        if (red_target < inner_tol) red_target = inner_tol;
        stop[q] = rn > 0.0 ? red_target * red_target : 1e300;
        rr[q] = rn > 0.0 ? 1.0 : 0.0;
      }
      HR_TRY(set_scalars(c, S_A, a));
      HR_TRY(set_scalars(c, S_B, zero));
      RedArgs red = c.red;
      red.out = S(w, S_OUT);
      HR_TRY(hr_blas_axpby(po, HR_F32, r, rl, f64, f32, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
      HR_TRY(set_scalars(c, S_A, one));
      HR_TRY(hr_blas_axpby(HR_F32, lo, rl, pl, f32, flo, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
      HR_CUDA(cudaMemsetAsync(xl, 0, fb32 * nsub * nrhs, c.s));
      HR_TRY(set_scalars(c, S_STOP, stop));
      HR_TRY(set_scalars(c, S_RR0, rr));
      int done = 0;
      status = cg_loop(c, HR_F32, lo, xl, rl, pl, Apl, tl, f32, flo, check_every, maxit - iters, &done);
      iters += done;
      ++outer;
      if (status != HR_OK) break;
      void *xacc = xl;  // the correction to add to x (FP32, unit-norm system)
      if (lo == HR_F16) {
        // middle level: e32 accumulates FP16 solves; rm = r32 - M e32 in FP32
        void *r32 = w->f[HR_F32][5], *e32 = w->f[HR_F32][1], *Ap32 = w->f[HR_F32][2], *t32 = w->f[HR_F32][3];
        double m2[HR_MAX_RHS], mx[HR_MAX_RHS], mz[HR_MAX_RHS], mo[HR_MAX_RHS], minv[HR_MAX_RHS];
        for (int q = 0; q < nrhs; ++q) {
          mx[q] = 1.0;
          mz[q] = 0.0;
          mo[q] = -1.0;
        }
        // r32 = rl_initial is gone (rl was iterated); rebuild it from r: r32 = r / |r|
        HR_TRY(set_scalars(c, S_A, a));  // a = 1/|r| still
        HR_TRY(set_scalars(c, S_B, mz));
        HR_TRY(hr_blas_axpby(po, HR_F32, r, r32, f64, f32, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
        // e32 = xl
        HR_TRY(set_scalars(c, S_A, mx));
        HR_TRY(hr_blas_axpby(HR_F32, HR_F32, xl, e32, f32, f32, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
        for (int mid = 0; mid < 20; ++mid) {
          // rm (in rl) = r32 - M e32, |rm|^2
          HR_TRY(hr_dphi_impl(lat, t32, e32, parity, m0, csw, HR_F32, nrhs, 0, c.s));
          HR_TRY(hr_dphi_impl(lat, Ap32, t32, parity, m0, csw, HR_F32, nrhs, 1, c.s));
          HR_TRY(set_scalars(c, S_A, mx));
          HR_TRY(set_scalars(c, S_B, mz));
          HR_TRY(hr_blas_axpby(HR_F32, HR_F32, r32, rl, f32, f32, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
          HR_TRY(set_scalars(c, S_A, mo));
          HR_TRY(set_scalars(c, S_B, mx));
          HR_TRY(hr_blas_axpby(HR_F32, HR_F32, Ap32, rl, f32, f32, nrhs, S(w, S_A), S(w, S_B), red, 1, c.s));
          HR_CUDA(cudaMemcpyAsync(m2, S(w, S_OUT), sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c.s));
          HR_CUDA(cudaStreamSynchronize(c.s));
          bool mid_done = true;
          for (int q = 0; q < nrhs; ++q) {
            const double goal = std::max(HR_MID_TOL, 0.5 * prm->tol * sqrt(bn2[q] / rn2[q]));
            if (!(m2[q] <= goal * goal)) mid_done = false;
          }
          if (mid_done || iters >= maxit) break;
          // next FP16 solve on M e' = rm / |rm|, then e32 += |rm| e'
          for (int q = 0; q < nrhs; ++q) {
            const double rn = sqrt(m2[q]);
            minv[q] = rn > 0.0 ? 1.0 / rn : 0.0;
            double tg = std::max(inner_tol, 0.5 * prm->tol * sqrt(bn2[q] / rn2[q]) / (rn > 0.0 ? rn : 1.0));
            stop[q] = rn > 0.0 ? tg * tg : 1e300;
            rr[q] = rn > 0.0 ? 1.0 : 0.0;
          }
          HR_TRY(set_scalars(c, S_A, minv));
          HR_TRY(set_scalars(c, S_B, mz));
          HR_TRY(hr_blas_axpby(HR_F32, HR_F32, rl, rl, f32, f32, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
          HR_TRY(set_scalars(c, S_A, mx));
          HR_TRY(hr_blas_axpby(HR_F32, lo, rl, pl, f32, flo, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
          HR_CUDA(cudaMemsetAsync(xl, 0, fb32 * nsub * nrhs, c.s));
          HR_TRY(set_scalars(c, S_STOP, stop));
          HR_TRY(set_scalars(c, S_RR0, rr));
          done = 0;
          status = cg_loop(c, HR_F32, lo, xl, rl, pl, Apl, tl, f32, flo, check_every, maxit - iters, &done);
          iters += done;
          if (status != HR_OK) break;
          for (int q = 0; q < nrhs; ++q) minv[q] = sqrt(m2[q]);
          HR_TRY(set_scalars(c, S_A, minv));
          HR_TRY(set_scalars(c, S_B, mx));
          HR_TRY(hr_blas_axpby(HR_F32, HR_F32, xl, e32, f32, f32, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
        }
        if (status != HR_OK) break;
        xacc = e32;
      }
      // x += |r| xacc
      for (int q = 0; q < nrhs; ++q) a[q] = sqrt(rn2[q]);
      HR_TRY(set_scalars(c, S_A, a));
      HR_TRY(set_scalars(c, S_B, one));
      HR_TRY(hr_blas_axpby(HR_F32, po, xacc, xo, f32, f64, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
      HR_TRY(true_residual(c, po, r, bo, xo, Ap, t, f64, rn2));
    }
    if (po == HR_FF) {  // x = the FP64 value of the float-float iterate
      double one[HR_MAX_RHS], zero[HR_MAX_RHS];
      for (int q = 0; q < HR_MAX_RHS; ++q) {
        one[q] = 1.0;
        zero[q] = 0.0;
      }
      HR_TRY(set_scalars(c, S_A, one));
      HR_TRY(set_scalars(c, S_B, zero));
      RedArgs red = c.red;
      red.out = S(w, S_OUT);
      HR_TRY(hr_blas_axpby(HR_FF, HR_F64, xo, x, f64, f64, nrhs, S(w, S_A), S(w, S_B), red, 0, c.s));
    }
  }
  HR_CUDA(cudaStreamSynchronize(c.s));
  if (st) {
    int it[HR_MAX_RHS];
    HR_CUDA(cudaMemcpy(it, w->iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost));
    int mx = 0;
    double res = 0.0;
    for (int q = 0; q < nrhs; ++q) {
      if (it[q] > mx) mx = it[q];
      const double rq = bn2[q] > 0.0 ? sqrt(rn2[q] / bn2[q]) : 0.0;
      if (rq > res) res = rq;
    }
    st->iterations = mx;
    st->outer_steps = outer;
    st->true_residual = res;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st->hop_launches = lat->hop_launches - hop0;
  }
  return status;
}
