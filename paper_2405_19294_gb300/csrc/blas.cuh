// Descriptors and launchers of the site-wise linear-algebra kernels (blas.cu).
#pragma once

#include "hr_internal.h"

#define HR_RED_MAXBLK 1216  // 8 blocks of 256 threads on each of the 152 SMs
#define HR_MAX_RHS 64

enum RedFinish {
  RED_NONE_SKIP = -1,  // caller-side: no reduction at all
  RED_PLAIN = 0,  // out[rhs] = sum
  RED_ALPHA = 1,  // out[rhs] = pAp; alpha[rhs] = rr / pAp (0 once rr <= stop)
  RED_BETA = 2    // out[rhs] = rr_new; beta[rhs] = rr_new / rr; rr_next[rhs] = rr_new
};

// nrhs x nsub single-parity fields of fb bytes back to back (nsub = 2 for
// full-lattice fields [even | odd]); grid.y runs over all of them and the
// right-hand side of sub-field y is y / nsub.
struct FieldDesc {
  int64_t Vh;
  int d;
  size_t fb;
  int nsub;
};

struct RedArgs {
  double *partials;   // [HR_MAX_RHS][2 * HR_RED_MAXBLK]
  unsigned *count;    // [HR_MAX_RHS], zero between uses
  double *out;        // [nrhs]
  const double *rr;   // current |r|^2 per rhs (RED_ALPHA, RED_BETA)
  double *rr_next;    // RED_BETA
  double *alpha;      // RED_ALPHA writes, RED_BETA reads
  double *beta;       // RED_BETA
  const double *stop; // |r|^2 threshold per rhs
  int *err;           // breakdown flag
  int *iters;         // per-rhs count of non-frozen iterations (RED_ALPHA), may be null
  int *frozen;        // RED_BETA: per-rhs flag rr_next <= stop (multi-lattice hops skip), may be null
};

int hr_blas_blocks(int64_t Vh);
int hr_red_scratch(hr_lattice *lat, int nrhs);
int hr_blas_norm2(const FieldDesc &f, int prec, const void *x, int nrhs, const RedArgs &red, int finish,
                  cudaStream_t s);
int hr_blas_cg_xr(int pr, int pp, void *x, void *r, const void *p, const void *Ap, const FieldDesc &fr,
                  const FieldDesc &fp, int nrhs, const RedArgs &red, cudaStream_t s);
int hr_blas_cg_p(int pr, int pp, const void *r, void *p, const FieldDesc &fr, const FieldDesc &fp, int nrhs,
                 const double *beta, const double *alpha, cudaStream_t s);
int hr_blas_axpby(int px, int py, const void *x, void *y, const FieldDesc &fx, const FieldDesc &fy, int nrhs,
                  const double *a, const double *b, const RedArgs &red, int want_norm, cudaStream_t s);
