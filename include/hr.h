/*
 * hr.h -- C ABI of libhr: the even-odd preconditioned Wilson(-clover) Dirac
 * operator D_R for fermions in a representation R of SU(N), and conjugate
 * gradient on the normal equations built on it, on one GB300 GPU.
 *
 * The paper ("GPU-accelerated Higher Representations of Wilson Fermions with
 * HiRep") provides, on GPUs, the Wilson-Dirac operator for general higher
 * representations of SU(N_c), single and double precision, even-odd
 * preconditioning, clover improvement and its exponentiated form (Sec. 3.1),
 * the spin projection to half-spinors and the bulk / receive-buffer geometry
 * with half-spinor sends (Sec. 2), site-wise linear algebra and reductions
 * (Sec. 3.2) and the conjugate-gradient and BiCGstab inverters (Sec. 3.3).
 * It prints no formula; this library implements the standard definitions:
 *
 *   D psi(x) = A(x) psi(x) - 1/2 sum_mu [ (1 - g_mu) U_R,mu(x) psi(x+mu)
 *                                       + (1 + g_mu) U_R,mu(x-mu)^+ psi(x-mu) ]
 *   A(x)     = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_mu_nu Fhat_mu_nu(x)
 *   Dhat_p   = A_pp - D_pq A_qq^{-1} D_qp          (p = EVEN or ODD, q = 1-p)
 *
 * with chiral Hermitian gammas (g_0 = [[0,-1],[-1,0]], g_k = [[0,-i s_k],
 * [i s_k,0]], g_5 = diag(1,1,-1,-1)), periodic space, antiperiodic time (the
 * sign sits on U_R,0 of the last time slice), parity (t+x+y+z) mod 2.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Return HR_OK (0) or a negative hr_status; nothing aborts or throws.
 * - "device" pointers are CUDA device addresses on the current device; the
 *   caller owns them (e.g. PyTorch tensors) and keeps them alive until the
 *   work queued on the lattice's stream has finished.  The library owns the
 *   represented links, the clover field and its workspaces.
 * - Work is queued on the stream given to hr_set_stream (default: the legacy
 *   default stream) and is asynchronous unless stated otherwise.  Kernel-side
 *   guards latch a device error word, reported (HR_ERR_DEVICE) by the next
 *   synchronising call.
 * - A lattice (or batch) handle is driven by one host thread at a time;
 *   different handles may be driven from different threads (the autotuner's
 *   shared table is locked), except for the calls whose scratch is
 *   process-wide and which say so: hr_bicgstab_solve and hr_norm2_static.
 *   hr_set_allocator is process-wide.
 * - Canonical layouts (what the caller sees), all FP64, complex as (re, im):
 *     site index   ((t*L + z)*L + y)*L + x,  direction 0 = t, 1..3 = x, y, z
 *     links        U[V][4][N][N]       complex, row-major
 *     U_R          UR[V][4][d][d]      complex (imaginary part 0 for adjoint)
 *     spinor       psi[nrhs][V][4][d]  complex (rhs, site, spin, colour)
 *   Internal fields (hr_pack_spinor output, hr_dphi operands) are opaque
 *   byte buffers of hr_field_bytes() bytes, 256-byte aligned.
 */
#ifndef HR_H
#define HR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hr_lattice hr_lattice;

typedef enum { HR_FUND = 0, HR_ADJ = 1, HR_SYM = 2, HR_ASYM = 3 } hr_rep;
/* EVEN/ODD: the Schur complement Dhat on that parity; FULL: D on the whole lattice */
typedef enum { HR_EVEN = 0, HR_ODD = 1, HR_FULL = 2 } hr_parity;
/* HR_FF (no counterpart in the paper, whose outer residuals are double
 * precision, Sec. 3.3): float-float, each real the unevaluated sum hi + lo of two FP32
 * numbers (about 48 significant bits, FP32 exponent range), stored in the FP64
 * layout with each 16-byte chunk (re.hi, re.lo, im.hi, im.lo); the FP64-accurate
 * operator of the mixed solvers' outer residuals, for a part whose FP64 units
 * run at a small fraction of its FP32 rate.  Accepted by hr_field_bytes,
 * hr_pack_spinor / hr_unpack_spinor, hr_dphi (whole lattices: every class
 * without clover, and with clover the d_R <= 8 classes), the shape calls,
 * and hr_cg_params.outer_prec. */
typedef enum { HR_F64 = 0, HR_F32 = 1, HR_F16 = 2, HR_FF = 3 } hr_prec;

typedef enum {
  HR_OK = 0,
  HR_ERR_ARG = -1,           /* invalid argument (null, size, enum, csw mismatch) */
  HR_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  HR_ERR_NOMEM = -3,         /* device allocation failed */
  HR_ERR_STATE = -4,         /* call out of order, e.g. hr_dphi before links */
  HR_ERR_BREAKDOWN = -5,     /* solver breakdown: <p,Ap> <= 0 or non-finite */
  HR_ERR_NOT_CONVERGED = -6, /* solver hit maxit before the tolerance */
  HR_ERR_UNSUPPORTED = -7,   /* combination not built (e.g. clover with d > 8) */
  HR_ERR_DEVICE = -8         /* a kernel-side guard latched an error */
} hr_status;

typedef struct {
  int T, L, N, rep;          /* as created */
  int d;                     /* d_R: N, N^2-1, N(N+1)/2, N(N-1)/2 */
  int is_real;               /* 1 for the adjoint (real links) */
  int64_t volume;            /* V = T L^3 */
  int64_t half_volume;       /* V/2 */
  double flops_hop_site;     /* flops of one hopping term per output site */
  double bytes_hop_site[3];  /* ideal-reuse bytes of one hop per output site, per hr_prec */
} hr_info;

typedef struct {
  double tol;        /* target true relative residual |b - M x| / |b| (FP64) */
  int maxit;         /* cap on inner iterations (all outer steps together) */
  int inner_prec;    /* hr_prec of the inner solver; HR_F64 = plain FP64 CG */
  double inner_tol;  /* relative residual reduction per inner solve (mixed only; 0: 1e-5 for
                        HR_F32, 3e-3 for HR_F16) */
  int nrhs;          /* number of right-hand sides stored back to back */
  int check_every;   /* inner iterations between residual checks on the host */
  int outer_prec;    /* mixed hr_cg_solve / hr_bicgstab_solve / hr_batch_cg_solve:
                        arithmetic of the outer residual, HR_F64 (0) or HR_FF
                        (float-float; time slabs use FP64).  Ignored elsewhere */
} hr_cg_params;

typedef struct {
  int iterations;      /* inner CG iterations, summed over outer steps (max over rhs) */
  int outer_steps;     /* FP64 residual recomputations (1 for plain FP64 CG) */
  double true_residual;/* max over rhs of |b - M x| / |b| at exit (outer arithmetic) */
  double seconds;      /* wall time of the call */
  double hop_launches; /* hopping-kernel launches issued */
} hr_cg_stats;

/* ---- device memory ------------------------------------------------------ */

/* Allocator for the library's large device buffers (represented links in all
 * precisions, the rows layout, clover blocks, the Schur intermediate, solver
 * workspaces, slab face buffers), e.g. PyTorch's caching allocator.  alloc
 * returns device memory of at least `bytes` on the current device (256-byte
 * aligned; NULL on failure -> HR_ERR_NOMEM) and release frees it; each block
 * is released through the function pair it was allocated with, so the
 * allocator may be changed at any time.  NULL, NULL restores cudaMalloc /
 * cudaFree.  Small control words stay on cudaMalloc.  Process-wide.
 * Errors: HR_ERR_ARG (only one of the two given). */
typedef void *(*hr_alloc_fn)(size_t bytes, void *ctx);
typedef void (*hr_free_fn)(void *ptr, size_t bytes, void *ctx);
int hr_set_allocator(hr_alloc_fn alloc, hr_free_fn release, void *ctx);

/* ---- lattice handle --------------------------------------------------- */

/* Create a T x L^3 lattice for SU(N) fermions in representation rep on the
 * current CUDA device.  T, L even and >= 2; 2 <= N <= 12 for FUND (the
 * large-N_c workload of Sec. 3.1.2), 2 <= N <= 6 for ADJ, SYM, ASYM; (N=2,
 * ASYM) is the trivial singlet and is rejected.  Allocates nothing large until links are
 * loaded.  Errors: HR_ERR_ARG.  (Sec. 3.1: any N_c and representation.) */
int hr_lattice_create(int T, int L, int N, int rep, hr_lattice **out);

/* Free the handle and everything the library allocated for it, and drop any
 * cached solver graph captured on it.  Synchronises the device.  No
 * counterpart in the paper (handle management).  Errors: HR_ERR_ARG (NULL). */
int hr_lattice_destroy(hr_lattice *lat);

/* Queue all further work of this lattice on `cuda_stream` (a cudaStream_t,
 * e.g. torch.cuda.current_stream().cuda_stream; NULL = legacy stream).  The
 * caller owns the stream.  No counterpart in the paper (stream plumbing).
 * Errors: HR_ERR_ARG (NULL lattice). */
int hr_set_stream(hr_lattice *lat, void *cuda_stream);

/* Sizes and the per-site work models (written to *info, caller-owned host
 * memory): d_R, real or complex links, V, V/2, flops of one hop per output
 * site and ideal-reuse bytes of one hop per output site per precision.  The
 * paper states that lattice codes are memory-bound and that the Dirac time
 * tracks the bytes moved (Sec. 2.1, Sec. 3.1.1); these are the models the
 * roofline uses.  Errors: HR_ERR_ARG. */
int hr_lattice_info(const hr_lattice *lat, hr_info *info);

/* Bytes of one internal spinor field: parity EVEN/ODD = one parity, FULL =
 * both; `nrhs` fields back to back (written to *bytes, host).  No counterpart
 * in the paper (layout query).  Errors: HR_ERR_ARG. */
int hr_field_bytes(const hr_lattice *lat, int parity, int prec, int nrhs, size_t *bytes);

/* Wait for the lattice's stream; report a latched device error
 * (HR_ERR_DEVICE) or a failed CUDA call (HR_ERR_CUDA).  No counterpart in the
 * paper. */
int hr_synchronize(hr_lattice *lat);

/* ---- gauge field ------------------------------------------------------- */

/* Synthetic links: U = exp(i eps sum_k a_k T_k) per link, generalised
 * Gell-Mann T_k (tr T_a T_b = delta/2), optionally reunitarised.
 *   a_dev : device, FP64 a[V][4][N*N-1]          (read)
 *   U_dev : device, FP64 complex U[V][4][N][N]   (written)
 * The exponential uses scaling and squaring of its Taylor series in FP64.
 * (The paper generates links with its HMC, Sec. 3.4; this is the synthetic
 * stand-in used for all benchmarks and tests.) */
int hr_links_from_algebra(hr_lattice *lat, double *U_dev, const double *a_dev, double eps,
                          int reunitarise);

/* Load fundamental links and build the represented gauge field U_R
 * (Sec. 3.1.2) in FP64, FP32 and FP16, with the antiperiodic-time sign.
 *   U_dev      : device, FP64 complex U[V][4][N][N] (read only)
 *   reunitarise: 1 = project each link onto SU(N) first (row Gram-Schmidt,
 *                then the last row times conj(det))
 *   csw        : clover coefficient; != 0 also builds the clover term
 *                c_sw (i/4) sigma.Fhat from U_R (Sec. 3.1, clover) for
 *                d <= 8, else HR_ERR_UNSUPPORTED
 * Synchronous with respect to the lattice's stream. */
int hr_represent_links(hr_lattice *lat, const double *U_dev, int reunitarise, double csw);

/* Export U_R (with the boundary sign) in canonical FP64 complex layout
 * UR[V][4][d][d] to device memory. */
int hr_export_represented_links(hr_lattice *lat, double *UR_dev);

/* Export the clover matrix A(x) for bare mass m0 as its two chiral blocks,
 * canonical FP64 complex A[V][2][2d][2d] (block 0 acts on spins 0,1, block 1
 * on spins 2,3; index spin_in_block*d + colour).  inverse = 1 exports
 * A(x)^{-1} instead.  Needs csw != 0 at hr_represent_links. */
int hr_export_clover(hr_lattice *lat, double *A_dev, double m0, int inverse);

/* Choose the form of the clover diagonal (Sec. 3.1, which lists both the
 * Sheikholeslami-Wohlert term and its exponentiated form of Francis,
 * Fritzsch, Luscher and Rago).  With C(x) = c_sw (i/4) sigma.Fhat(x):
 *   on = 0 (default): A(x) = (4 + m0) + C(x)
 *   on = 1          : A(x) = (4 + m0) exp(C(x) / (4 + m0))
 * The exponential is taken in FP64 per chiral block (scaling and squaring of
 * a Taylor series); A^{-1} follows by Gauss-Jordan as for the plain term.
 * Affects every later hr_dphi / solver / export call on this lattice.
 * Errors: HR_ERR_ARG (on not 0 or 1; at use, 4 + m0 == 0 with on = 1). */
int hr_set_clover_exponential(hr_lattice *lat, int on);

/* ---- spinor fields ------------------------------------------------------ */

/* Canonical FP64 spinors psi[nrhs][V][4][d] -> internal field of the given
 * parity and precision (device, caller-owned, hr_field_bytes() bytes).  The
 * internal layout is this library's own blocked structure of arrays; the
 * paper's GPU fields are likewise strided, structure-of-arrays blocks
 * (Sec. 2.1), in single or double precision (Sec. 3.2); FP16 with a per-site
 * scale has no counterpart in the paper.  Errors: HR_ERR_ARG (NULL, bad enum,
 * nrhs < 1, pageable host memory).  Only sites of that parity are read (both
 * for FULL).  `canonical` may be device memory or page-locked host memory
 * (cudaHostAlloc / cudaHostRegister / pinned torch tensors): the kernel then
 * reads the host buffer directly through its mapped address, so only that
 * parity's sites cross the host link; pageable host memory -> HR_ERR_ARG.  FP16 code: per site, scale = max |fp32(v)| over its
 * 8d reals, stored values fp16_rn(fp32(v) / scale) with IEEE division. */
int hr_pack_spinor(hr_lattice *lat, void *internal, const double *canonical, int parity,
                   int prec, int nrhs);

/* Internal field -> canonical FP64 spinors (device or page-locked host
 * memory, written directly as for hr_pack_spinor; layouts of Sec. 2.1 as
 * there).  Sites of the other parity are left untouched (set to zero first
 * if that matters).  Errors: HR_ERR_ARG. */
int hr_unpack_spinor(hr_lattice *lat, double *canonical, const void *internal, int parity,
                     int prec, int nrhs);

/* ---- operator ------------------------------------------------------------ */

/* The Wilson(-clover) Dirac operator of Sec. 3.1 (even-odd preconditioned,
 * clover term as set at hr_represent_links), applied with the half-spinor
 * projection of Sec. 2.2 (each neighbour is projected to two spin rows before
 * the link product and rebuilt after it):
 * out = Dhat_p in (parity EVEN/ODD) or D in (FULL), or the adjoint with
 * dagger = 1 (= g5 D g5), on `nrhs` internal fields of precision prec.
 *   out, in : device internal fields (nrhs back to back; in read, out written)
 * FP64 fields compute in FP64; FP32 and FP16 fields accumulate in FP32.
 * With FP16 fields the projected half-spinor may be rounded to FP16 before
 * the link product (FP16 x FP16 -> FP32 multiply-add); the relative error
 * against FP64 stays about 3e-4 of the field norm.  csw must equal the value given to hr_represent_links.  `in` and `out`
 * must not overlap.  Two hopping launches (the second, for the one-site-per-thread
 * kernel, a programmatic dependent launch that starts while the first one
 * finishes), no host synchronisation. */
int hr_dphi(hr_lattice *lat, void *out, const void *in, int parity, double m0, double csw,
            int prec, int nrhs, int dagger);

/* ---- linear algebra (Sec. 3.2) ------------------------------------------ */

/* Global sums |x_r|^2 over internal fields (the reductions of Sec. 3.2, which
 * the paper runs as a site kernel plus a library reduction; here one kernel
 * with a deterministic last-block sum), FP64 accumulation, fixed order.
 *   x        : device internal field(s), nrhs back to back (read)
 *   out_host : host double[nrhs] (written)
 * Synchronises the stream.  Errors: HR_ERR_ARG, HR_ERR_CUDA. */
int hr_norm2(hr_lattice *lat, const void *x, int parity, int prec, int nrhs,
             double *out_host);

/* y_r = a_r x_r + b_r y_r for every rhs r (the site-wise linear algebra of
 * Sec. 3.2, one fused launch), on internal fields of this lattice's geometry:
 *   x, y : device internal fields of the same parity and precision, nrhs back
 *          to back (x read, y read and written; x == y allowed)
 *   a, b : host double[nrhs] (copied before the call returns)
 * FP64 fields compute in FP64, FP32 / FP16 fields in FP32 (FP16 results
 * re-encoded with their per-site scale).  Asynchronous on the lattice's stream.
 * The building block of solvers driven from outside the library, such as the
 * conjugate gradient over time slabs on several ranks.
 * Errors: HR_ERR_ARG (NULL, bad enum, nrhs outside 1..64). */
int hr_axpby(hr_lattice *lat, const void *x, void *y, const double *a, const double *b, int parity, int prec,
             int nrhs);

/* Variant of hr_norm2 that allocates nothing (the paper has no counterpart).
 * For callers that cannot call cudaMalloc/cudaFree: code whose device memory
 * all comes from a framework's pool allocator, code under a fixed memory
 * budget, real-time callers that forbid allocation after start-up.  Its
 * reduction scratch is a file-scope device array of about
 * 312 KB (partial sums and arrival counters for up to 16 right-hand sides),
 * present on every GPU that loads the library until the process exits.
 *   x           : device, internal field(s) as for hr_norm2 (read)
 *   half_volume : V/2 of the lattice; d: d_R; parity, prec, nrhs as for hr_norm2
 *   out_dev     : device, double[nrhs], receives |x_r|^2 (written)
 *   stream      : cudaStream_t the work is queued on (asynchronous; no sync)
 * The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress with that device current); make that first call
 * before any stream capture.  Every call shares the one array, so calls that
 * overlap on the GPU (other streams, other threads) race: serialise them.
 * Errors: HR_ERR_ARG for nrhs > 16 or a bad argument, HR_ERR_CUDA. */
int hr_norm2_static(const void *x, int64_t half_volume, int d, int parity, int prec, int nrhs,
                    double *out_dev, void *stream);

/* ---- solver (Sec. 3.3) ----------------------------------------------------- */

/* Solve (Dhat_p^+ Dhat_p) x = b (parity EVEN/ODD) or (D^+ D) x = b (FULL)
 * for nrhs FP64 internal fields, to a true FP64 relative residual
 * params->tol per rhs.  inner_prec = HR_F64: plain CG.  HR_F32 / HR_F16:
 * the inner CG runs in that precision (FP32 accumulation) and an FP64
 * defect-correction loop recomputes b - M x in FP64 until params->tol
 * (params->outer_prec = HR_FF: in float-float, the iterate kept as a
 * float-float field and rounded to FP64 into x at exit).
 * x is overwritten (initial guess ignored: x0 = 0).  Synchronous.
 * Errors: HR_ERR_NOT_CONVERGED (stats still filled), HR_ERR_BREAKDOWN. */
int hr_cg_solve(hr_lattice *lat, void *x, const void *b, int parity, double m0, double csw,
                const hr_cg_params *params, hr_cg_stats *stats);

/* ---- many small lattices in one solve ----------------------------------- */

typedef struct hr_batch hr_batch;

/* Group n lattices (each created, links loaded, csw = 0; any mix of T, L, N,
 * representation) for batched operator applications and solves.  The
 * lattices must outlive the batch.  Lattices of equal (d_R, real links) form a
 * class; each class runs one persistent multi-lattice launch per hopping
 * stage, so a batched Dhat costs 2 x (number of classes) launches however
 * many lattices there are (kernel-call overhead at small volumes, Sec. 3.1.1).
 * Errors: HR_ERR_STATE (links missing), HR_ERR_UNSUPPORTED (clover). */
int hr_batch_create(int n, hr_lattice *const *lats, hr_batch **out);
/* Free the batch (not its lattices).  Synchronises.  No counterpart in the
 * paper (handle management).  Errors: HR_ERR_ARG. */
int hr_batch_destroy(hr_batch *batch);
/* Stream the batch's work is ordered after (default: the first lattice's);
 * a cudaStream_t owned by the caller.  No counterpart in the paper. */
int hr_batch_set_stream(hr_batch *batch, void *cuda_stream);

/* Pin the hopping launch shape of the class (d_R = d, real links is_real) at
 * precision prec instead of timing its candidates.  `shape` is one of the
 * codes hr_hop_shape_candidates reports for such a lattice (nrhs = 1, no
 * clover).  Errors: HR_ERR_ARG (no such class or shape). */
int hr_batch_set_shape(hr_batch *batch, int d, int is_real, int prec, int shape);

/* The even-odd Wilson operator of Sec. 3.1 on many small lattices at once
 * (kernel-call overhead dominates small volumes, Sec. 3.1.1, Sec. 3.2):
 * out[i] = Dhat_p in[i] (or its adjoint) on lattice i, parity EVEN or ODD,
 * bare mass m0[i] (host array); internal single-parity fields of precision
 * prec (HR_FF included), one rhs each.  The first call per precision times
 * each class's launch shapes (outside stream capture). */
int hr_batch_dphi(hr_batch *batch, void *const *out, const void *const *in, int parity, const double *m0,
                  int prec, int dagger);

/* CG (Sec. 3.3) on many small lattices at once.
 * Solve (Dhat_p^+ Dhat_p) x[i] = b[i] on every lattice to a true FP64
 * relative residual params->tol per lattice (x, b: FP64 internal fields;
 * x overwritten).  params->inner_prec HR_F32 or HR_F16: the inner CG of all
 * lattices runs in lock step as one CUDA graph per chunk of
 * params->check_every iterations; converged lattices are frozen on the device
 * and skipped; FP64 defect correction per lattice between chunks
 * (params->outer_prec = HR_FF: the outer residuals in float-float, batched
 * over the lattices as the FP64 ones are).
 * stats[i] (n entries) receives each lattice's iterations and residual.
 * Synchronous.  Errors as hr_cg_solve. */
int hr_batch_cg_solve(hr_batch *batch, void *const *x, const void *const *b, int parity, const double *m0,
                      const hr_cg_params *params, hr_cg_stats *stats);

/* Launch-shape autotuning (no counterpart in the paper, which fixes its kernel
 * shapes at compile time, Sec. 2 and Sec. 3.1.2).
 * The hopping-kernel launch shape the autotuner chose for this lattice at
 * (prec, nrhs, clover): rows * 100000000 + mrhs * 1000000 + regs * 100000 +
 * split_g * 1000 + threads per block.  mrhs = S > 0: the multi-right-hand-
 * side kernel with S sites per block (links staged once per site for all
 * right-hand sides), mrhs = 66: the tensor-core multi-right-hand-side kernel
 * (16 sites per block, link products as MMA tiles); rows = R > 0: the rows kernel for large d_R (R output
 * colour rows per warp, 32 sites per block on the lanes); otherwise
 * split_g = 0: one site per thread with register budget regs = 0 compiler's
 * choice, 1 up to ~170, 2 at most ~85, 3 at most 128 registers; split_g = G > 0: G threads
 * per site.  -1 if not tuned yet.  The
 * first hr_dphi / hr_cg_solve call for a new shape key times the candidate
 * shapes on the caller's stream (make it outside any stream capture). */
int hr_tuned_shape(const hr_lattice *lat, int prec, int nrhs, int clover);

/* The candidate shapes for this lattice at (prec, nrhs, clover), encoded as
 * above, into out[0..max); returns how many exist (may exceed max) or an error. */
int hr_hop_shape_candidates(const hr_lattice *lat, int prec, int nrhs, int clover, int *out, int max);

/* Pin the shape for (prec, nrhs, clover) instead of timing candidates
 * (reproducible runs, tests of every shape).  HR_ERR_ARG unless `shape` is
 * one of the candidates. */
int hr_set_tuned_shape(const hr_lattice *lat, int prec, int nrhs, int clover, int shape);

/* Solve Dhat_p x = b (parity EVEN/ODD) or D x = b (FULL) directly with
 * BiCGstab (Sec. 3.3; van der Vorst's stabilised bi-conjugate gradient), for
 * nrhs FP64 internal fields, to a true FP64 relative residual
 * |b - A x| / |b| <= params->tol per rhs.  inner_prec HR_F64: plain FP64
 * BiCGstab; HR_F32: FP32 inner BiCGstab inside FP64 defect correction
 * (params->outer_prec = HR_FF: outer residuals in float-float, as for
 * hr_cg_solve).  x overwritten (x0 = 0).  Synchronous.  The solver's workspace is shared
 * by all lattices of the process: do not call it concurrently from several
 * threads.  Errors: HR_ERR_ARG (HR_F16 inner not offered),
 * HR_ERR_NOT_CONVERGED, HR_ERR_BREAKDOWN (rho or <t,t> vanished). */
int hr_bicgstab_solve(hr_lattice *lat, void *x, const void *b, int parity, double m0, double csw,
                      const hr_cg_params *params, hr_cg_stats *stats);

/* ---- time-slab domain decomposition (Sec. 2, halo-ready geometry) -------- */

/* A sub-domain: the time slab [t0, t0 + T_loc) of a T_global x L^3 lattice,
 * with the same N and rep.  T_loc >= 2, t0 and T_global even, t0 + T_loc <=
 * T_global.  Load its links with hr_represent_links from the canonical FP64
 * links of its own sites U[V_loc][4][N][N] (lexicographic in local
 * coordinates, local t = global t - t0); the antiperiodic sign is applied at
 * global t = T_global - 1.  Only csw = 0 (the clover leaves would need a link
 * halo: HR_ERR_UNSUPPORTED); hr_dphi and the solvers treat the slab as
 * periodic on its own, the calls below couple the slabs.  Errors: HR_ERR_ARG. */
int hr_lattice_create_domain(int T_loc, int L, int N, int rep, int t0, int T_global, hr_lattice **out);

/* Bytes of one face buffer for nrhs right-hand sides: [rhs][2][d][L^3/2]
 * complex, FP64 for prec HR_F64 and FP32 otherwise. */
int hr_domain_halo_bytes(const hr_lattice *lat, int prec, int nrhs, size_t *bytes);

/* One of the two hops of Dhat_p on a slab, first half (Sec. 2: send-buffer
 * synchronisation with half-spinors, masked directions):
 *   stage 0: out = tmp_q = -1/(2(4+m0)) H in_hop, out_parity = q = 1-p;
 *   stage 1: out = out_p = (4+m0) self + 1/2 H in_hop, out_parity = p,
 *            in_hop = tmp_q, self = the Dhat input (parity p).
 * Writes the send buffers from in_hop's boundary sites -- send_down: the
 * projected half-spinors of the bottom face (local t = 0) for the slab below;
 * send_up: U_0^+ times the projected half-spinors of the top face for the
 * slab above -- and runs the bulk hop with the two t hops that cross a face
 * masked.  Fields: internal, precision prec, nrhs consecutive rhs; buffers:
 * device memory of hr_domain_halo_bytes, caller-owned.  Asynchronous on the
 * lattice's stream.  Errors: HR_ERR_ARG, HR_ERR_STATE (not a slab, links
 * missing), HR_ERR_UNSUPPORTED (clover). */
int hr_domain_hop_begin(hr_lattice *lat, void *out, const void *in_hop, const void *self, int out_parity,
                        double m0, int prec, int nrhs, int dagger, int stage, void *send_up, void *send_down);

/* Second half, after the exchange: recv_up holds the send_down buffer of the
 * slab above, recv_down the send_up buffer of the slab below (periodically:
 * with one slab, its own).  Adds the masked face terms to out. */
int hr_domain_hop_end(hr_lattice *lat, void *out, int out_parity, double m0, int prec, int nrhs, int dagger,
                      int stage, const void *recv_up, const void *recv_down);

/* All n slabs of one lattice in this process (lats in time order, covering
 * [0, T_global)): out[k] = Dhat_p in[k] on slab k, the exchange done as
 * device-to-device copies between the slabs' own buffers, everything on the
 * first slab's stream.  Errors as above. */
int hr_domains_dphi(int n, hr_lattice *const *lats, void *const *out, const void *const *in, int parity, double m0,
                    int prec, int nrhs, int dagger);

/* Human-readable text of an hr_status (no counterpart in the paper; the
 * returned string is library-owned, never NULL).  For HR_ERR_CUDA it names the failing
 * CUDA call last seen by the calling host thread; the text stays valid until
 * that thread's next CUDA error. */
const char *hr_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* HR_H */
