// Internal declarations of libhr: the lattice handle, field layouts, small
// complex helpers and the kernel launchers shared between translation units.
//
// Internal layouts (all per parity, all "structure of arrays" over the V/2
// sites of that parity, checkerboard index i = ((t*L + z)*L + y)*(L/2) + x/2):
//
//   spinor field : nchunk 16-byte chunks per site, chunk k of site i at byte
//                  (k*Vh + i)*16.  FP64: chunk = one complex (double2),
//                  k = 4*colour + spin.  FP32: chunk = two complex (float4),
//                  k = 2*colour + spin/2.  FP16: chunk = four complex (4 x
//                  half2), k = colour, followed by one float scale per site.
//   links        : [parity][mu][chunk][Vh] of "2-real" chunks (double2,
//                  float2, half2).  Complex reps: chunk k = entry k = a*d + c
//                  of the d x d matrix.  Real reps (adjoint): chunk k holds
//                  entries 2k, 2k+1 (the last one padded with 0 for odd d*d).
//                  Slot [p][mu] holds the forward link U_R,mu(x) of the sites
//                  x of parity p.
//   clover       : [parity][chunk][Vh] double2/float2; per site two
//                  Hermitian 2d x 2d blocks, each stored as 2d diagonal reals
//                  (d chunks) then the strictly lower triangle row by row.
//
// A warp therefore reads 32 consecutive 8- or 16-byte chunks per access, and
// neighbour sites along t, z, y are fixed index offsets (x changes xh by 0/1).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/hr.h"

#define HR_MAX_D 35

struct hr_cg_work;

struct hr_lattice {
  int T, L, N, rep, d, is_real;
  int64_t V, Vh;
  cudaStream_t stream;
  int device;
  int nch_link;          // 2-real chunks per link
  void *links[4];        // per hr_prec (HR_FF: made from the FP64 links on first use)
  int ff_links_ok;       // links[HR_FF] matches links[HR_F64]
  int have_links;
  void *rlinks[4];       // per hr_prec: rows-kernel link layout (see hr_rows_nch), or null
  int dom;               // 1: a time slab [t0, t0 + T) of a T_global lattice (faces via halo buffers)
  int t0, Tg;            // global time origin and extent (0 and T for a whole lattice)
  void *halo[4];         // single-process exchange buffers: send_up, send_down, recv_up, recv_down
  size_t halo_bytes;
  double csw;            // clover coefficient given at represent time
  void *clover_term;     // FP64 packed blocks of csw (i/4) sigma.F (no mass term)
  double clover_m0;      // m0 of the cached A and A^{-1} below
  int clover_cached;
  int clover_exp;         // 1: A = (4+m0) exp(term / (4+m0)) (exponentiated clover)
  void *clover_A[3];     // FP64, FP32, float-float packed A = (4+m0) + term
  void *clover_Ainv[3];  // FP64, FP32, float-float packed A^{-1}
  int clover_ff_ok;      // clover_A[2], clover_Ainv[2] match the FP64 blocks
  void *tmp;             // Schur intermediate spinor (other parity)
  size_t tmp_bytes;
  int *dev_err;          // latched device error word
  double *red_partials;  // reduction scratch: per-block partial sums
  unsigned *red_count;   // reduction scratch: arrival counter
  double *red_out;       // reduction result (device)
  double *red_out_host;  // pinned host mirror
  hr_cg_work *cg;        // solver workspace (lazily allocated)
  double hop_launches;   // statistics
};

// ---------------------------------------------------------------- errors ----
#define HR_TRY(expr)                 \
  do {                               \
    int hr_rc_ = (expr);             \
    if (hr_rc_ != HR_OK) return hr_rc_; \
  } while (0)

#define HR_CUDA(call)                            \
  do {                                           \
    cudaError_t hr_e_ = (call);                  \
    if (hr_e_ != cudaSuccess) {                  \
      hr_note_cuda_error(hr_e_, #call, __FILE__, __LINE__); \
      return hr_e_ == cudaErrorMemoryAllocation ? HR_ERR_NOMEM : HR_ERR_CUDA; \
    }                                            \
  } while (0)

void hr_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// A CUDA event owned by the enclosing scope: every return path (including the
// early returns of HR_TRY / HR_CUDA) releases it.
struct HrEvent {
  cudaEvent_t e = nullptr;
  HrEvent() = default;
  HrEvent(const HrEvent &) = delete;
  HrEvent &operator=(const HrEvent &) = delete;
  ~HrEvent() {
    if (e) cudaEventDestroy(e);
  }
};
// library-owned large buffers: through the allocator of hr_set_allocator, else cudaMalloc
int hr_dev_alloc(void **p, size_t bytes);
void hr_dev_free(void *p);
int hr_check_launch(const char *what);

// ------------------------------------------------------------- geometry ----
struct HrGeom {
  int T, L, Lh;
  int64_t Vh;
};

static inline HrGeom hr_geom(const hr_lattice *lat) {
  HrGeom g;
  g.T = lat->T;
  g.L = lat->L;
  g.Lh = lat->L / 2;
  g.Vh = lat->Vh;
  return g;
}

// chunks and bytes of one single-parity, single-rhs spinor field
static inline int hr_spinor_chunks(int d, int prec) {
  return (prec == HR_F64 || prec == HR_FF) ? 4 * d : (prec == HR_F32 ? 2 * d : d);
}
static inline size_t hr_spinor_field_bytes(int64_t Vh, int d, int prec) {
  size_t b = (size_t)hr_spinor_chunks(d, prec) * 16u * (size_t)Vh;
  if (prec == HR_F16) b += 4u * (size_t)Vh;
  return (b + 255u) & ~(size_t)255u;
}
static inline size_t hr_real_size(int prec) {
  return (prec == HR_F64 || prec == HR_FF) ? 8 : (prec == HR_F32 ? 4 : 2);
}

// ------------------------------------------------------------ launchers ----
// Hopping kernel epilogue modes.
enum HopMode {
  HOP_SCALED = 0,   // out = Ainv (coef * H)      (clover) | coef * H        (no clover)
  HOP_SELF = 1      // out = A self + coef * H     (clover) | diag*self + coef*H (no clover)
};

struct HopArgs {
  void *out;
  const void *in;         // field hopped from (parity 1-p)
  const void *self;       // field of parity p for HOP_SELF
  const void *links;      // internal links of the precision
  const void *rlinks;     // rows-kernel layout of the same links (null if not built)
  const void *clover;     // packed A (HOP_SELF) or A^{-1} (HOP_SCALED); null = no clover
  int out_parity;
  int dagger;
  int mode;
  double coef;            // multiplies H
  double diag;            // multiplies self when no clover
  size_t field_stride;    // bytes between rhs fields (in, out, self)
  int nrhs;
  int tmask;              // 1: skip the t hops that cross the slab faces (sub-domain bulk pass)
  const double *skip_rr;  // with skip_stop: a rhs whose skip_rr <= skip_stop is done, its blocks
  const double *skip_stop;  // return at once (CG chunks past convergence); null = never skip
  int pdl;                  // 1: programmatic dependent launch after the previous hop (site kernel)
};

// One launch shape of the hopping stencil: split_g = 0 is the one-site-per-
// thread kernel with `bs` threads per block and register-budget variant
// `regs` (0: compiler's choice for 256 threads, 1: up to ~170 registers,
// 2: at most ~85 registers, 3: at most 128 registers, 4: the budget of 1
// with a one-wave grid whose blocks loop over the work items, FP32 only);
// split_g = G > 0 is the colour-split kernel with
// G threads per site (128 threads per block).
// mrhs = S > 0 selects the multi-right-hand-side kernel (S sites per block,
// links staged once per site for all right-hand sides of the block);
// mrhs = HR_TC_MRHS + 16 the tensor-core multi-right-hand-side kernel
// (hop_tc.cuh: 16 sites per block, the link products of up to 12 rhs as MMA
// tiles; FP32 and FP16, complex d_R = 3 ... 6).
// rows = R > 0 selects the rows kernel: R output colour rows per warp,
// ceil(d/R) warps per block, 32 sites per block on the lanes.
struct HopShape {
  int split_g;
  int bs;
  int regs;
  int mrhs;
  int rows;
};
// Integer form of a shape (hr_tuned_shape and friends):
// rows * 1e8 + mrhs * 1e6 + regs * 1e5 + split_g * 1e3 + bs.
static inline int hr_shape_code(const HopShape &s) {
  return s.rows * 100000000 + s.mrhs * 1000000 + s.regs * 100000 + s.split_g * 1000 + s.bs;
}
// sites covered by one block (one work-list tile) of a shape
static inline int hr_shape_tile(const HopShape &s) {
  return s.rows ? 32 : (s.split_g ? 128 / s.split_g : s.bs);
}
#define HR_MAX_SHAPES 24
#define HR_TC_MRHS 50

// largest N of SU(N) (fundamental representation; the 2-index ones stop at 6)
#define HR_MAX_NC 12

// Rows-kernel link layout: for output parity p, direction n = 2 mu + back,
// and output site i, the matrix V_n(x) the hop applies -- U_R,mu(x) (forward)
// or U_R,mu(x - mu)^+ (backward) -- stored row-major at the output site, so
// all 8 matrices of a tile of consecutive output sites are read at
// consecutive indices: [p][n][chunk][Vh].  Complex links: chunk a*d + c holds
// V[a][c].  Real links: rows padded to an even length dp, chunk (a*dp + c)/2
// holds V[a][c], V[a][c+1] for even c (the pad element is 0).
__host__ __device__ constexpr int hr_rows_dp(int d, int is_real) { return is_real ? d + (d & 1) : d; }
__host__ __device__ constexpr int hr_rows_nch(int d, int is_real) {
  return is_real ? d * hr_rows_dp(d, is_real) / 2 : d * d;
}
// The rows layout holds 16 matrices of hr_rows_nch chunk rows, then
// HR_ROWS_SLACK zeroed chunk rows that the rows kernel's last column batch may
// read past the last matrix.
#define HR_ROWS_SLACK 16

// The (d_R, rows per warp) pairs built for the rows kernel; one X(D, REAL, R)
// line each.  Shared by the candidate list and every dispatch.
#define HR_ROWS_SHAPES(X)                                                                               \
  X(6, false, 2) X(6, false, 3) X(7, false, 2) X(7, false, 4) X(8, false, 2) X(8, false, 4)             \
  X(8, true, 2) X(8, true, 4) X(9, false, 2) X(9, false, 3) X(10, false, 2) X(10, false, 5)             \
  X(11, false, 2) X(11, false, 3) X(12, false, 2) X(12, false, 3) X(15, false, 2) X(15, false, 3)       \
  X(15, true, 2) X(15, true, 3) X(21, false, 2) X(21, false, 3) X(24, true, 2) X(24, true, 3)           \
  X(35, true, 2) X(35, true, 4)


// The (d_R, threads per site G) pairs built for the colour-split kernel.
#define HR_SPLIT_SHAPES(X)                                                                              \
  X(8, true, 2) X(15, true, 4) X(24, true, 8) X(35, true, 16) X(6, false, 2) X(10, false, 2)            \
  X(12, false, 4) X(15, false, 4) X(21, false, 4)

// whether the rows kernel is built for (d, real)
static inline bool hr_has_rows_shapes(int d, int is_real) {
#define HR_ROWS_HAS(DD, RE, RR) \
  if (d == DD && (is_real != 0) == RE) return true;
  HR_ROWS_SHAPES(HR_ROWS_HAS)
#undef HR_ROWS_HAS
  return false;
}

// Candidate shapes for (d, real, precision, several rhs); clover restricts to
// split_g = 0.
int hr_hop_shapes(int d, int is_real, int prec, int clover, int multi_rhs, HopShape *out);
int hr_launch_hop(const hr_lattice *lat, int prec, const HopArgs &a, cudaStream_t s);
int hr_launch_hop_f64(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh);
int hr_launch_hop_f32(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh);
int hr_launch_hop_f16(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh);
int hr_launch_hop_ff(const hr_lattice *lat, const HopArgs &a, cudaStream_t s, HopShape sh);
// hop_ff.cu: float-float copies of FP64 arrays, and of the links (and of the
// clover blocks at m0) of a lattice, made on stream st when missing or stale
int hr_f64_to_ff(void *out, const void *in, size_t nreal, cudaStream_t s);
int hr_ff_prepare(hr_lattice *lat, int clover, double m0, cudaStream_t st);
// *use = 1 when a mixed solve's outer residuals on lat can run in float-float:
// a kernel exists for the class (whole lattices only) and the float-float
// links and clover blocks are in place on st (made here if needed); 0 when
// not, including when the device has no room for them (FP64 is used then)
int hr_ff_outer_usable(hr_lattice *lat, int clover, double m0, int nrhs, cudaStream_t st, int *use);
// tensor-core multi-rhs kernel (complex d_R = 3 ... 6), FP32 (FP16 pairs) / FP16
int hr_launch_hop_tc_f32(const hr_lattice *lat, const HopArgs &a, cudaStream_t s);
int hr_launch_hop_tc_f16(const hr_lattice *lat, const HopArgs &a, cudaStream_t s);
static inline bool hr_has_tc_mrhs(int d, int is_real, int prec) {
  return !is_real && d >= 3 && d <= 6 && prec != HR_F64;
}

// multi-lattice persistent hop (descs: one HopK per lattice; items: (lattice, tile))
struct HopK;
int hr_launch_hop_multi_f64(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                            const int *frozen, cudaStream_t s);
int hr_launch_hop_multi_f32(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                            const int *frozen, cudaStream_t s);
int hr_launch_hop_multi_f16(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                            const int *frozen, cudaStream_t s);
int hr_launch_hop_multi_ff(int d, int is_real, HopShape sh, const HopK *descs, const int2 *items, int nitems,
                           const int *frozen, cudaStream_t s);

// cg.cu: per-lattice solver workspace (5 fields per precision: r, p, Ap, t, x)
int hr_cg_workspace(hr_lattice *lat, int prec, size_t bytes);
void *hr_cg_field(hr_lattice *lat, int prec, int which);

// dirac.cu
int hr_dphi_impl(hr_lattice *lat, void *out, const void *in, int parity, double m0, double csw,
                 int prec, int nrhs, int dagger, cudaStream_t s);
// the same, with the converged-rhs skip of HopArgs (rr, stop: device arrays per rhs)
int hr_dphi_impl_skip(hr_lattice *lat, void *out, const void *in, int parity, double m0, double csw, int prec,
                      int nrhs, int dagger, cudaStream_t st, const double *rr, const double *stop);
int hr_ensure_tmp(hr_lattice *lat, size_t bytes);
int hr_clover_prepare(hr_lattice *lat, double m0);


