// hr_norm2_static: the field-norm reduction with its scratch memory in a
// fixed, file-scope device array instead of memory the library allocates.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree -- code whose
// device memory all comes from a framework's pool allocator (a raw cudaMalloc
// would bypass the pool and can fail or fragment memory the pool believes it
// owns), code running under a fixed memory budget decided up front, and
// real-time or embedded callers that forbid allocation after start-up.
//
// The reduction kernel is the one hr_norm2 uses (blas.cu); only where its
// per-block partial sums and arrival counters live differs.  That scratch is
// the array below: HR_STATIC_MAX_RHS x 2 x HR_RED_MAXBLK doubles for the
// partials plus HR_STATIC_MAX_RHS arrival counters, about 312 KB, held on
// every GPU that loads the library until the process exits.
#include <string.h>

#include "blas.cuh"
#include "hr_internal.h"

#define HR_STATIC_MAX_RHS 16
#define HR_STATIC_PARTIALS ((size_t)HR_STATIC_MAX_RHS * 2 * HR_RED_MAXBLK)
#define HR_STATIC_BYTES (HR_STATIC_PARTIALS * sizeof(double) + 2 * HR_STATIC_MAX_RHS * sizeof(unsigned))

static __device__ __align__(256) unsigned char g_norm2_scratch[HR_STATIC_BYTES];

// Device address of g_norm2_scratch per device, looked up once per device.
// (In host code the symbol itself is only a host-side stand-in; a kernel
// handed that stand-in would read the wrong memory or fault.)
#define HR_STATIC_MAX_DEVICES 64
static void *g_scratch_addr[HR_STATIC_MAX_DEVICES];

static int static_scratch(void **out) {
  int dev = 0;
  HR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= HR_STATIC_MAX_DEVICES) return HR_ERR_UNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    HR_CUDA(cudaGetSymbolAddress(&p, g_norm2_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HR_OK;
}

extern "C" int hr_norm2_static(const void *x, int64_t half_volume, int d, int parity, int prec, int nrhs,
                               double *out_dev, void *stream) {
  if (!x || !out_dev || half_volume < 1 || d < 1 || d > HR_MAX_D || nrhs < 1 || prec < HR_F64 || prec > HR_F16 ||
      parity < HR_EVEN || parity > HR_FULL)
    return HR_ERR_ARG;
  if (nrhs > HR_STATIC_MAX_RHS) return HR_ERR_ARG;
  void *base = nullptr;
  HR_TRY(static_scratch(&base));
  cudaStream_t s = (cudaStream_t)stream;
  double *partials = reinterpret_cast<double *>(base);
  unsigned *count = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(base) + HR_STATIC_PARTIALS * sizeof(double));
  int *err = reinterpret_cast<int *>(count + HR_STATIC_MAX_RHS);
  // the arrival counters must start at zero (a call that never finished could
  // have left them set)
  HR_CUDA(cudaMemsetAsync(count, 0, 2 * HR_STATIC_MAX_RHS * sizeof(unsigned), s));
  FieldDesc f;
  f.Vh = half_volume;
  f.d = d;
  f.fb = hr_spinor_field_bytes(half_volume, d, prec);
  f.nsub = parity == HR_FULL ? 2 : 1;
  RedArgs red;
  memset(&red, 0, sizeof(red));
  red.partials = partials;
  red.count = count;
  red.out = out_dev;
  red.err = err;
  return hr_blas_norm2(f, prec, x, nrhs, red, RED_PLAIN, s);
}
