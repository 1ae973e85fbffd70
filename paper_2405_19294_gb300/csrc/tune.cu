// Autotuner for the hopping-kernel launch shape.
//
// The best shape depends on d_R, real/complex links, precision and lattice
// size: the one-site-per-thread kernel with 32..256 threads per block
// (register-limited occupancy changes with the block size) or the
// colour-split kernel with G threads per site.  The first launch with a new
// key (precision, d_R, real, clover, multi-rhs, slab, log2 of the volume)
// times every candidate shape with CUDA events on the caller's stream (two
// sweeps of one warm-up and 4 (16 on small lattices) timed launches each,
// keeping each shape's faster sweep, on the caller's own buffers -- the kernel is a pure function
// of its inputs, so repeating it is harmless) and keeps the fastest.  While the stream is being captured into a CUDA graph no timing is
// possible; the cached choice, else the first candidate, is used.  Setting
// HR_TUNE=0 in the environment disables tuning (first candidate always).
#include <map>
#include <mutex>
#include <stdlib.h>
#include <string.h>

#include "hr_internal.h"

int hr_hop_shapes(int d, int is_real, int prec, int clover, int multi_rhs, HopShape *out) {
  int n = 0;
  const bool site = is_real ? (d == 3 || d == 8) : (d >= 2 && d <= 8);
  const bool site_mrhs = is_real ? (d == 3 || d == 8) : (d >= 2 && d <= 6);
  if (prec == HR_FF) {
    // float-float: its site kernel (hop_ff.cuh), compiler's register choice
    // or (d_R <= 3, where it does not spill) the high budget, and the rows
    // kernel (no clover)
    if (site) {
      // complex d_R >= 5 keeps its accumulator in shared memory (hop_ff.cuh):
      // blocks of at most 64 threads keep that under 48 KB
      const int bss[4] = {64, 128, 32, 256};
      const bool small_blocks = !is_real && d >= 5;
      for (int k = 0; k < 4; ++k)
        if (!small_blocks || bss[k] <= 64) out[n++] = HopShape{0, bss[k], 0, 0};
      if (d <= 3) {
        out[n++] = HopShape{0, 64, 1, 0};
        out[n++] = HopShape{0, 128, 1, 0};
      }
    }
    if (!clover) {
#define HR_ROWS_CAND(DD, RE, RR) \
  if (d == DD && (is_real != 0) == RE) out[n++] = HopShape{0, 32 * ((DD + RR - 1) / RR), 0, 0, RR};
      HR_ROWS_SHAPES(HR_ROWS_CAND)
#undef HR_ROWS_CAND
    }
    return n;
  }
  if (multi_rhs && hr_has_tc_mrhs(d, is_real, prec))
    out[n++] = HopShape{0, 0, 0, HR_TC_MRHS + 16};  // link products of all rhs as MMA tiles
  if (site_mrhs && multi_rhs) {
    // links staged once per site for all right-hand sides of a block
    out[n++] = HopShape{0, 0, 0, 16};
    out[n++] = HopShape{0, 0, 0, 8};
  }
  if (site) {
    // compiler's register choice at 64 / 128 / 32 / 256 threads, then (not
    // for FP64, which is ALU-bound) the high- and low-register budgets
    const int bss[4] = {64, 128, 32, 256};
    for (int k = 0; k < 4; ++k) out[n++] = HopShape{0, bss[k], 0, 0};
    if (prec != HR_F64) {
      out[n++] = HopShape{0, 32, 1, 0};
      out[n++] = HopShape{0, 64, 1, 0};
      out[n++] = HopShape{0, 128, 1, 0};
      out[n++] = HopShape{0, 32, 2, 0};
      out[n++] = HopShape{0, 64, 2, 0};
      out[n++] = HopShape{0, 32, 3, 0};
      out[n++] = HopShape{0, 64, 3, 0};
      if (prec == HR_F32) {  // one-wave grids
        out[n++] = HopShape{0, 32, 4, 0};
        out[n++] = HopShape{0, 64, 4, 0};
      }
    }
  }
  if (!clover) {
    // rows kernel: every (d_R, R) pair built in hop_rows.cuh
#define HR_ROWS_CAND(DD, RE, RR) \
  if (d == DD && (is_real != 0) == RE) out[n++] = HopShape{0, 32 * ((DD + RR - 1) / RR), 0, 0, RR};
    HR_ROWS_SHAPES(HR_ROWS_CAND)
#undef HR_ROWS_CAND
    // colour-split kernel: every (d_R, G) pair built in hop_split.cuh
#define HR_SPLIT_CAND(DD, RE, GG) \
  if (d == DD && (is_real != 0) == RE) out[n++] = HopShape{GG, 128, 0, 0, 0};
    HR_SPLIT_SHAPES(HR_SPLIT_CAND)
#undef HR_SPLIT_CAND
  }
  return n;
}

// The candidates for this lattice: on a time slab only the site kernel with
// the compiler's register choice, the one built to mask the t hops across the
// slab faces.
static int lattice_shapes(const hr_lattice *lat, int prec, int clover, int multi_rhs, HopShape *out) {
  int n = hr_hop_shapes(lat->d, lat->is_real, prec, clover, multi_rhs, out);
  if (!lat->dom) return n;
  int m = 0;
  for (int k = 0; k < n; ++k)
    if (out[k].split_g == 0 && out[k].rows == 0 && out[k].mrhs == 0 && out[k].regs == 0) out[m++] = out[k];
  return m;
}

static int launch_shape(const hr_lattice *lat, int prec, const HopArgs &a, cudaStream_t s, HopShape sh) {
  switch (prec) {
    case HR_F64: return hr_launch_hop_f64(lat, a, s, sh);
    case HR_F32: return hr_launch_hop_f32(lat, a, s, sh);
    case HR_F16: return hr_launch_hop_f16(lat, a, s, sh);
    case HR_FF: return hr_launch_hop_ff(lat, a, s, sh);
  }
  return HR_ERR_ARG;
}

static std::mutex g_mu;
static std::map<long long, HopShape> g_best;

static long long tune_key(const hr_lattice *lat, int prec, const HopArgs &a) {
  int lg = 0;
  while (((int64_t)1 << lg) < lat->Vh) ++lg;
  int dev = lat->device;
  return (((((((long long)dev * 4 + prec) * 64 + lat->d) * 2 + lat->is_real) * 2 + (a.clover != nullptr)) * 2 +
           (a.nrhs > 1)) * 2 + lat->dom) * 64 + lg;
}

static bool tuning_enabled() {
  const char *e = getenv("HR_TUNE");
  return !(e && e[0] == '0');
}

int hr_launch_hop(const hr_lattice *lat, int prec, const HopArgs &a, cudaStream_t s) {
  HopShape shapes[HR_MAX_SHAPES];
  const int n = lattice_shapes(lat, prec, a.clover != nullptr, a.nrhs > 1, shapes);
  if (n == 0) return HR_ERR_UNSUPPORTED;
  const long long key = tune_key(lat, prec, a);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_best.find(key);
    if (it != g_best.end()) return launch_shape(lat, prec, a, s, it->second);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone || n == 1 ||
      !tuning_enabled())
    return launch_shape(lat, prec, a, s, shapes[0]);
  HrEvent e0_owner, e1_owner;
  HR_CUDA(cudaEventCreate(&e0_owner.e));
  HR_CUDA(cudaEventCreate(&e1_owner.e));
  cudaEvent_t e0 = e0_owner.e, e1 = e1_owner.e;
  // two sweeps over the candidates (the second in reverse order, so that no
  // shape always runs right after the same neighbour); each candidate keeps
  // the faster of its two timings of `reps` launches: 4 on large lattices,
  // 16 below 2^20 sites per parity, where one launch lasts only tens of
  // microseconds and 4 of them did not separate shapes 8 % apart
  float t[HR_MAX_SHAPES];
  for (int c = 0; c < n; ++c) t[c] = 1e30f;
  const int reps = lat->Vh < ((int64_t)1 << 20) ? 16 : 4;
  for (int sweep = 0; sweep < 2; ++sweep)
    for (int cc = 0; cc < n; ++cc) {
      const int c = sweep ? n - 1 - cc : cc;
      if (launch_shape(lat, prec, a, s, shapes[c]) != HR_OK) continue;  // warm-up; unsupported shapes drop out
      HR_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r) HR_TRY(launch_shape(lat, prec, a, s, shapes[c]));
      HR_CUDA(cudaEventRecord(e1, s));
      HR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      HR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < t[c]) t[c] = ms;
    }
  float best_ms = 1e30f;
  HopShape best = shapes[0];
  for (int c = 0; c < n; ++c)
    if (t[c] < best_ms) {
      best_ms = t[c];
      best = shapes[c];
    }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_best[key] = best;
  }
  return launch_shape(lat, prec, a, s, best);
}

// Report the tuned shape for the lattice's hop at (prec, nrhs, clover): returns
// its hr_shape_code, or -1 if not tuned yet.
extern "C" int hr_tuned_shape(const hr_lattice *lat, int prec, int nrhs, int clover) {
  if (!lat) return -1;
  HopArgs a;
  memset(&a, 0, sizeof(a));
  a.nrhs = nrhs;
  a.clover = clover ? (const void *)1 : nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_best.find(tune_key(lat, prec, a));
  if (it == g_best.end()) return -1;
  return hr_shape_code(it->second);
}

// Candidate shapes of this lattice's hop, encoded as hr_tuned_shape reports them.
extern "C" int hr_hop_shape_candidates(const hr_lattice *lat, int prec, int nrhs, int clover, int *out, int max) {
  if (!lat || !out || max < 1 || prec < HR_F64 || prec > HR_FF || nrhs < 1) return HR_ERR_ARG;
  HopShape shapes[HR_MAX_SHAPES];
  const int n = lattice_shapes(lat, prec, clover, nrhs > 1, shapes);
  for (int k = 0; k < n && k < max; ++k)
    out[k] = hr_shape_code(shapes[k]);
  return n;
}

// Pin the shape used for (prec, nrhs, clover) on this lattice's size class,
// bypassing the timing; the shape must be one of the candidates.
extern "C" int hr_set_tuned_shape(const hr_lattice *lat, int prec, int nrhs, int clover, int shape) {
  if (!lat || prec < HR_F64 || prec > HR_FF || nrhs < 1) return HR_ERR_ARG;
  HopShape shapes[HR_MAX_SHAPES];
  const int n = lattice_shapes(lat, prec, clover, nrhs > 1, shapes);
  for (int k = 0; k < n; ++k)
    if (hr_shape_code(shapes[k]) == shape) {
      HopArgs a;
      memset(&a, 0, sizeof(a));
      a.nrhs = nrhs;
      a.clover = clover ? (const void *)1 : nullptr;
      std::lock_guard<std::mutex> lk(g_mu);
      g_best[tune_key(lat, prec, a)] = shapes[k];
      return HR_OK;
    }
  return HR_ERR_ARG;
}
