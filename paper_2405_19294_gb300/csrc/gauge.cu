// Gauge-field set-up on the GPU, all in FP64:
//   * synthetic links U = exp(i eps sum_k a_k T_k) (scaling and squaring of
//     the Taylor series) with optional reunitarisation;
//   * the represented field U_R (Sec. 3.1.2, "represented gauge field") for
//     the fundamental, adjoint, 2-index symmetric and antisymmetric
//     representations, with the antiperiodic-time sign, written in the
//     internal link layout in FP64, FP32 and FP16;
//   * export of U_R back to the canonical layout (for checking).
//
// The map U -> U_R is evaluated entry by entry from closed forms derived from
// the definitions (T_a generalised Gell-Mann, tr T_a T_b = delta/2; e^(ab)
// the orthonormal (anti)symmetric basis, a <= b resp. a < b, lexicographic):
//   adj : (U_R)_ab = 2 Re tr(T_a U T_b U^+)
//                  = 2 Re sum_{(i,j,t) in T_a} sum_{(k,l,t') in T_b} t t' U_jk conj(U_il)
//   sym : (U_R)_(ab),(cd) = n_ab n_cd (U_ac U_bd + U_ad U_bc),
//         n = 1 for a != b, 1/sqrt2 for a == b  (so (aa),(cc) -> U_ac^2)
//   asym: (U_R)_(ab),(cd) = U_ac U_bd - U_ad U_bc
#include <math.h>

#include "cplx.cuh"
#include "hr_internal.h"

typedef cx<double> zd;

__device__ __forceinline__ zd zmul(zd a, zd b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ zd zconj(zd a) { return mk(a.x, -a.y); }

// nonzero entries of generator T_a of su(N): count, rows, cols, values
struct GenNZ {
  int n;
  int r[HR_MAX_NC], c[HR_MAX_NC];
  zd v[HR_MAX_NC];
};

__device__ void generator_nz(int N, int a, GenNZ &g) {
  const int noff = N * (N - 1);
  if (a < noff) {
    int q = a >> 1, j = 0;
    while (q >= N - 1 - j) {  // pair q in lexicographic order of (j < k)
      q -= N - 1 - j;
      ++j;
    }
    const int k = j + 1 + q;
    g.n = 2;
    g.r[0] = j; g.c[0] = k;
    g.r[1] = k; g.c[1] = j;
    if ((a & 1) == 0) {
      g.v[0] = mk(0.5, 0.0);
      g.v[1] = mk(0.5, 0.0);
    } else {
      g.v[0] = mk(0.0, -0.5);
      g.v[1] = mk(0.0, 0.5);
    }
  } else {
    const int m = a - noff + 1;
    const double nrm = 1.0 / sqrt(2.0 * m * (m + 1));
    g.n = m + 1;
    for (int i = 0; i < m; ++i) {
      g.r[i] = g.c[i] = i;
      g.v[i] = mk(nrm, 0.0);
    }
    g.r[m] = g.c[m] = m;
    g.v[m] = mk(-m * nrm, 0.0);
  }
}

// index pair (a, b) of basis vector q of the 2-index representation
__device__ void two_index_pair(int N, bool sym, int q, int &a, int &b) {
  for (a = 0; a < N; ++a) {
    const int cnt = sym ? N - a : N - a - 1;
    if (q < cnt) {
      b = sym ? a + q : a + 1 + q;
      return;
    }
    q -= cnt;
  }
  a = b = 0;
}

// --------------------------------------------------------- SU(N) helpers ----
__device__ zd det_lu(zd *M, int N) {
  // Gaussian elimination with partial pivoting on a scratch copy
  zd det = mk(1.0, 0.0);
  for (int k = 0; k < N; ++k) {
    int piv = k;
    double best = M[k * N + k].x * M[k * N + k].x + M[k * N + k].y * M[k * N + k].y;
    for (int r = k + 1; r < N; ++r) {
      const double v = M[r * N + k].x * M[r * N + k].x + M[r * N + k].y * M[r * N + k].y;
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (best == 0.0) return mk(0.0, 0.0);
    if (piv != k) {
      for (int c = 0; c < N; ++c) {
        zd t = M[k * N + c];
        M[k * N + c] = M[piv * N + c];
        M[piv * N + c] = t;
      }
      det = mk(-det.x, -det.y);
    }
    const zd pk = M[k * N + k];
    det = zmul(det, pk);
    const double inv = 1.0 / best;
    const zd pinv = mk(pk.x * inv, -pk.y * inv);
    for (int r = k + 1; r < N; ++r) {
      const zd f = zmul(M[r * N + k], pinv);
      for (int c = k; c < N; ++c) M[r * N + c] = M[r * N + c] - zmul(f, M[k * N + c]);
    }
  }
  return det;
}

// rows Gram-Schmidt (modified), then last row times conj(det)
template <int NM>
__device__ void reunitarise_dev(zd *U, int N) {
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < i; ++j) {
      zd pr = mk(0.0, 0.0);
      for (int c = 0; c < N; ++c) pr = pr + zmul(zconj(U[j * N + c]), U[i * N + c]);
      for (int c = 0; c < N; ++c) U[i * N + c] = U[i * N + c] - zmul(pr, U[j * N + c]);
    }
    double n2 = 0.0;
    for (int c = 0; c < N; ++c) n2 += U[i * N + c].x * U[i * N + c].x + U[i * N + c].y * U[i * N + c].y;
    const double inv = 1.0 / sqrt(n2);
    for (int c = 0; c < N; ++c) U[i * N + c] = scale(inv, U[i * N + c]);
  }
  zd M[NM * NM];
  for (int e = 0; e < N * N; ++e) M[e] = U[e];
  const zd dt = zconj(det_lu(M, N));
  for (int c = 0; c < N; ++c) U[(N - 1) * N + c] = zmul(U[(N - 1) * N + c], dt);
}

// ------------------------------------------------------ link generation ----
template <int NM>
__global__ void links_from_algebra_kernel(double *U_out, const double *a_in, double eps, int N, int64_t nlinks,
                                          int reun) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  const int ng = N * N - 1;
  const double *a = a_in + l * ng;
  // X = i eps H, H = sum_k a_k T_k
  zd X[NM * NM];
  for (int e = 0; e < N * N; ++e) X[e] = mk(0.0, 0.0);
  for (int k = 0; k < ng; ++k) {
    GenNZ g;
    generator_nz(N, k, g);
    for (int q = 0; q < g.n; ++q) {
      const zd v = g.v[q];  // i eps a_k v
      X[g.r[q] * N + g.c[q]] = X[g.r[q] * N + g.c[q]] + mk(-eps * a[k] * v.y, eps * a[k] * v.x);
    }
  }
  // scaling: |X|_F / 2^s <= 1/2
  double fn = 0.0;
  for (int e = 0; e < N * N; ++e) fn += X[e].x * X[e].x + X[e].y * X[e].y;
  fn = sqrt(fn);
  int s = 0;
  while (fn > 0.5) {
    fn *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  for (int e = 0; e < N * N; ++e) X[e] = scale(sc, X[e]);
  // Taylor series to order 18: E = sum_k X^k / k!
  zd E[NM * NM], Tm[NM * NM], W[NM * NM];
  for (int e = 0; e < N * N; ++e) {
    E[e] = mk((e % (N + 1) == 0) ? 1.0 : 0.0, 0.0);
    Tm[e] = E[e];
  }
  for (int k = 1; k <= 18; ++k) {
    const double ik = 1.0 / k;
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {
        zd acc = mk(0.0, 0.0);
        for (int q = 0; q < N; ++q) acc = acc + zmul(Tm[r * N + q], X[q * N + c]);
        W[r * N + c] = scale(ik, acc);
      }
    for (int e = 0; e < N * N; ++e) {
      Tm[e] = W[e];
      E[e] = E[e] + W[e];
    }
  }
  // squaring
  for (int q2 = 0; q2 < s; ++q2) {
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {
        zd acc = mk(0.0, 0.0);
        for (int q = 0; q < N; ++q) acc = acc + zmul(E[r * N + q], E[q * N + c]);
        W[r * N + c] = acc;
      }
    for (int e = 0; e < N * N; ++e) E[e] = W[e];
  }
  if (reun) reunitarise_dev<NM>(E, N);
  double *o = U_out + l * 2 * N * N;
  for (int e = 0; e < N * N; ++e) {
    o[2 * e] = E[e].x;
    o[2 * e + 1] = E[e].y;
  }
}

extern "C" int hr_links_from_algebra(hr_lattice *lat, double *U_dev, const double *a_dev, double eps,
                                     int reunitarise) {
  if (!lat || !U_dev || !a_dev) return HR_ERR_ARG;
  const int64_t nl = lat->V * 4;
  const unsigned nb = (unsigned)((nl + 127) / 128);
  if (lat->N <= 6)  // smaller per-thread scratch for the common groups
    links_from_algebra_kernel<6><<<nb, 128, 0, lat->stream>>>(U_dev, a_dev, eps, lat->N, nl, reunitarise);
  else
    links_from_algebra_kernel<HR_MAX_NC><<<nb, 128, 0, lat->stream>>>(U_dev, a_dev, eps, lat->N, nl, reunitarise);
  return hr_check_launch("links_from_algebra_kernel");
}

// ----------------------------------------------------------- U -> U_R ------
struct RepK {
  int T, L, Lh, N, rep, d, nch, reun, t0, Tg;
  int64_t V, Vh;
};

__device__ zd rep_entry(const zd *U, int N, int rep, int ra, int rb) {
  if (rep == HR_FUND) return U[ra * N + rb];
  if (rep == HR_ADJ) {
    GenNZ ga, gb;
    generator_nz(N, ra, ga);
    generator_nz(N, rb, gb);
    zd s = mk(0.0, 0.0);
    for (int p = 0; p < ga.n; ++p)      // (T_a)_{ij}, i = ga.r, j = ga.c
      for (int q = 0; q < gb.n; ++q) {  // (T_b)_{kl}
        const zd t = zmul(ga.v[p], gb.v[q]);
        const zd u = zmul(U[ga.c[p] * N + gb.r[q]], zconj(U[ga.r[p] * N + gb.c[q]]));
        s = s + zmul(t, u);
      }
    return mk(2.0 * s.x, 0.0);
  }
  const bool sym = rep == HR_SYM;
  int a, b, c, dd;
  two_index_pair(N, sym, ra, a, b);
  two_index_pair(N, sym, rb, c, dd);
  const zd t1 = zmul(U[a * N + c], U[b * N + dd]);
  const zd t2 = zmul(U[a * N + dd], U[b * N + c]);
  if (!sym) return t1 - t2;
  const double nab = (a == b) ? M_SQRT1_2 : 1.0;
  const double ncd = (c == dd) ? M_SQRT1_2 : 1.0;
  return scale(nab * ncd, t1 + t2);
}

template <int NM>
__global__ void represent_kernel(void *l64, void *l32, void *l16, const double *U_in, RepK k) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= k.V * 4) return;
  const int64_t x = l >> 2;
  const int mu = (int)(l & 3);
  const int N = k.N, d = k.d;
  zd U[NM * NM];
  const double *src = U_in + l * 2 * N * N;
  for (int e = 0; e < N * N; ++e) U[e] = mk(src[2 * e], src[2 * e + 1]);
  if (k.reun) reunitarise_dev<NM>(U, N);
  // coordinates from the lexicographic index
  const int xx = (int)(x % k.L);
  const int yy = (int)((x / k.L) % k.L);
  const int zz = (int)((x / ((int64_t)k.L * k.L)) % k.L);
  const int tt = (int)(x / ((int64_t)k.L * k.L * k.L));
  const int par = (tt + xx + yy + zz) & 1;
  const int64_t i = cb_index(tt, xx, yy, zz, k.L, k.Lh);
  const double sg = (mu == 0 && k.t0 + tt == k.Tg - 1) ? -1.0 : 1.0;  // antiperiodic in global time
  const int64_t base = ((int64_t)(par * 4 + mu) * k.nch) * k.Vh;
  if (k.rep == HR_ADJ) {
    for (int q = 0; q < k.nch; ++q) {
      double v[2];
      for (int h = 0; h < 2; ++h) {
        const int e = 2 * q + h;
        v[h] = (e < d * d) ? sg * rep_entry(U, N, k.rep, e / d, e % d).x : 0.0;
      }
      const int64_t idx = base + (int64_t)q * k.Vh + i;
      reinterpret_cast<double2 *>(l64)[idx] = make_double2(v[0], v[1]);
      reinterpret_cast<float2 *>(l32)[idx] = make_float2((float)v[0], (float)v[1]);
      reinterpret_cast<__half2 *>(l16)[idx] = __floats2half2_rn((float)v[0], (float)v[1]);
    }
  } else {
    for (int e = 0; e < d * d; ++e) {
      const zd v = scale(sg, rep_entry(U, N, k.rep, e / d, e % d));
      const int64_t idx = base + (int64_t)e * k.Vh + i;
      reinterpret_cast<double2 *>(l64)[idx] = make_double2(v.x, v.y);
      reinterpret_cast<float2 *>(l32)[idx] = make_float2((float)v.x, (float)v.y);
      reinterpret_cast<__half2 *>(l16)[idx] = __floats2half2_rn((float)v.x, (float)v.y);
    }
  }
}

int hr_clover_build(hr_lattice *lat);

// ------------------------------------------------ rows-kernel link layout ----
// One thread per (output parity p, direction n, output site i): V_n(x) from
// the FP64 internal links -- U_R,mu(x) itself (n even) or the adjoint of
// U_R,mu(x - mu) (n odd, read from the other parity's slot) -- written
// row-major at the output site in all three precisions (hr_rows_nch).
__global__ void rows_links_kernel(void *r64, void *r32, void *r16, const void *l64, RepK k) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= 16 * k.Vh) return;
  const int64_t i = g % k.Vh;
  const int pn = (int)(g / k.Vh);  // p * 8 + n
  const int p = pn >> 3, n = pn & 7, mu = n >> 1;
  const bool back = n & 1;
  const int d = k.d;
  const bool real = k.rep == HR_ADJ;
  const Site s = site_of(i, p, k.L, k.Lh);
  int c4[4] = {s.t, s.x, s.y, s.z};
  const int ext[4] = {k.T, k.L, k.L, k.L};
  int64_t j = i;
  int sp = p;
  if (back) {
    c4[mu] = (c4[mu] + ext[mu] - 1) % ext[mu];
    j = cb_index(c4[0], c4[1], c4[2], c4[3], k.L, k.Lh);
    sp = 1 - p;
  }
  const double2 *src = reinterpret_cast<const double2 *>(l64) + ((int64_t)(sp * 4 + mu) * k.nch) * k.Vh;
  const int dp = hr_rows_dp(d, real), nch = hr_rows_nch(d, real);
  const int64_t obase = (int64_t)pn * nch * k.Vh + i;
  double2 *o64 = reinterpret_cast<double2 *>(r64);
  float2 *o32 = reinterpret_cast<float2 *>(r32);
  __half2 *o16 = reinterpret_cast<__half2 *>(r16);
  // U element (a, c) at the source site
  auto uel = [&](int a, int c) -> zd {
    const int e = a * d + c;
    if (real) {
      const double2 v = src[(int64_t)(e >> 1) * k.Vh + j];
      return mk((e & 1) ? v.y : v.x, 0.0);
    }
    const double2 v = src[(int64_t)e * k.Vh + j];
    return mk(v.x, v.y);
  };
  auto vel = [&](int a, int c) -> zd {  // V[a][c]
    if (c >= d) return mk(0.0, 0.0);
    return back ? zconj(uel(c, a)) : uel(a, c);
  };
  if (real) {
    for (int a = 0; a < d; ++a)
      for (int c = 0; c < dp; c += 2) {
        const double v0 = vel(a, c).x, v1 = vel(a, c + 1).x;
        const int64_t idx = obase + (int64_t)((a * dp + c) >> 1) * k.Vh;
        o64[idx] = make_double2(v0, v1);
        o32[idx] = make_float2((float)v0, (float)v1);
        o16[idx] = __floats2half2_rn((float)v0, (float)v1);
      }
  } else {
    for (int a = 0; a < d; ++a)
      for (int c = 0; c < d; ++c) {
        const zd v = vel(a, c);
        const int64_t idx = obase + (int64_t)(a * d + c) * k.Vh;
        o64[idx] = make_double2(v.x, v.y);
        o32[idx] = make_float2((float)v.x, (float)v.y);
        o16[idx] = __floats2half2_rn((float)v.x, (float)v.y);
      }
  }
}

// 16 matrices of hr_rows_nch chunk rows, then HR_ROWS_SLACK zeroed chunk rows
// (hr_internal.h)
static int hr_rows_links_build(hr_lattice *lat, const RepK &k) {
  const size_t nrows = (size_t)16 * hr_rows_nch(lat->d, lat->is_real);
  const size_t es[3] = {16, 8, 4};
  for (int p = 0; p < 3; ++p) {
    if (!lat->rlinks[p])
      HR_TRY(hr_dev_alloc(&lat->rlinks[p], (nrows + HR_ROWS_SLACK) * (size_t)lat->Vh * es[p]));
    HR_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(lat->rlinks[p]) + nrows * (size_t)lat->Vh * es[p], 0,
                            (size_t)HR_ROWS_SLACK * lat->Vh * es[p], lat->stream));
  }
  const int64_t nt = 16 * lat->Vh;
  rows_links_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, lat->stream>>>(lat->rlinks[0], lat->rlinks[1],
                                                                          lat->rlinks[2], lat->links[0], k);
  return hr_check_launch("rows_links_kernel");
}

extern "C" int hr_represent_links(hr_lattice *lat, const double *U_dev, int reunitarise, double csw) {
  if (!lat || !U_dev) return HR_ERR_ARG;
  if (lat->dom && csw != 0.0) return HR_ERR_UNSUPPORTED;  // the clover leaves would need a link halo
  const size_t nchunks = (size_t)2 * 4 * lat->nch_link * (size_t)lat->Vh;
  const size_t es[3] = {16, 8, 4};
  for (int p = 0; p < 3; ++p)
    if (!lat->links[p]) HR_TRY(hr_dev_alloc(&lat->links[p], nchunks * es[p]));
  RepK k;
  k.T = lat->T;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.N = lat->N;
  k.rep = lat->rep;
  k.d = lat->d;
  k.nch = lat->nch_link;
  k.reun = reunitarise;
  k.V = lat->V;
  k.Vh = lat->Vh;
  k.t0 = lat->t0;
  k.Tg = lat->Tg;
  const int64_t nl = lat->V * 4;
  if (lat->N <= 6)
    represent_kernel<6><<<(unsigned)((nl + 63) / 64), 64, 0, lat->stream>>>(lat->links[0], lat->links[1],
                                                                          lat->links[2], U_dev, k);
  else
    represent_kernel<HR_MAX_NC><<<(unsigned)((nl + 63) / 64), 64, 0, lat->stream>>>(lat->links[0], lat->links[1],
                                                                                  lat->links[2], U_dev, k);
  HR_TRY(hr_check_launch("represent_kernel"));
  // the rows kernel (no clover) reads its own layout of the same links
  if (csw == 0.0 && !lat->dom && hr_has_rows_shapes(lat->d, lat->is_real)) HR_TRY(hr_rows_links_build(lat, k));
  lat->have_links = 1;
  lat->ff_links_ok = 0;
  lat->csw = csw;
  lat->clover_cached = 0;
  if (csw != 0.0) HR_TRY(hr_clover_build(lat));
  HR_CUDA(cudaStreamSynchronize(lat->stream));
  return HR_OK;
}

__global__ void export_links_kernel(double *out, const void *l64, RepK k) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= k.V * 4) return;
  const int64_t x = l >> 2;
  const int mu = (int)(l & 3);
  const int xx = (int)(x % k.L);
  const int yy = (int)((x / k.L) % k.L);
  const int zz = (int)((x / ((int64_t)k.L * k.L)) % k.L);
  const int tt = (int)(x / ((int64_t)k.L * k.L * k.L));
  const int par = (tt + xx + yy + zz) & 1;
  const int64_t i = cb_index(tt, xx, yy, zz, k.L, k.Lh);
  const int64_t base = ((int64_t)(par * 4 + mu) * k.nch) * k.Vh;
  const int d = k.d;
  double *o = out + l * 2 * d * d;
  const double2 *src = reinterpret_cast<const double2 *>(l64);
  for (int e = 0; e < d * d; ++e) {
    if (k.rep == HR_ADJ) {
      const double2 v = src[base + (int64_t)(e >> 1) * k.Vh + i];
      o[2 * e] = (e & 1) ? v.y : v.x;
      o[2 * e + 1] = 0.0;
    } else {
      const double2 v = src[base + (int64_t)e * k.Vh + i];
      o[2 * e] = v.x;
      o[2 * e + 1] = v.y;
    }
  }
}

extern "C" int hr_export_represented_links(hr_lattice *lat, double *UR_dev) {
  if (!lat || !UR_dev) return HR_ERR_ARG;
  if (!lat->have_links) return HR_ERR_STATE;
  RepK k;
  k.T = lat->T;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.N = lat->N;
  k.rep = lat->rep;
  k.d = lat->d;
  k.nch = lat->nch_link;
  k.reun = 0;
  k.V = lat->V;
  k.Vh = lat->Vh;
  k.t0 = lat->t0;
  k.Tg = lat->Tg;
  const int64_t nl = lat->V * 4;
  export_links_kernel<<<(unsigned)((nl + 127) / 128), 128, 0, lat->stream>>>(UR_dev, lat->links[0], k);
  return hr_check_launch("export_links_kernel");
}
