// hr_dphi (the full operator and the even-odd Schur complement, Sec. 3.1) and
// the clover term (Sheikholeslami-Wohlert, Sec. 3.1): its FP64 build from
// U_R and the per-m0 diagonal blocks A and A^{-1}.
//
// Clover algebra used by the build (derived from sigma_mu_nu = (i/2)[g_mu, g_nu]
// in the chiral basis, where g_mu = [[0, e_mu], [e_mu^+, 0]], e_0 = -1,
// e_k = -i s_k):  sigma_mu_nu = diag(sigma+_mu_nu, sigma-_mu_nu) with
//   sigma+-_0k = +-s_k,   sigma+-_jk = -eps_jkl s_l.
// Hence the term csw (i/4) sum_{mu,nu} sigma_mu_nu Fhat_mu_nu splits into two
// Hermitian 2d x 2d chiral blocks
//   C+- = csw (i/2) sum_l s_l (x) G+-_l,   G+-_l = +-Fhat_0l - (1/2) eps_ljk Fhat_jk,
// i.e. with G = G+- :  C = csw (i/2) [[G_3, G_1 - i G_2], [G_1 + i G_2, -G_3]].
#include <math.h>
#include <string.h>

#include "cplx.cuh"
#include "hr_internal.h"

#define HR_CLOVER_MAX_D 8

typedef cx<double> zd;
__device__ __forceinline__ zd zmul2(zd a, zd b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

int hr_ensure_tmp(hr_lattice *lat, size_t bytes) {
  if (lat->tmp_bytes >= bytes) return HR_OK;
  cudaStreamSynchronize(lat->stream);
  hr_dev_free(lat->tmp);
  lat->tmp = nullptr;
  lat->tmp_bytes = 0;
  HR_TRY(hr_dev_alloc(&lat->tmp, bytes));
  lat->tmp_bytes = bytes;
  return HR_OK;
}

// ------------------------------------------------------------ clover build --
struct ClK {
  int T, L, Lh, d, nch;
  int64_t V, Vh;
  double csw;
};

// U_R,mu at lexicographic site x (FP64 internal links), into M[d*d]
__device__ void load_link(const ClK &k, const void *l64, int t, int x, int y, int z, int mu, zd *M, bool is_real) {
  const int par = (t + x + y + z) & 1;
  const int64_t i = cb_index(t, x, y, z, k.L, k.Lh);
  const int64_t base = ((int64_t)(par * 4 + mu) * k.nch) * k.Vh;
  const double2 *src = reinterpret_cast<const double2 *>(l64);
  const int d = k.d;
  for (int e = 0; e < d * d; ++e) {
    if (is_real) {
      const double2 v = src[base + (int64_t)(e >> 1) * k.Vh + i];
      M[e] = mk((e & 1) ? v.y : v.x, 0.0);
    } else {
      const double2 v = src[base + (int64_t)e * k.Vh + i];
      M[e] = mk(v.x, v.y);
    }
  }
}

// C = A * B (dagA / dagB: use the adjoint of that operand)
__device__ void matmul(const zd *A, const zd *B, zd *C, int d, bool dagA, bool dagB) {
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      zd s = mk(0.0, 0.0);
      for (int q = 0; q < d; ++q) {
        zd a = dagA ? mk(A[q * d + r].x, -A[q * d + r].y) : A[r * d + q];
        zd b = dagB ? mk(B[c * d + q].x, -B[c * d + q].y) : B[q * d + c];
        s = s + zmul2(a, b);
      }
      C[r * d + c] = s;
    }
}

// Q_mu_nu(x): the four leaves, each circling its plaquette from +mu to +nu
__device__ void leaves(const ClK &k, const void *l64, int t, int x, int y, int z, int mu, int nu, zd *Q,
                       bool is_real) {
  const int d = k.d;
  zd A[HR_CLOVER_MAX_D * HR_CLOVER_MAX_D], B[HR_CLOVER_MAX_D * HR_CLOVER_MAX_D],
      W[HR_CLOVER_MAX_D * HR_CLOVER_MAX_D];
  int ext[4] = {k.T, k.L, k.L, k.L};
  auto sh = [&](int c[4], int m, int dir) { c[m] = (c[m] + dir + ext[m]) % ext[m]; };
  for (int e = 0; e < d * d; ++e) Q[e] = mk(0.0, 0.0);
  // leaf = L1 L2 L3 L4 with links given by (start point offsets, direction, dagger)
  // encoded as: for each leaf, 4 links (site shift in mu, site shift in nu, dir, dag)
  const int legs[4][4][4] = {
      {{0, 0, 0, 0}, {1, 0, 1, 0}, {0, 1, 0, 1}, {0, 0, 1, 1}},      // U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
      {{0, 0, 1, 0}, {-1, 1, 0, 1}, {-1, 0, 1, 1}, {-1, 0, 0, 0}},   // U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
      {{-1, 0, 0, 1}, {-1, -1, 1, 1}, {-1, -1, 0, 0}, {0, -1, 1, 0}},  // U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
      {{0, -1, 1, 1}, {0, -1, 0, 0}, {1, -1, 1, 0}, {0, 0, 0, 1}}};  // U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
  for (int lf = 0; lf < 4; ++lf) {
    for (int g = 0; g < 4; ++g) {
      int c[4] = {t, x, y, z};
      if (legs[lf][g][0]) sh(c, mu, legs[lf][g][0]);
      if (legs[lf][g][1]) sh(c, nu, legs[lf][g][1]);
      const int dir = legs[lf][g][2] ? nu : mu;
      load_link(k, l64, c[0], c[1], c[2], c[3], dir, B, is_real);
      if (g == 0) {
        for (int e = 0; e < d * d; ++e)
          A[e] = legs[lf][g][3] ? mk(B[(e % d) * d + e / d].x, -B[(e % d) * d + e / d].y) : B[e];
      } else {
        matmul(A, B, W, d, false, legs[lf][g][3] != 0);
        for (int e = 0; e < d * d; ++e) A[e] = W[e];
      }
    }
    for (int e = 0; e < d * d; ++e) Q[e] = Q[e] + A[e];
  }
}

// packed index of entry (r, c) of a Hermitian n x n block; returns chunk and
// whether it is a diagonal real (half = component) or a complex lower entry
__device__ __forceinline__ int64_t herm_chunk(int d, int r, int c) {
  if (r == c) return r >> 1;
  return d + (int64_t)r * (r - 1) / 2 + c;  // requires r > c
}

__global__ void clover_term_kernel(void *term, const void *l64, ClK k, int is_real) {
  const int64_t xl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (xl >= k.V) return;
  const int d = k.d, n = 2 * d;
  const int xx = (int)(xl % k.L);
  const int yy = (int)((xl / k.L) % k.L);
  const int zz = (int)((xl / ((int64_t)k.L * k.L)) % k.L);
  const int tt = (int)(xl / ((int64_t)k.L * k.L * k.L));
  const int par = (tt + xx + yy + zz) & 1;
  const int64_t i = cb_index(tt, xx, yy, zz, k.L, k.Lh);
  // G+-_l, l = 1..3 accumulated from the six planes
  zd Gp[3][HR_CLOVER_MAX_D * HR_CLOVER_MAX_D], Gm[3][HR_CLOVER_MAX_D * HR_CLOVER_MAX_D];
  zd Q[HR_CLOVER_MAX_D * HR_CLOVER_MAX_D];
  for (int l = 0; l < 3; ++l)
    for (int e = 0; e < d * d; ++e) Gp[l][e] = Gm[l][e] = mk(0.0, 0.0);
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu) {
      leaves(k, l64, tt, xx, yy, zz, mu, nu, Q, is_real != 0);
      // Fhat = (Q - Q^+)/8
      zd F[HR_CLOVER_MAX_D * HR_CLOVER_MAX_D];
      for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
          const zd a = Q[r * d + c], b = Q[c * d + r];
          F[r * d + c] = mk((a.x - b.x) * 0.125, (a.y + b.y) * 0.125);
        }
      if (mu == 0) {
        const int l = nu - 1;  // Fhat_0l
        for (int e = 0; e < d * d; ++e) {
          Gp[l][e] = Gp[l][e] + F[e];
          Gm[l][e] = Gm[l][e] - F[e];
        }
      } else {
        // -(1/2) eps_ljk Fhat_jk summed over j,k = -eps_l(mu)(nu) Fhat_mu_nu for mu < nu
        const int l = 6 - mu - nu - 1;  // the remaining spatial direction, 0-based
        const int sgn = (mu == 1 && nu == 3) ? 1 : -1;  // eps_{l mu nu}: (1,2)->3 +, (1,3)->2 -, (2,3)->1 +
        for (int e = 0; e < d * d; ++e) {
          Gp[l][e] = Gp[l][e] + scale((double)sgn, F[e]);
          Gm[l][e] = Gm[l][e] + scale((double)sgn, F[e]);
        }
      }
    }
  // C = csw (i/2) [[G3, G1 - i G2], [G1 + i G2, -G3]]; store the lower triangle + diagonal
  double2 *out = reinterpret_cast<double2 *>(term);
  const int64_t pbase = (int64_t)par * (4 * d * d) * k.Vh;
  const double h = 0.5 * k.csw;
  for (int b = 0; b < 2; ++b) {
    zd(*G)[HR_CLOVER_MAX_D * HR_CLOVER_MAX_D] = b == 0 ? Gp : Gm;
    const int64_t boff = pbase + (int64_t)b * 2 * d * d * k.Vh;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c <= r; ++c) {
        const int sr = r / d, ar = r % d, sc = c / d, ac = c % d;
        zd g;
        const int e = ar * d + ac;
        if (sr == 0 && sc == 0) g = G[2][e];
        else if (sr == 1 && sc == 1) g = mk(-G[2][e].x, -G[2][e].y);
        else if (sr == 1 && sc == 0) g = mk(G[0][e].x - G[1][e].y, G[0][e].y + G[1][e].x);  // G1 + i G2
        else g = mk(G[0][e].x + G[1][e].y, G[0][e].y - G[1][e].x);                          // G1 - i G2
        const zd v = mk(-h * g.y, h * g.x);  // csw (i/2) g
        if (r == c) {
          // diagonal: real part only (Hermitian); two diagonal reals per chunk
          double2 *slot = out + boff + herm_chunk(d, r, c) * k.Vh + i;
          if (r & 1) slot->y = v.x;
          else slot->x = v.x;
        } else {
          out[boff + herm_chunk(d, r, c) * k.Vh + i] = make_double2(v.x, v.y);
        }
      }
  }
}

int hr_clover_build(hr_lattice *lat) {
  if (lat->d > HR_CLOVER_MAX_D) return HR_ERR_UNSUPPORTED;
  const int d = lat->d;
  const size_t bytes = (size_t)2 * 4 * d * d * (size_t)lat->Vh * 16u;
  if (!lat->clover_term) HR_TRY(hr_dev_alloc(&lat->clover_term, bytes));
  ClK k;
  k.T = lat->T;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.d = d;
  k.nch = lat->nch_link;
  k.V = lat->V;
  k.Vh = lat->Vh;
  k.csw = lat->csw;
  clover_term_kernel<<<(unsigned)((lat->V + 63) / 64), 64, 0, lat->stream>>>(lat->clover_term, lat->links[0], k,
                                                                             lat->is_real);
  HR_TRY(hr_check_launch("clover_term_kernel"));
  lat->clover_cached = 0;
  return HR_OK;
}

// exp(X) of an n x n complex matrix in place, by scaling and squaring: with
// 2^s >= 4 |X|_F, Y = X / 2^s has norm <= 1/4, its Taylor series is summed to
// order 16 by Horner's rule (truncation below 1e-23 relative), and the result
// is squared s times.  E and W are n x n scratch.
__device__ void expm_taylor(zd *X, zd *E, zd *W, int n) {
  double f = 0.0;
  for (int e = 0; e < n * n; ++e) f += X[e].x * X[e].x + X[e].y * X[e].y;
  f = sqrt(f);
  int s = 0;
  while (f > 0.25 && s < 60) {
    f *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  for (int e = 0; e < n * n; ++e) X[e] = mk(X[e].x * sc, X[e].y * sc);
  for (int e = 0; e < n * n; ++e) E[e] = mk((e / n == e % n) ? 1.0 : 0.0, 0.0);
  for (int q = 16; q >= 1; --q) {  // E <- 1 + Y E / q
    matmul(X, E, W, n, false, false);
    const double iq = 1.0 / q;
    for (int e = 0; e < n * n; ++e) E[e] = mk(W[e].x * iq + ((e / n == e % n) ? 1.0 : 0.0), W[e].y * iq);
  }
  for (int r = 0; r < s; ++r) {
    matmul(E, E, W, n, false, false);
    for (int e = 0; e < n * n; ++e) E[e] = W[e];
  }
  for (int e = 0; e < n * n; ++e) X[e] = E[e];
}

// A = (4 + m0) + C, or with `expo` the exponentiated clover term of Francis,
// Fritzsch, Luscher and Rago (Sec. 3.1): A = (4 + m0) exp(C / (4 + m0));
// and A^{-1}, per chiral block, by Gauss-Jordan elimination with partial
// pivoting in FP64.  exp maps each chiral block to itself, so the exponential
// is taken block by block.
__global__ void clover_diag_kernel(void *A64, void *A32, void *I64, void *I32, const void *term, ClK k,
                                   double m0, int expo) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (parity, block, site)
  if (g >= 4 * k.Vh) return;
  const int64_t i = g % k.Vh;
  const int pb = (int)(g / k.Vh);  // parity*2 + block
  const int d = k.d, n = 2 * d;
  const int64_t boff = (int64_t)pb * 2 * d * d * k.Vh;
  const double2 *tm = reinterpret_cast<const double2 *>(term);
  zd M[4 * HR_CLOVER_MAX_D * HR_CLOVER_MAX_D], Inv[4 * HR_CLOVER_MAX_D * HR_CLOVER_MAX_D];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c <= r; ++c) {
      const double2 v = tm[boff + herm_chunk(d, r, c) * k.Vh + i];
      if (r == c) {
        M[r * n + r] = mk(((r & 1) ? v.y : v.x) + 4.0 + m0, 0.0);
      } else {
        M[r * n + c] = mk(v.x, v.y);
        M[c * n + r] = mk(v.x, -v.y);
      }
    }
  if (expo) {  // M <- c exp((M - c) / c), Inv as scratch
    zd W[4 * HR_CLOVER_MAX_D * HR_CLOVER_MAX_D];
    const double c = 4.0 + m0, ic = 1.0 / c;
    for (int e = 0; e < n * n; ++e) M[e] = mk((M[e].x - ((e / n == e % n) ? c : 0.0)) * ic, M[e].y * ic);
    expm_taylor(M, Inv, W, n);
    for (int e = 0; e < n * n; ++e) M[e] = mk(M[e].x * c, M[e].y * c);
  }
  // store A
  double2 *a64 = reinterpret_cast<double2 *>(A64);
  float2 *a32 = reinterpret_cast<float2 *>(A32);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < r; ++c) {
      const int64_t idx = boff + herm_chunk(d, r, c) * k.Vh + i;
      a64[idx] = make_double2(M[r * n + c].x, M[r * n + c].y);
      a32[idx] = make_float2((float)M[r * n + c].x, (float)M[r * n + c].y);
    }
  for (int q = 0; q < d; ++q) {
    const int64_t idx = boff + (int64_t)q * k.Vh + i;
    a64[idx] = make_double2(M[2 * q * n + 2 * q].x, M[(2 * q + 1) * n + 2 * q + 1].x);
    a32[idx] = make_float2((float)M[2 * q * n + 2 * q].x, (float)M[(2 * q + 1) * n + 2 * q + 1].x);
  }
  // Gauss-Jordan
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Inv[r * n + c] = mk(r == c ? 1.0 : 0.0, 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = -1.0;
    for (int r = col; r < n; ++r) {
      const double v = M[r * n + col].x * M[r * n + col].x + M[r * n + col].y * M[r * n + col].y;
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        zd t = M[col * n + c];
        M[col * n + c] = M[piv * n + c];
        M[piv * n + c] = t;
        t = Inv[col * n + c];
        Inv[col * n + c] = Inv[piv * n + c];
        Inv[piv * n + c] = t;
      }
    const zd p = M[col * n + col];
    const double ib = 1.0 / (p.x * p.x + p.y * p.y);
    const zd pi = mk(p.x * ib, -p.y * ib);
    for (int c = 0; c < n; ++c) {
      M[col * n + c] = zmul2(M[col * n + c], pi);
      Inv[col * n + c] = zmul2(Inv[col * n + c], pi);
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const zd f = M[r * n + col];
      if (f.x == 0.0 && f.y == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        M[r * n + c] = M[r * n + c] - zmul2(f, M[col * n + c]);
        Inv[r * n + c] = Inv[r * n + c] - zmul2(f, Inv[col * n + c]);
      }
    }
  }
  double2 *i64 = reinterpret_cast<double2 *>(I64);
  float2 *i32 = reinterpret_cast<float2 *>(I32);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < r; ++c) {
      const int64_t idx = boff + herm_chunk(d, r, c) * k.Vh + i;
      i64[idx] = make_double2(Inv[r * n + c].x, Inv[r * n + c].y);
      i32[idx] = make_float2((float)Inv[r * n + c].x, (float)Inv[r * n + c].y);
    }
  for (int q = 0; q < d; ++q) {
    const int64_t idx = boff + (int64_t)q * k.Vh + i;
    i64[idx] = make_double2(Inv[2 * q * n + 2 * q].x, Inv[(2 * q + 1) * n + 2 * q + 1].x);
    i32[idx] = make_float2((float)Inv[2 * q * n + 2 * q].x, (float)Inv[(2 * q + 1) * n + 2 * q + 1].x);
  }
}

int hr_clover_prepare(hr_lattice *lat, double m0) {
  if (!lat->clover_term) return HR_ERR_STATE;
  if (lat->clover_cached && lat->clover_m0 == m0) return HR_OK;
  if (lat->clover_exp && 4.0 + m0 == 0.0) return HR_ERR_ARG;
  const int d = lat->d;
  const size_t n64 = (size_t)2 * 4 * d * d * (size_t)lat->Vh * 16u;
  for (int q = 0; q < 2; ++q) {
    if (!lat->clover_A[q]) HR_TRY(hr_dev_alloc(&lat->clover_A[q], q == 0 ? n64 : n64 / 2));
    if (!lat->clover_Ainv[q]) HR_TRY(hr_dev_alloc(&lat->clover_Ainv[q], q == 0 ? n64 : n64 / 2));
  }
  ClK k;
  memset(&k, 0, sizeof(k));
  k.d = d;
  k.Vh = lat->Vh;
  k.V = lat->V;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.T = lat->T;
  const int64_t nt = 4 * lat->Vh;
  clover_diag_kernel<<<(unsigned)((nt + 63) / 64), 64, 0, lat->stream>>>(
      lat->clover_A[0], lat->clover_A[1], lat->clover_Ainv[0], lat->clover_Ainv[1], lat->clover_term, k, m0, lat->clover_exp);
  HR_TRY(hr_check_launch("clover_diag_kernel"));
  lat->clover_m0 = m0;
  lat->clover_cached = 1;
  lat->clover_ff_ok = 0;
  return HR_OK;
}

extern "C" int hr_set_clover_exponential(hr_lattice *lat, int on) {
  if (!lat || (on != 0 && on != 1)) return HR_ERR_ARG;
  if (lat->clover_exp != on) lat->clover_cached = 0;
  lat->clover_exp = on;
  return HR_OK;
}

// export A or A^{-1} as [V][2][2d][2d] complex
__global__ void export_clover_kernel(double *out, const void *P64, ClK k) {
  const int64_t xl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (xl >= k.V) return;
  const int d = k.d, n = 2 * d;
  const int xx = (int)(xl % k.L);
  const int yy = (int)((xl / k.L) % k.L);
  const int zz = (int)((xl / ((int64_t)k.L * k.L)) % k.L);
  const int tt = (int)(xl / ((int64_t)k.L * k.L * k.L));
  const int par = (tt + xx + yy + zz) & 1;
  const int64_t i = cb_index(tt, xx, yy, zz, k.L, k.Lh);
  const double2 *src = reinterpret_cast<const double2 *>(P64);
  for (int b = 0; b < 2; ++b) {
    const int64_t boff = (int64_t)(par * 2 + b) * 2 * d * d * k.Vh;
    double *o = out + (xl * 2 + b) * 2 * n * n;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double re, im;
        if (r == c) {
          const double2 v = src[boff + herm_chunk(d, r, r) * k.Vh + i];
          re = (r & 1) ? v.y : v.x;
          im = 0.0;
        } else if (r > c) {
          const double2 v = src[boff + herm_chunk(d, r, c) * k.Vh + i];
          re = v.x;
          im = v.y;
        } else {
          const double2 v = src[boff + herm_chunk(d, c, r) * k.Vh + i];
          re = v.x;
          im = -v.y;
        }
        o[2 * (r * n + c)] = re;
        o[2 * (r * n + c) + 1] = im;
      }
  }
}

extern "C" int hr_export_clover(hr_lattice *lat, double *A_dev, double m0, int inverse) {
  if (!lat || !A_dev) return HR_ERR_ARG;
  if (!lat->have_links || lat->csw == 0.0) return HR_ERR_STATE;
  HR_TRY(hr_clover_prepare(lat, m0));
  ClK k;
  memset(&k, 0, sizeof(k));
  k.d = lat->d;
  k.Vh = lat->Vh;
  k.V = lat->V;
  k.L = lat->L;
  k.Lh = lat->L / 2;
  k.T = lat->T;
  export_clover_kernel<<<(unsigned)((lat->V + 127) / 128), 128, 0, lat->stream>>>(
      A_dev, inverse ? lat->clover_Ainv[0] : lat->clover_A[0], k);
  return hr_check_launch("export_clover_kernel");
}

// ------------------------------------------------------------------ dphi --
static const void *clover_ptr(const hr_lattice *lat, int prec, bool inverse, int parity) {
  const int q = prec == HR_F64 ? 0 : (prec == HR_FF ? 2 : 1);
  const void *base = inverse ? lat->clover_Ainv[q] : lat->clover_A[q];
  const size_t es = q == 1 ? 8 : 16;
  return reinterpret_cast<const char *>(base) + (size_t)parity * 4 * lat->d * lat->d * (size_t)lat->Vh * es;
}

int hr_dphi_impl(hr_lattice *lat, void *out, const void *in, int parity, double m0, double csw, int prec, int nrhs,
                 int dagger, cudaStream_t st) {
  return hr_dphi_impl_skip(lat, out, in, parity, m0, csw, prec, nrhs, dagger, st, nullptr, nullptr);
}

int hr_dphi_impl_skip(hr_lattice *lat, void *out, const void *in, int parity, double m0, double csw, int prec,
                      int nrhs, int dagger, cudaStream_t st, const double *skip_rr, const double *skip_stop) {
  const bool clover = csw != 0.0;
  if (prec == HR_FF) HR_TRY(hr_ff_prepare(lat, clover, m0, st));
  else if (clover) HR_TRY(hr_clover_prepare(lat, m0));
  const size_t fb = hr_spinor_field_bytes(lat->Vh, lat->d, prec);
  const double diag = 4.0 + m0;
  HopArgs a;
  memset(&a, 0, sizeof(a));
  a.links = lat->links[prec];
  a.rlinks = lat->rlinks[prec];
  a.dagger = dagger;
  a.nrhs = nrhs;
  a.skip_rr = skip_rr;
  a.skip_stop = skip_stop;
  if (parity == HR_FULL) {
    // out_p = A_pp in_p - 1/2 H in_q, both parities; rhs fields are [even | odd]
    for (int p = 0; p < 2; ++p) {
      a.out = reinterpret_cast<char *>(out) + (size_t)p * fb;
      a.in = reinterpret_cast<const char *>(in) + (size_t)(1 - p) * fb;
      a.self = reinterpret_cast<const char *>(in) + (size_t)p * fb;
      a.out_parity = p;
      a.mode = HOP_SELF;
      a.coef = -0.5;
      a.diag = diag;
      a.clover = clover ? clover_ptr(lat, prec, false, p) : nullptr;
      a.field_stride = 2 * fb;
      HR_TRY(hr_launch_hop(lat, prec, a, st));
      lat->hop_launches += 1;
    }
    return HR_OK;
  }
  const int p = parity, q = 1 - parity;
  HR_TRY(hr_ensure_tmp(lat, fb * (size_t)nrhs));
  // tmp_q = A_qq^{-1} D_qp in_p = A_qq^{-1} (-1/2 H in_p)
  a.out = lat->tmp;
  a.in = in;
  a.self = nullptr;
  a.out_parity = q;
  a.mode = HOP_SCALED;
  a.coef = clover ? -0.5 : -0.5 / diag;
  a.clover = clover ? clover_ptr(lat, prec, true, q) : nullptr;
  a.field_stride = fb;
  HR_TRY(hr_launch_hop(lat, prec, a, st));
  // out_p = A_pp in_p - D_pq tmp_q = A_pp in_p + 1/2 H tmp_q
  a.out = out;
  a.in = lat->tmp;
  a.self = in;
  a.out_parity = p;
  a.mode = HOP_SELF;
  a.coef = 0.5;
  a.diag = diag;
  a.clover = clover ? clover_ptr(lat, prec, false, p) : nullptr;
  a.pdl = 1;  // the site kernel may launch while the first hop finishes (it waits for its results)
  HR_TRY(hr_launch_hop(lat, prec, a, st));
  lat->hop_launches += 2;
  return HR_OK;
}

extern "C" int hr_dphi(hr_lattice *lat, void *out, const void *in, int parity, double m0, double csw, int prec,
                       int nrhs, int dagger) {
  if (!lat || !out || !in || nrhs < 1 || prec < HR_F64 || prec > HR_FF || parity < HR_EVEN || parity > HR_FULL)
    return HR_ERR_ARG;
  if (!lat->have_links) return HR_ERR_STATE;
  if (csw != lat->csw) return HR_ERR_ARG;
  if (out == in) return HR_ERR_ARG;
  if (prec == HR_FF && lat->dom) return HR_ERR_UNSUPPORTED;
  return hr_dphi_impl(lat, out, in, parity, m0, csw, prec, nrhs, dagger, lat->stream);
}
