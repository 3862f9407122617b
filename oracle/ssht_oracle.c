/*
 * ssht_oracle.c -- plain, slow FP64 CPU oracle for the exact spin spherical
 * harmonic transform of McEwen, "Fast, exact (but unstable) spin spherical
 * harmonic transforms" (arXiv:0807.4494).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Everything is IEEE double, built with -ffp-contract=off (no FMA contraction).
 * OpenMP only splits independent output rows across threads; it never changes
 * the order of any sum.
 *
 * Index conventions (API band-limit L is exclusive: 0 <= l < L):
 *   Lp = L - 1 (the paper's inclusive band-limit), N = 2 L - 1.
 *   Coefficients flm[b][l*l + l + m] as (re, im) pairs.
 *   Torus arrays T[b][m + Lp][m' + Lp] as (re, im) pairs, m, m' in [-Lp, Lp];
 *   the first index is the phi frequency m, the second the theta frequency m'.
 *   Full Wigner matrices of degree j = tj/2 are (tj+1) x (tj+1), row-major,
 *   entry (m, n) at [(j + m) * (tj + 1) + (j + n)].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------------------
 * Wigner d by the Risbo recursion (the paper uses it: Sec. 2.2, "we employ the
 * recursion formulae described in [Risbo 1996]"; the formulae are not written
 * out in the paper).  Restated from the mathematics: d^j is the coupling of
 * d^{j-1/2} with the spin-1/2 matrix d^{1/2}(beta) = [[p, -q], [q, p]],
 * p = cos(beta/2), q = sin(beta/2), projected on the maximal spin j.  With
 * a = j + m and b = j + n:
 *
 *   d^j_{mn} = (1/(2j)) [ sqrt(a b)           p d^{j-1/2}_{m-1/2, n-1/2}
 *                       - sqrt(a (2j-b))      q d^{j-1/2}_{m-1/2, n+1/2}
 *                       + sqrt((2j-a) b)      q d^{j-1/2}_{m+1/2, n-1/2}
 *                       + sqrt((2j-a)(2j-b))  p d^{j-1/2}_{m+1/2, n+1/2} ]
 *
 * where entries of d^{j-1/2} outside |index| <= j - 1/2 are zero.
 * ------------------------------------------------------------------------- */
static double prev_at(const double* prev, int dprev, int a, int b) {
  if (a < 0 || b < 0 || a >= dprev || b >= dprev) return 0.0;
  return prev[(size_t)a * dprev + b];
}

/* One half step: prev has degree (tj-1)/2 (dimension tj), out has degree tj/2
 * (dimension tj+1).  tj >= 1. */
static void risbo_half_step(int tj, const double* prev, double* out, double p, double q) {
  const int d = tj + 1;
  const double inv = 1.0 / (double)tj;
#pragma omp parallel for schedule(static)
  for (int a = 0; a < d; ++a) {
    for (int b = 0; b < d; ++b) {
      double x1 = prev_at(prev, tj, a - 1, b - 1);
      double x2 = prev_at(prev, tj, a - 1, b);
      double x3 = prev_at(prev, tj, a, b - 1);
      double x4 = prev_at(prev, tj, a, b);
      double t = sqrt((double)a * (double)b) * p * x1
               - sqrt((double)a * (double)(tj - b)) * q * x2
               + sqrt((double)(tj - a) * (double)b) * q * x3
               + sqrt((double)(tj - a) * (double)(tj - b)) * p * x4;
      out[(size_t)a * d + b] = t * inv;
    }
  }
}

/* Recursion state: two full matrices large enough for degree tjmax/2. */
typedef struct {
  double* cur;
  double* nxt;
  int tj; /* degree of cur is tj/2 */
  double p, q;
} risbo_t;

static int risbo_init(risbo_t* r, int tjmax, double beta) {
  size_t cap = (size_t)(tjmax + 1) * (size_t)(tjmax + 1);
  r->cur = (double*)calloc(cap, sizeof(double));
  r->nxt = (double*)calloc(cap, sizeof(double));
  if (!r->cur || !r->nxt) { free(r->cur); free(r->nxt); return -1; }
  r->cur[0] = 1.0; /* d^0 = [1] */
  r->tj = 0;
  r->p = cos(0.5 * beta);
  r->q = sin(0.5 * beta);
  return 0;
}

static void risbo_advance(risbo_t* r) {
  risbo_half_step(r->tj + 1, r->cur, r->nxt, r->p, r->q);
  double* t = r->cur; r->cur = r->nxt; r->nxt = t;
  r->tj += 1;
}

static void risbo_free(risbo_t* r) { free(r->cur); free(r->nxt); }

/* Full matrix d^{tj/2}(beta), written to out[(tj+1)^2]. */
int oracle_wigner_full(int tj, double beta, double* out) {
  if (tj < 0) return -1;
  risbo_t r;
  if (risbo_init(&r, tj, beta)) return -2;
  while (r.tj < tj) risbo_advance(&r);
  memcpy(out, r.cur, sizeof(double) * (size_t)(tj + 1) * (size_t)(tj + 1));
  risbo_free(&r);
  return 0;
}

/* Quadrant table of d^l(beta) for l = 0 .. L-1: entry (m', m), 0 <= m', m <= l,
 * at offset(l) + m' (l+1) + m with offset(l) = sum_{k<l} (k+1)^2.  At beta =
 * pi/2 this is the precomputed table of Sec. 4.1 (non-negative m and n). */
int oracle_delta_quadrant(int L, double beta, double* out) {
  if (L < 1) return -1;
  risbo_t r;
  if (risbo_init(&r, 2 * (L - 1), beta)) return -2;
  size_t off = 0;
  for (int l = 0; l < L; ++l) {
    while (r.tj < 2 * l) risbo_advance(&r);
    const int d = 2 * l + 1;
    for (int mp = 0; mp <= l; ++mp)
      for (int m = 0; m <= l; ++m)
        out[off + (size_t)mp * (l + 1) + m] = r.cur[(size_t)(l + mp) * d + (l + m)];
    off += (size_t)(l + 1) * (size_t)(l + 1);
  }
  risbo_free(&r);
  return 0;
}

/* i^k for integer k, as (re, im). */
static void ipow(int k, double* re, double* im) {
  int r = ((k % 4) + 4) % 4;
  *re = (r == 0) ? 1.0 : (r == 2) ? -1.0 : 0.0;
  *im = (r == 1) ? 1.0 : (r == 3) ? -1.0 : 0.0;
}

static double delta_at(const double* full, int l, int mp, int m) {
  return full[(size_t)(l + mp) * (2 * l + 1) + (l + m)];
}

/* ---------------------------------------------------------------------------
 * Eqn fourier_coeff (Sec. 3.1):
 *   F_{m m'} = (-1)^s i^{-(m+s)} sum_{l} sqrt((2l+1)/(4 pi))
 *              Delta^l_{m' m} Delta^l_{m', -s} sf_{lm},
 * summed over l >= max(|m|, |m'|, |s|) (terms with |m| > l or |m'| > l are zero
 * by the convention stated right after the equation).  Computed for every
 * m, m' in [-Lp, Lp] directly from the sum; no symmetry is used.
 * flm: [B][L*L][2]; F: [B][N][N][2].
 * ------------------------------------------------------------------------- */
int oracle_fourier_coeff(int L, int s, int B, const double* flm, double* F) {
  if (L < 1 || B < 1 || abs(s) >= L) return -1;
  const int Lp = L - 1, N = 2 * L - 1;
  const size_t fsz = (size_t)N * N * 2;
  memset(F, 0, sizeof(double) * fsz * B);
  risbo_t r;
  if (risbo_init(&r, 2 * Lp, ORACLE_PI / 2)) return -2;
  for (int l = 0; l < L; ++l) {
    while (r.tj < 2 * l) risbo_advance(&r);
    if (l < abs(s)) continue;
    const double cl = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI));
    for (int b = 0; b < B; ++b) {
      const double* a = flm + (size_t)b * L * L * 2;
      double* Fb = F + (size_t)b * fsz;
#pragma omp parallel for schedule(static)
      for (int m = -l; m <= l; ++m) {
        const double are = a[2 * ((size_t)l * l + l + m)];
        const double aim = a[2 * ((size_t)l * l + l + m) + 1];
        for (int mp = -l; mp <= l; ++mp) {
          const double k = cl * delta_at(r.cur, l, mp, m) * delta_at(r.cur, l, mp, -s);
          double* dst = Fb + 2 * ((size_t)(m + Lp) * N + (mp + Lp));
          dst[0] += k * are;
          dst[1] += k * aim;
        }
      }
    }
  }
  risbo_free(&r);
  /* the factor (-1)^s i^{-(m+s)} */
  const double sgn = (abs(s) % 2) ? -1.0 : 1.0;
  for (int b = 0; b < B; ++b) {
    double* Fb = F + (size_t)b * fsz;
    for (int m = -Lp; m <= Lp; ++m) {
      double pr, pi;
      ipow(-(m + s), &pr, &pi);
      pr *= sgn; pi *= sgn;
      for (int mp = -Lp; mp <= Lp; ++mp) {
        double* x = Fb + 2 * ((size_t)(m + Lp) * N + (mp + Lp));
        const double re = x[0], im = x[1];
        x[0] = pr * re - pi * im;
        x[1] = pr * im + pi * re;
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Harmonic projection of a torus array X (the forward contraction and the
 * adjoint contraction).  From eqn ssht_fwd with eqn ssh_wigner and eqn
 * wigner_sum_reln substituted (conjugated):
 *   sf_{lm} = (-1)^s i^{m+s} sqrt((2l+1)/(4 pi))
 *             sum_{m'=-l}^{l} Delta^l_{m' m} Delta^l_{m', -s} X_{m m'},
 * for l >= |s|, |m| <= l; zero for l < |s|.  The full m' sum is taken; no
 * symmetry is used.  X: [B][N][N][2]; flm: [B][L*L][2].
 * ------------------------------------------------------------------------- */
int oracle_harmonic_project(int L, int s, int B, const double* X, double* flm) {
  if (L < 1 || B < 1 || abs(s) >= L) return -1;
  const int Lp = L - 1, N = 2 * L - 1;
  const size_t fsz = (size_t)N * N * 2;
  memset(flm, 0, sizeof(double) * (size_t)B * L * L * 2);
  risbo_t r;
  if (risbo_init(&r, 2 * Lp, ORACLE_PI / 2)) return -2;
  const double sgn = (abs(s) % 2) ? -1.0 : 1.0;
  for (int l = 0; l < L; ++l) {
    while (r.tj < 2 * l) risbo_advance(&r);
    if (l < abs(s)) continue;
    const double cl = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI));
    for (int b = 0; b < B; ++b) {
      const double* Xb = X + (size_t)b * fsz;
      double* a = flm + (size_t)b * L * L * 2;
#pragma omp parallel for schedule(static)
      for (int m = -l; m <= l; ++m) {
        double sre = 0.0, sim = 0.0;
        for (int mp = -l; mp <= l; ++mp) {
          const double k = delta_at(r.cur, l, mp, m) * delta_at(r.cur, l, mp, -s);
          const double* x = Xb + 2 * ((size_t)(m + Lp) * N + (mp + Lp));
          sre += k * x[0];
          sim += k * x[1];
        }
        double pr, pi;
        ipow(m + s, &pr, &pi);
        pr *= sgn * cl; pi *= sgn * cl;
        a[2 * ((size_t)l * l + l + m)] = pr * sre - pi * sim;
        a[2 * ((size_t)l * l + l + m) + 1] = pr * sim + pi * sre;
      }
    }
  }
  risbo_free(&r);
  return 0;
}

/* ---------------------------------------------------------------------------
 * sin(theta) quadrature weight of the forward transform (derived from eqn
 * ssht_fwd with eqn sht_inv_fast; the paper itself inverts eqn fourier_coeff
 * instead, see oracle_triangular_forward):
 *   G_{m m'} = 2 pi sum_{m''=-Lp}^{Lp} F_{m m''} w(m'' - m'),
 *   w(p) = int_0^pi sin(theta) e^{i p theta} d theta
 *        = 2 / (1 - p^2) for even p,  +/- i pi / 2 for p = +/- 1,  0 otherwise.
 * Direct O(N^3) sum.  F, G: [B][N][N][2].
 * ------------------------------------------------------------------------- */
static void weight(int p, double* re, double* im) {
  if (p == 1) { *re = 0.0; *im = ORACLE_PI / 2; return; }
  if (p == -1) { *re = 0.0; *im = -ORACLE_PI / 2; return; }
  if (p % 2 == 0) { *re = 2.0 / (1.0 - (double)p * (double)p); *im = 0.0; return; }
  *re = 0.0; *im = 0.0;
}

int oracle_weight_conv(int L, int B, const double* F, double* G) {
  if (L < 1 || B < 1) return -1;
  const int Lp = L - 1, N = 2 * L - 1;
  const size_t fsz = (size_t)N * N * 2;
  for (int b = 0; b < B; ++b) {
    const double* Fb = F + (size_t)b * fsz;
    double* Gb = G + (size_t)b * fsz;
#pragma omp parallel for schedule(static)
    for (int m = -Lp; m <= Lp; ++m) {
      for (int mp = -Lp; mp <= Lp; ++mp) {
        double sre = 0.0, sim = 0.0;
        for (int mpp = -Lp; mpp <= Lp; ++mpp) {
          double wr, wi;
          weight(mpp - mp, &wr, &wi);
          if (wr == 0.0 && wi == 0.0) continue;
          const double* x = Fb + 2 * ((size_t)(m + Lp) * N + (mpp + Lp));
          sre += x[0] * wr - x[1] * wi;
          sim += x[0] * wi + x[1] * wr;
        }
        double* g = Gb + 2 * ((size_t)(m + Lp) * N + (mp + Lp));
        g[0] = 2.0 * ORACLE_PI * sre;
        g[1] = 2.0 * ORACLE_PI * sim;
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * The paper's forward transform (Sec. 3.4.2, eqn matrix_fwd): for each m,
 * solve the triangular system relating F_{m, m'} (m' >= 0) to sf_{lm} by back
 * substitution.  The matrix entries are eqn fourier_coeff's:
 *   D_m[m'][l] = (-1)^s i^{-(m+s)} sqrt((2l+1)/(4 pi)) Delta^l_{m' m} Delta^l_{m',-s},
 * nonzero for l >= m'.  Rows and columns run over [lmin, Lp], lmin = max(|m|, |s|)
 * (the diagonal entry Delta^l_{l m} Delta^l_{l,-s} never vanishes there; rows
 * below lmin are implied by the others).  For even m+s the even-extension
 * coefficients Fe are used, for odd m+s the odd-extension Fo (the case split
 * after eqn matrix_fwd).  Fe, Fo: [B][N][N][2]; flm: [B][L*L][2].
 * ------------------------------------------------------------------------- */
int oracle_triangular_forward(int L, int s, int B, const double* Fe, const double* Fo, double* flm) {
  if (L < 1 || B < 1 || abs(s) >= L) return -1;
  const int Lp = L - 1, N = 2 * L - 1;
  const size_t fsz = (size_t)N * N * 2;
  /* Keep the quadrant-free full Delta for all l (needed for each m column). */
  size_t total = 0;
  for (int l = 0; l < L; ++l) total += (size_t)(2 * l + 1) * (2 * l + 1);
  double* all = (double*)malloc(sizeof(double) * total);
  if (!all) return -2;
  size_t* off = (size_t*)malloc(sizeof(size_t) * L);
  risbo_t r;
  if (!off || risbo_init(&r, 2 * Lp, ORACLE_PI / 2)) { free(all); free(off); return -2; }
  size_t o = 0;
  for (int l = 0; l < L; ++l) {
    while (r.tj < 2 * l) risbo_advance(&r);
    off[l] = o;
    memcpy(all + o, r.cur, sizeof(double) * (size_t)(2 * l + 1) * (2 * l + 1));
    o += (size_t)(2 * l + 1) * (2 * l + 1);
  }
  risbo_free(&r);
  memset(flm, 0, sizeof(double) * (size_t)B * L * L * 2);
  const double sgn = (abs(s) % 2) ? -1.0 : 1.0;
  for (int b = 0; b < B; ++b) {
#pragma omp parallel for schedule(dynamic)
    for (int m = -Lp; m <= Lp; ++m) {
      const int lmin = abs(m) > abs(s) ? abs(m) : abs(s);
      const int par = ((m + s) % 2 + 2) % 2;
      const double* Fb = (par == 0 ? Fe : Fo) + (size_t)b * fsz;
      double* a = flm + (size_t)b * L * L * 2;
      double pr, pi;
      ipow(-(m + s), &pr, &pi);
      pr *= sgn; pi *= sgn;
      for (int l = Lp; l >= lmin; --l) {
        /* row m' = l: F_{m,l} = sum_{l' >= l} D[l][l'] f_{l'} */
        double rre = Fb[2 * ((size_t)(m + Lp) * N + (l + Lp))];
        double rim = Fb[2 * ((size_t)(m + Lp) * N + (l + Lp)) + 1];
        for (int lq = l + 1; lq <= Lp; ++lq) {
          const double* dq = all + off[lq];
          const double k = sqrt((2.0 * lq + 1.0) / (4.0 * ORACLE_PI)) * delta_at(dq, lq, l, m) * delta_at(dq, lq, l, -s);
          const double dre = pr * k, dim = pi * k;
          const double fre = a[2 * ((size_t)lq * lq + lq + m)], fim = a[2 * ((size_t)lq * lq + lq + m) + 1];
          rre -= dre * fre - dim * fim;
          rim -= dre * fim + dim * fre;
        }
        const double* dl = all + off[l];
        const double k = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI)) * delta_at(dl, l, l, m) * delta_at(dl, l, l, -s);
        const double dre = pr * k, dim = pi * k;
        const double den = dre * dre + dim * dim;
        a[2 * ((size_t)l * l + l + m)] = (rre * dre + rim * dim) / den;
        a[2 * ((size_t)l * l + l + m) + 1] = (rim * dre - rre * dim) / den;
      }
    }
  }
  free(all);
  free(off);
  return 0;
}

/* The matrix of eqn matrix_fwd for one m (rows m' = 0..Lp, columns l = 0..Lp),
 * as (re, im) pairs, for the conditioning experiment of Sec. 4.2. */
int oracle_triangular_matrix(int L, int s, int m, double* D) {
  if (L < 1 || abs(s) >= L || abs(m) >= L) return -1;
  const int Lp = L - 1;
  memset(D, 0, sizeof(double) * (size_t)L * L * 2);
  risbo_t r;
  if (risbo_init(&r, 2 * Lp, ORACLE_PI / 2)) return -2;
  const double sgn = (abs(s) % 2) ? -1.0 : 1.0;
  double pr, pi;
  ipow(-(m + s), &pr, &pi);
  pr *= sgn; pi *= sgn;
  for (int l = 0; l < L; ++l) {
    while (r.tj < 2 * l) risbo_advance(&r);
    if (l < abs(s) || l < abs(m)) continue;
    const double cl = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI));
    for (int mp = 0; mp <= l; ++mp) {
      const double k = cl * delta_at(r.cur, l, mp, m) * delta_at(r.cur, l, mp, -s);
      D[2 * ((size_t)mp * L + l)] = pr * k;
      D[2 * ((size_t)mp * L + l) + 1] = pi * k;
    }
  }
  risbo_free(&r);
  (void)Lp;
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
