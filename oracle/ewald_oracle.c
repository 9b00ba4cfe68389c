/*
 * Exact Ewald decomposition of the Stokes potentials, plain FP64 C (OpenMP over targets).
 *
 * TEST INFRASTRUCTURE ONLY: the oracle the CUDA path is checked against. Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may load it. It
 * shares no code, header, table or helper with the library under paper_2210_01255_gb300/.
 *
 * What it computes (Bagge & Tornberg 2022, Sec. 2):
 *   u = u^R (Eq. real-space-potential-Dp, kernels Eqs. stokeslet-real .. stresslet-real)
 *     + u^F (3P: Eq. fourier-space-potential-3p summed directly over |k| <= kmax;
 *            2P: Eqs. 2p-evaluated-integrals-nonzero / -k0 with the App. A tensors;
 *            1P: Eqs. 1p-evaluated-integrals-nonzero / -k0 with the App. B tensors)
 *     + u^{k=0} (3P stresslet only, Eq. k0-stresslet-3p)
 *     + u^self (Eq. self-term), or, for D = 0, the direct sum of Eq. periodic-potential.
 * The caller chooses xi, rc and kmax so that the neglected tails are below rounding.
 *
 * Every function is pinned by tests/test_oracle_ewald.py against something outside itself
 * (xi-independence of the total, quadrature of the App. A/B defining integrals, brute-force
 * image sums, the stresslet integral identity, hand-computed kernel values); nothing here is
 * tuned for speed beyond evaluating a complex exponential per term.
 */
#include "ewald_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
static const double SQRTPI = 1.77245385090551602729816748334;
static const double EULER_GAMMA = 0.57721566490153286060651209008240;

/* ---------------------------------------------------------------- small tensor helpers */

static int levi(int j, int l, int m) {
  /* Levi-Civita symbol epsilon_{jlm}, indices 0..2 */
  if (j == l || l == m || j == m) return 0;
  return ((j == 0 && l == 1) || (j == 1 && l == 2) || (j == 2 && l == 0)) ? 1 : -1;
}
static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

static int ncomp_in(int kernel) { return kernel == ORC_STRESSLET ? 6 : 3; }

/* u_j += sum_l G_jl f_l (S, Omega) or u_j += sum_lm T_jlm q_l nu_m (T), Eq. tensor-products.
 * G is given as 9 (or 27) real numbers. */
static void contract_add(int kernel, const double* G, const double* f, double* u) {
  if (kernel == ORC_STRESSLET) {
    const double* q = f;
    const double* nu = f + 3;
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) u[j] += G[j * 9 + l * 3 + m] * q[l] * nu[m];
  } else {
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) u[j] += G[j * 3 + l] * f[l];
  }
}

/* Complex contraction: v_j = sum G_j.. f_.. for complex G (re, im) and real f. */
static void contract_c(int kernel, const double* Gre, const double* Gim, const double* f,
                       double complex v[3]) {
  v[0] = v[1] = v[2] = 0;
  if (kernel == ORC_STRESSLET) {
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          int i = j * 9 + l * 3 + m;
          v[j] += (Gre[i] + I * Gim[i]) * f[l] * f[3 + m];
        }
  } else {
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) v[j] += (Gre[j * 3 + l] + I * Gim[j * 3 + l]) * f[l];
  }
}

/* ------------------------------------------------------------- real-space kernels */

/* Eq. (stokeslet-real) */
static void stokeslet_real(double xi, const double* r, double* G) {
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rr = sqrt(r2);
  double e = exp(-xi * xi * r2);
  double c = erfc(xi * rr) / rr + 2.0 * xi * e / SQRTPI;
  for (int j = 0; j < 3; ++j)
    for (int l = 0; l < 3; ++l)
      G[j * 3 + l] = (kd(j, l) + r[j] * r[l] / r2) * c - kd(j, l) * 4.0 * xi * e / SQRTPI;
}

/* Eq. (rotlet-real) */
static void rotlet_real(double xi, const double* r, double* G) {
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rr = sqrt(r2);
  double e = exp(-xi * xi * r2);
  double c = erfc(xi * rr) / rr + 2.0 * xi * e / SQRTPI;
  for (int j = 0; j < 3; ++j)
    for (int l = 0; l < 3; ++l) {
      double s = 0;
      for (int m = 0; m < 3; ++m) s += levi(j, l, m) * r[m] / r2;
      G[j * 3 + l] = s * c;
    }
}

/* Eq. (stresslet-real) */
static void stresslet_real(double xi, const double* r, double* T) {
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rr = sqrt(r2);
  double e = exp(-xi * xi * r2);
  double a = 3.0 * erfc(xi * rr) / rr + (3.0 + 2.0 * xi * xi * r2) * 2.0 * xi * e / SQRTPI;
  double b = 4.0 * xi * xi * xi * e / SQRTPI;
  for (int j = 0; j < 3; ++j)
    for (int l = 0; l < 3; ++l)
      for (int m = 0; m < 3; ++m)
        T[j * 9 + l * 3 + m] = -2.0 * r[j] * r[l] * r[m] / (r2 * r2) * a +
                               (kd(j, l) * r[m] + kd(m, j) * r[l] + kd(l, m) * r[j]) * b;
}

/* Eq. (stokes-kernels): the unsplit kernels, used by the free-space direct sum. */
static void kernel_full(int kernel, const double* r, double* G) {
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double rr = sqrt(r2);
  double r3 = r2 * rr;
  if (kernel == ORC_STOKESLET) {
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) G[j * 3 + l] = kd(j, l) / rr + r[j] * r[l] / r3;
  } else if (kernel == ORC_ROTLET) {
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) {
        double s = 0;
        for (int m = 0; m < 3; ++m) s += levi(j, l, m) * r[m];
        G[j * 3 + l] = s / r3;
      }
  } else {
    double r5 = r3 * r2;
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) G[j * 9 + l * 3 + m] = -6.0 * r[j] * r[l] * r[m] / r5;
  }
}

static int valid_kernel(int kernel) {
  return kernel == ORC_STOKESLET || kernel == ORC_ROTLET || kernel == ORC_STRESSLET;
}

/* ------------------------------------------------------------------ real-space sum */

int orc_real(int D, const double L[3], double xi, double rc, int kernel, long N,
             const double* x, const double* f, long Nt, const double* t, double* u) {
  if (D < 0 || D > 3 || !valid_kernel(kernel) || !(xi > 0) || !(rc > 0) || N < 0) return -1;
  const int star = (t == NULL);
  if (star) { t = x; Nt = N; }
  const int nc = ncomp_in(kernel);
  int pmax[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) pmax[d] = (int)floor(rc / L[d]) + 1;
#pragma omp parallel for schedule(dynamic, 4)
  for (long m = 0; m < Nt; ++m) {
    double acc[3] = {0, 0, 0};
    double G[27];
    for (long n = 0; n < N; ++n) {
      for (int p0 = -pmax[0]; p0 <= pmax[0]; ++p0)
        for (int p1 = -pmax[1]; p1 <= pmax[1]; ++p1)
          for (int p2 = -pmax[2]; p2 <= pmax[2]; ++p2) {
            double r[3] = {t[m * 3 + 0] - x[n * 3 + 0] + p0 * L[0],
                           t[m * 3 + 1] - x[n * 3 + 1] + p1 * L[1],
                           t[m * 3 + 2] - x[n * 3 + 2] + p2 * L[2]};
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (r2 == 0.0) continue; /* omitted term of the star sum */
            if (r2 >= rc * rc) continue;
            if (kernel == ORC_STOKESLET) stokeslet_real(xi, r, G);
            else if (kernel == ORC_ROTLET) rotlet_real(xi, r, G);
            else stresslet_real(xi, r, G);
            contract_add(kernel, G, f + n * nc, acc);
          }
    }
    for (int j = 0; j < 3; ++j) u[m * 3 + j] += acc[j];
  }
  return 0;
}

/* ----------------------------------------------------- Fourier-space kernel, Eq. 3-D */

int orc_GF(int kernel, double xi, const double* k, double* re, double* im) {
  if (!valid_kernel(kernel)) return -1;
  double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  if (!(k2 > 0)) return -1;
  double gE = exp(-k2 / (4.0 * xi * xi));        /* Eq. (ewald-screening) */
  double gH = gE * (1.0 + k2 / (4.0 * xi * xi)); /* Eq. (hasimoto-screening) */
  double Bh = -8.0 * M_PI / (k2 * k2);           /* B^(k) = -8 pi / k^4 */
  double Hh = 4.0 * M_PI / k2;                   /* H^(k) = 4 pi / k^2 */
  if (kernel == ORC_STOKESLET) {                 /* Eq. (stokeslet-fourier) */
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) {
        re[j * 3 + l] = (-kd(j, l) * k2 + k[j] * k[l]) * Bh * gH;
        im[j * 3 + l] = 0.0;
      }
  } else if (kernel == ORC_ROTLET) { /* Eq. (rotlet-fourier): -eps_jlm i k_m H^ gE */
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) {
        double s = 0;
        for (int m = 0; m < 3; ++m) s += levi(j, l, m) * k[m];
        re[j * 3 + l] = 0.0;
        im[j * 3 + l] = -s * Hh * gE;
      }
  } else { /* Eq. (stresslet-fourier) */
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          double K = -(kd(j, l) * k[m] + kd(m, j) * k[l] + kd(l, m) * k[j]) * k2 +
                     2.0 * k[j] * k[l] * k[m]; /* imaginary part of K^T */
          re[j * 9 + l * 3 + m] = 0.0;
          im[j * 9 + l * 3 + m] = K * Bh * gH;
        }
  }
  return 0;
}

/* ------------------------------------------------------------ triply periodic, k != 0 */

int orc_fourier3p(const double L[3], double xi, double kmax, int kernel, long N,
                  const double* x, const double* f, long Nt, const double* t, double* u) {
  if (!valid_kernel(kernel) || !(xi > 0) || !(kmax > 0)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  const int nc = ncomp_in(kernel);
  int K[3];
  for (int d = 0; d < 3; ++d) K[d] = (int)floor(kmax * L[d] / (2.0 * M_PI));
  /* enumerate the modes */
  long nmax = (long)(2 * K[0] + 1) * (2 * K[1] + 1) * (2 * K[2] + 1);
  double* kv = (double*)malloc(sizeof(double) * 3 * nmax);
  long nk = 0;
  for (int a = -K[0]; a <= K[0]; ++a)
    for (int b = -K[1]; b <= K[1]; ++b)
      for (int c = -K[2]; c <= K[2]; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        double k[3] = {2.0 * M_PI * a / L[0], 2.0 * M_PI * b / L[1], 2.0 * M_PI * c / L[2]};
        if (k[0] * k[0] + k[1] * k[1] + k[2] * k[2] > kmax * kmax) continue;
        kv[nk * 3 + 0] = k[0];
        kv[nk * 3 + 1] = k[1];
        kv[nk * 3 + 2] = k[2];
        ++nk;
      }
  /* V_j(k) = sum_n G^F(k) . f_n exp(-i k . x_n) */
  double complex* V = (double complex*)malloc(sizeof(double complex) * 3 * (nk > 0 ? nk : 1));
#pragma omp parallel for schedule(dynamic, 16)
  for (long q = 0; q < nk; ++q) {
    double Gre[27], Gim[27];
    orc_GF(kernel, xi, kv + q * 3, Gre, Gim);
    double complex acc[3] = {0, 0, 0};
    for (long n = 0; n < N; ++n) {
      const double* xn = x + n * 3;
      double ph = -(kv[q * 3] * xn[0] + kv[q * 3 + 1] * xn[1] + kv[q * 3 + 2] * xn[2]);
      double complex e = cexp(I * ph);
      double complex v[3];
      contract_c(kernel, Gre, Gim, f + n * nc, v);
      for (int j = 0; j < 3; ++j) acc[j] += v[j] * e;
    }
    for (int j = 0; j < 3; ++j) V[q * 3 + j] = acc[j];
  }
  const double vol = L[0] * L[1] * L[2];
#pragma omp parallel for schedule(dynamic, 16)
  for (long m = 0; m < Nt; ++m) {
    const double* xm = t + m * 3;
    double acc[3] = {0, 0, 0};
    for (long q = 0; q < nk; ++q) {
      double ph = kv[q * 3] * xm[0] + kv[q * 3 + 1] * xm[1] + kv[q * 3 + 2] * xm[2];
      double complex e = cexp(I * ph);
      for (int j = 0; j < 3; ++j) acc[j] += creal(V[q * 3 + j] * e);
    }
    for (int j = 0; j < 3; ++j) u[m * 3 + j] += acc[j] / vol;
  }
  free(kv);
  free(V);
  return 0;
}

int orc_k0_stresslet3p(const double L[3], long N, const double* x, const double* f,
                       long Nt, const double* t, double* u) {
  if (t == NULL) { t = x; Nt = N; }
  const double vol = L[0] * L[1] * L[2];
  for (long m = 0; m < Nt; ++m) {
    double acc[3] = {0, 0, 0};
    for (long n = 0; n < N; ++n) {
      const double* q = f + n * 6;
      const double* nu = q + 3;
      double qn = q[0] * nu[0] + q[1] * nu[1] + q[2] * nu[2];
      for (int j = 0; j < 3; ++j) acc[j] += (t[m * 3 + j] - x[n * 3 + j]) * qn;
    }
    for (int j = 0; j < 3; ++j) u[m * 3 + j] += -8.0 * M_PI / vol * acc[j];
  }
  return 0;
}

/* ------------------------------------------------------- App. A: doubly periodic tensors */

/* e^{+/- alpha r3} erfc(alpha/(2 xi) +/- xi r3), guarded against overflow of the exponential */
static double theta(double s, double alpha, double xi, double r3) {
  double y = alpha / (2.0 * xi) + s * xi * r3;
  double e = erfc(y);
  if (e == 0.0) return 0.0;
  double a = s * alpha * r3;
  if (a < 700.0) return exp(a) * e;
  return exp(a + log(e));
}

/* symmetric 3-tensor: entries in the order 111,112,113,122,123,133,222,223,233,333 */
static int sym_index(int j, int l, int m) {
  int a = j, b = l, c = m, s;
  if (a > b) { s = a; a = b; b = s; }
  if (b > c) { s = b; b = c; c = s; }
  if (a > b) { s = a; a = b; b = s; }
  static const int tab[3][3][3] = {
      {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}}, {{1, 3, 4}, {3, 6, 7}, {4, 7, 8}},
      {{2, 4, 5}, {4, 7, 8}, {5, 8, 9}}};
  return tab[a][b][c];
}
static void sym_fill(const double complex* q10, double* re, double* im) {
  for (int j = 0; j < 3; ++j)
    for (int l = 0; l < 3; ++l)
      for (int m = 0; m < 3; ++m) {
        double complex v = q10[sym_index(j, l, m)];
        re[j * 9 + l * 3 + m] = creal(v);
        im[j * 9 + l * 3 + m] = cimag(v);
      }
}

/* Q^{2P}(k1,k2,r3;xi), Eqs. (2p-rotlet-Q), (2p-stokeslet-Q), (2p-stresslet-Q),
 * auxiliary variables Eq. (2p-aux). */
int orc_Q2p(int kernel, double xi, double k1, double k2, double r3, double* re, double* im) {
  if (!valid_kernel(kernel)) return -1;
  double alpha = sqrt(k1 * k1 + k2 * k2);
  if (!(alpha > 0)) return -1;
  double kt1 = k1 / alpha, kt2 = k2 / alpha;
  double thp = theta(+1.0, alpha, xi, r3);
  double thm = theta(-1.0, alpha, xi, r3);
  double bp = thp + thm, bm = thp - thm;
  double lam = 2.0 / (SQRTPI * xi) * exp(-alpha * alpha / (4.0 * xi * xi)) * exp(-xi * xi * r3 * r3);
  double Lam = lam + bp / alpha - r3 * bm;
  double Psi = -bp / alpha - r3 * bm;
  double complex Q[27];
  if (kernel == ORC_ROTLET) {
    double complex q[9] = {0,        -bm,       I * kt2 * bp, bm, 0, -I * kt1 * bp,
                           -I * kt2 * bp, I * kt1 * bp, 0};
    for (int i = 0; i < 9; ++i) Q[i] = M_PI * q[i];
    for (int i = 0; i < 9; ++i) { re[i] = creal(Q[i]); im[i] = cimag(Q[i]); }
  } else if (kernel == ORC_STOKESLET) {
    double complex q[9] = {kt2 * kt2 * Lam - Psi, -kt1 * kt2 * Lam,       -I * kt1 * r3 * bp,
                           -kt1 * kt2 * Lam,      kt1 * kt1 * Lam - Psi,  -I * kt2 * r3 * bp,
                           -I * kt1 * r3 * bp,    -I * kt2 * r3 * bp,     Lam};
    for (int i = 0; i < 9; ++i) Q[i] = M_PI * q[i];
    for (int i = 0; i < 9; ++i) { re[i] = creal(Q[i]); im[i] = cimag(Q[i]); }
  } else {
    double complex q[10];
    double x2 = xi * xi;
    q[0] = I * M_PI * kt1 * alpha * ((2.0 * kt2 * kt2 + 1.0) * Lam - 3.0 * Psi); /* 111 */
    q[1] = I * M_PI * kt2 * alpha * ((2.0 * kt2 * kt2 - 1.0) * Lam - Psi);       /* 112 */
    /* Entries 113, 223, 333: the printed App. A forms carry a factor 2 on both beta terms;
     * applying K^T_{jlm} to Q^{B,2P} = -pi Lambda / alpha^2 (Eq. 2p-QB-result) with the
     * derivative relations stated under Eq. (2p-stokeslet-Q) gives the forms below, which
     * agree with quadrature of the defining integral. */
    q[2] = -2.0 * M_PI * (x2 * r3 * lam - kt1 * kt1 * r3 * alpha * bp - bm);    /* 113 */
    q[3] = I * M_PI * kt1 * alpha * ((2.0 * kt1 * kt1 - 1.0) * Lam - Psi);       /* 122 */
    q[4] = 2.0 * M_PI * kt1 * kt2 * r3 * alpha * bp;                              /* 123 */
    q[5] = I * M_PI * kt1 * alpha * (Lam + Psi);                                  /* 133 */
    q[6] = I * M_PI * kt2 * alpha * ((2.0 * kt1 * kt1 + 1.0) * Lam - 3.0 * Psi); /* 222 */
    q[7] = -2.0 * M_PI * (x2 * r3 * lam - kt2 * kt2 * r3 * alpha * bp - bm);    /* 223 */
    q[8] = I * M_PI * kt2 * alpha * (Lam + Psi);                                  /* 233 */
    q[9] = -2.0 * M_PI * (x2 * r3 * lam + r3 * alpha * bp - bm);                /* 333 */
    sym_fill(q, re, im);
  }
  return 0;
}

/* Q^{2P,(0)}(r3;xi), Eqs. (2p-rotlet-Q0), (2p-stokeslet-Q0), (2p-stresslet-Q0). Real. */
int orc_Q2p0(int kernel, double xi, double r3, double* re) {
  if (!valid_kernel(kernel)) return -1;
  double ef = erf(xi * r3);
  double g = exp(-xi * xi * r3 * r3);
  if (kernel == ORC_ROTLET) {
    double c = 2.0 * M_PI * ef;
    double q[9] = {0, c, 0, -c, 0, 0, 0, 0, 0};
    memcpy(re, q, sizeof q);
  } else if (kernel == ORC_STOKESLET) {
    double c = -2.0 * M_PI * (2.0 * r3 * ef + g / (SQRTPI * xi));
    double q[9] = {c, 0, 0, 0, c, 0, 0, 0, 0};
    memcpy(re, q, sizeof q);
  } else {
    double c = -4.0 * M_PI * (ef + xi * r3 / SQRTPI * g);
    /* C_{1lm}: (1,3),(3,1); C_{2lm}: (2,3),(3,2); C_{3lm}: identity */
    memset(re, 0, 27 * sizeof(double));
    re[0 * 9 + 0 * 3 + 2] = c;
    re[0 * 9 + 2 * 3 + 0] = c;
    re[1 * 9 + 1 * 3 + 2] = c;
    re[1 * 9 + 2 * 3 + 1] = c;
    re[2 * 9 + 0 * 3 + 0] = c;
    re[2 * 9 + 1 * 3 + 1] = c;
    re[2 * 9 + 2 * 3 + 2] = c;
  }
  return 0;
}

int orc_fourier2p(const double L[3], double xi, double kmax, int kernel, long N,
                  const double* x, const double* f, long Nt, const double* t, double* u) {
  if (!valid_kernel(kernel) || !(xi > 0) || !(kmax > 0)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  const int nc = ncomp_in(kernel);
  int K1 = (int)floor(kmax * L[0] / (2.0 * M_PI));
  int K2 = (int)floor(kmax * L[1] / (2.0 * M_PI));
  long nmax = (long)(2 * K1 + 1) * (2 * K2 + 1);
  double* kv = (double*)malloc(sizeof(double) * 2 * nmax);
  long nk = 0;
  for (int a = -K1; a <= K1; ++a)
    for (int b = -K2; b <= K2; ++b) {
      if (a == 0 && b == 0) continue;
      double k1 = 2.0 * M_PI * a / L[0], k2 = 2.0 * M_PI * b / L[1];
      if (k1 * k1 + k2 * k2 > kmax * kmax) continue;
      kv[nk * 2] = k1;
      kv[nk * 2 + 1] = k2;
      ++nk;
    }
  const double area = L[0] * L[1];
#pragma omp parallel for schedule(dynamic, 1)
  for (long m = 0; m < Nt; ++m) {
    double acc[3] = {0, 0, 0};
    double Qre[27], Qim[27];
    for (long n = 0; n < N; ++n) {
      const double* fn = f + n * nc;
      double dx = t[m * 3 + 0] - x[n * 3 + 0];
      double dy = t[m * 3 + 1] - x[n * 3 + 1];
      double r3 = t[m * 3 + 2] - x[n * 3 + 2];
      for (long q = 0; q < nk; ++q) {
        orc_Q2p(kernel, xi, kv[q * 2], kv[q * 2 + 1], r3, Qre, Qim);
        double complex v[3];
        contract_c(kernel, Qre, Qim, fn, v);
        double complex e = cexp(I * (kv[q * 2] * dx + kv[q * 2 + 1] * dy));
        for (int j = 0; j < 3; ++j) acc[j] += creal(v[j] * e);
      }
      orc_Q2p0(kernel, xi, r3, Qre);
      contract_add(kernel, Qre, fn, acc);
    }
    for (int j = 0; j < 3; ++j) u[m * 3 + j] += acc[j] / area;
  }
  free(kv);
  return 0;
}

/* ---------------------------------------------------------- special functions, App. B */

/* E_1 by its power series (x <= 1) or continued fraction (x > 1); E_n by the recurrence
 * E_{n+1}(x) = (e^{-x} - x E_n(x)) / n; E_0(x) = e^{-x} / x. */
static double expint1(double x) {
  if (x <= 1.0) {
    double sum = 0.0, term = 1.0;
    for (int k = 1; k < 200; ++k) {
      term *= -x / k;                 /* (-x)^k / k! */
      double add = -term / k;         /* (-1)^{k+1} x^k / (k k!) */
      sum += add;
      if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return -EULER_GAMMA - log(x) + sum;
  }
  /* E_1(x) = e^{-x} / g with g = (x+1) - 1/((x+3) - 4/((x+5) - 9/(...))), modified Lentz */
  const double tiny = 1e-300;
  double fval = x + 1.0, C = fval, Dd = 0.0;
  for (int j = 1; j < 10000; ++j) {
    double a = -(double)j * j, b = x + 1.0 + 2.0 * j;
    Dd = b + a * Dd;
    if (fabs(Dd) < tiny) Dd = tiny;
    C = b + a / C;
    if (fabs(C) < tiny) C = tiny;
    Dd = 1.0 / Dd;
    double delta = C * Dd;
    fval *= delta;
    if (fabs(delta - 1.0) < 1e-17) break;
  }
  return exp(-x) / fval;
}

double orc_En(int n, double x) {
  if (!(x > 0) || n < 0) return NAN;
  if (n == 0) return exp(-x) / x;
  double e = expint1(x);
  for (int k = 1; k < n; ++k) e = (exp(-x) - x * e) / k;
  return e;
}

/* Gauss-Legendre nodes on [-1,1] by Newton's method on P_n. */
#define GL_N 24
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;
static void legendre(double z, double* p, double* dp) {
  double p0 = 1.0, p1 = 0.0;
  for (int j = 1; j <= GL_N; ++j) {
    double p2 = p1;
    p1 = p0;
    p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
  }
  *p = p0;
  *dp = GL_N * (z * p0 - p1) / (z * z - 1.0);
}
static void gl_init(void) {
  for (int i = 0; i < GL_N; ++i) {
    double z = cos(M_PI * (i + 0.75) / (GL_N + 0.5)), p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre(z, &p, &dp);
    gl_x[i] = z;
    gl_w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  gl_ready = 1;
}

/* Integrand of Eq. (Knu-def) after t = e^s:  exp(-a e^s - b e^{-s} - nu s), for
 * nu = -1, 0, 1, 2 at once. */
static void knu_integrand(double a, double b, double s, double out[4]) {
  double base = -a * exp(s) - b * exp(-s);
  out[0] = exp(base + s);
  out[1] = exp(base);
  out[2] = exp(base - s);
  out[3] = exp(base - 2.0 * s);
}
static void gl_panel(double a, double b, double lo, double hi, double out[4]) {
  double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
  out[0] = out[1] = out[2] = out[3] = 0;
  for (int i = 0; i < GL_N; ++i) {
    double v[4];
    knu_integrand(a, b, c + h * gl_x[i], v);
    for (int j = 0; j < 4; ++j) out[j] += gl_w[i] * h * v[j];
  }
}
/* Adaptive bisection: accept a panel when its two halves agree with the whole to 1e-14
 * relative, or to 1e-18 of the whole integral's scale; at most 20 levels deep. */
static void knu_adapt(double a, double b, double lo, double hi, const double whole[4],
                      const double scale[4], int depth, double out[4]) {
  double m = 0.5 * (lo + hi), l4[4], r4[4];
  gl_panel(a, b, lo, m, l4);
  gl_panel(a, b, m, hi, r4);
  int ok = 1;
  for (int j = 0; j < 4; ++j) {
    double both = l4[j] + r4[j];
    double err = fabs(both - whole[j]);
    if (err > 1e-14 * fabs(both) && err > 1e-18 * scale[j]) ok = 0;
  }
  if (ok || depth >= 20) {
    for (int j = 0; j < 4; ++j) out[j] = l4[j] + r4[j];
    return;
  }
  double lo4[4], hi4[4];
  knu_adapt(a, b, lo, m, l4, scale, depth + 1, lo4);
  knu_adapt(a, b, m, hi, r4, scale, depth + 1, hi4);
  for (int j = 0; j < 4; ++j) out[j] = lo4[j] + hi4[j];
}

/* K_nu(a,b) for nu = -1,0,1,2: out[nu+1]. Integration over s in [0, s_max], where the
 * log-integrand (concave in s) has dropped 60 below its maximum. */
static void knu_all(double a, double b, double out[4]) {
  if (!gl_ready) {
#pragma omp critical(gl_init_once)
    if (!gl_ready) gl_init();
  }
  /* peak of -a e^s - b e^{-s} + s (the nu = -1 member, the widest on the right) */
  double s0 = 0.0;
  {
    double lo = 0.0, hi = 1.0;
    while (-a * exp(hi) + b * exp(-hi) + 1.0 > 0) hi *= 2.0;
    if (-a * exp(lo) + b * exp(-lo) + 1.0 > 0) {
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (-a * exp(mid) + b * exp(-mid) + 1.0 > 0) lo = mid; else hi = mid;
      }
      s0 = 0.5 * (lo + hi);
    }
  }
  double fpk = -a * exp(s0) - b * exp(-s0) + s0;
  double smax = s0 + 1.0;
  while (-a * exp(smax) - b * exp(-smax) + smax > fpk - 60.0) smax += 1.0;
  /* panels of width <= 1 */
  int np = (int)ceil(smax);
  if (np > 64) np = 64;
  double wholes[64][4], scale[4] = {0, 0, 0, 0};
  for (int p = 0; p < np; ++p) {
    gl_panel(a, b, smax * p / np, smax * (p + 1) / np, wholes[p]);
    for (int j = 0; j < 4; ++j) scale[j] += fabs(wholes[p][j]);
  }
  double acc[4] = {0, 0, 0, 0};
  for (int p = 0; p < np; ++p) {
    double part[4];
    knu_adapt(a, b, smax * p / np, smax * (p + 1) / np, wholes[p], scale, 0, part);
    for (int j = 0; j < 4; ++j) acc[j] += part[j];
  }
  for (int j = 0; j < 4; ++j) out[j] = acc[j];
}

double orc_Knu(int nu, double a, double b) {
  if (nu < -1 || nu > 2 || !(a > 0) || b < 0) return NAN;
  double out[4];
  knu_all(a, b, out);
  return out[nu + 1];
}

/* Q^{1P}(k1,r2,r3;xi), Eqs. (1p-rotlet-Q), (1p-stokeslet-Q), (1p-stresslet-Q), with
 * U, V from Eq. (1p-aux). Kn[0..3] = K_{-1}, K_0, K_1, K_2 at (U,V). */
static void q1p_from_k(int kernel, double xi, double k1, double r2, double r3,
                       const double* Kn, double* re, double* im) {
  double U = k1 * k1 / (4.0 * xi * xi);
  double V = xi * xi * (r2 * r2 + r3 * r3);
  double Km1 = Kn[0], K0 = Kn[1], K1 = Kn[2], K2 = Kn[3];
  double x2 = xi * xi;
  if (kernel == ORC_ROTLET) {
    double complex q[9] = {0,
                           2.0 * x2 * r3 * K1,
                           -2.0 * x2 * r2 * K1,
                           -2.0 * x2 * r3 * K1,
                           0,
                           -I * k1 * K0,
                           2.0 * x2 * r2 * K1,
                           I * k1 * K0,
                           0};
    for (int i = 0; i < 9; ++i) { re[i] = creal(q[i]); im[i] = cimag(q[i]); }
  } else if (kernel == ORC_STOKESLET) {
    double complex q[9] = {2.0 * K0 - 2.0 * V * K1,
                           -I * k1 * r2 * K0,
                           -I * k1 * r3 * K0,
                           -I * k1 * r2 * K0,
                           2.0 * U * Km1 + K0 - 2.0 * x2 * r3 * r3 * K1,
                           2.0 * x2 * r2 * r3 * K1,
                           -I * k1 * r3 * K0,
                           2.0 * x2 * r2 * r3 * K1,
                           2.0 * U * Km1 + K0 - 2.0 * x2 * r2 * r2 * K1};
    for (int i = 0; i < 9; ++i) { re[i] = creal(q[i]); im[i] = cimag(q[i]); }
  } else {
    double complex q[10];
    q[0] = 2.0 * I * k1 * (U * Km1 + 3.0 * K0 - 3.0 * V * K1);                    /* 111 */
    q[1] = 4.0 * x2 * r2 * (U * K0 - 2.0 * K1 + V * K2);                         /* 112 */
    q[2] = 4.0 * x2 * r3 * (U * K0 - 2.0 * K1 + V * K2);                         /* 113 */
    q[3] = 2.0 * I * k1 * (U * Km1 + x2 * (r2 * r2 - r3 * r3) * K1);             /* 122 */
    q[4] = 4.0 * x2 * I * k1 * r2 * r3 * K1;                                     /* 123 */
    q[5] = 2.0 * I * k1 * (U * Km1 + x2 * (r3 * r3 - r2 * r2) * K1);             /* 133 */
    q[6] = -4.0 * x2 * r2 * (3.0 * U * K0 + 3.0 * K1 - x2 * (r2 * r2 + 3.0 * r3 * r3) * K2); /* 222 */
    q[7] = -4.0 * x2 * r3 * (U * K0 + K1 + x2 * (r2 * r2 - r3 * r3) * K2);       /* 223 */
    q[8] = -4.0 * x2 * r2 * (U * K0 + K1 + x2 * (r3 * r3 - r2 * r2) * K2);       /* 233 */
    q[9] = -4.0 * x2 * r3 * (3.0 * U * K0 + 3.0 * K1 - x2 * (3.0 * r2 * r2 + r3 * r3) * K2); /* 333 */
    sym_fill(q, re, im);
  }
}

int orc_Q1p(int kernel, double xi, double k1, double r2, double r3, double* re, double* im) {
  if (!valid_kernel(kernel) || !(k1 != 0)) return -1;
  double Kn[4];
  knu_all(k1 * k1 / (4.0 * xi * xi), xi * xi * (r2 * r2 + r3 * r3), Kn);
  q1p_from_k(kernel, xi, k1, r2, r3, Kn, re, im);
  return 0;
}

/* Q^{1P,(0)}(r2,r3;xi), Eqs. (1p-rotlet-Q0), (1p-stokeslet-Q0) (l_B = 1),
 * (1p-stresslet-Q0), auxiliary variables Eq. (1p-aux-zero); the limits at rho = 0 are
 * Eq. (1p-stokeslet-Q0-limit) and zero for the rotlet and stresslet. Real. */
int orc_Q1p0(int kernel, double xi, double r2, double r3, double* re) {
  if (!valid_kernel(kernel)) return -1;
  double rho2 = r2 * r2 + r3 * r3;
  int n = (kernel == ORC_STRESSLET) ? 27 : 9;
  memset(re, 0, n * sizeof(double));
  if (rho2 == 0.0) {
    if (kernel == ORC_STOKESLET) {
      double c = EULER_GAMMA + log(xi * xi) - 1.0;
      re[0] = 2.0 * c;
      re[4] = c;
      re[8] = c;
    }
    return 0;
  }
  double rho = sqrt(rho2);
  double V = xi * xi * rho2;
  double rt2 = r2 / rho, rt3 = r3 / rho;
  double phi0 = orc_En(1, V) + log(rho2) + 1.0;
  double phi1 = 1.0 - exp(-V);
  double phi2 = phi1 - V * exp(-V);
  if (kernel == ORC_ROTLET) {
    double c = 2.0 * phi1 / rho;
    double q[9] = {0, c * rt3, -c * rt2, -c * rt3, 0, 0, c * rt2, 0, 0};
    memcpy(re, q, sizeof q);
  } else if (kernel == ORC_STOKESLET) {
    double q[9] = {-2.0 * (phi0 + phi1), 0, 0,
                   0, -(phi0 + 2.0 * rt3 * rt3 * phi1), 2.0 * rt2 * rt3 * phi1,
                   0, 2.0 * rt2 * rt3 * phi1, -(phi0 + 2.0 * rt2 * rt2 * phi1)};
    memcpy(re, q, sizeof q);
  } else {
    double R4 = -4.0 / rho; /* the symbol R of Eq. (1p-stresslet-Q0); not the truncation radius */
    double complex q[10];
    q[0] = 0;                                                           /* 111 */
    q[1] = R4 * rt2 * (2.0 * phi1 - phi2);                              /* 112 */
    q[2] = R4 * rt3 * (2.0 * phi1 - phi2);                              /* 113 */
    q[3] = 0;                                                           /* 122 */
    q[4] = 0;                                                           /* 123 */
    q[5] = 0;                                                           /* 133 */
    q[6] = R4 * rt2 * (3.0 * phi1 - (rt2 * rt2 + 3.0 * rt3 * rt3) * phi2); /* 222 */
    q[7] = R4 * rt3 * (phi1 - (rt3 * rt3 - rt2 * rt2) * phi2);          /* 223 */
    q[8] = R4 * rt2 * (phi1 - (rt2 * rt2 - rt3 * rt3) * phi2);          /* 233 */
    q[9] = R4 * rt3 * (3.0 * phi1 - (3.0 * rt2 * rt2 + rt3 * rt3) * phi2); /* 333 */
    double im[27];
    sym_fill(q, re, im);
  }
  return 0;
}

int orc_fourier1p(const double L[3], double xi, double kmax, int kernel, long N,
                  const double* x, const double* f, long Nt, const double* t, double* u) {
  if (!valid_kernel(kernel) || !(xi > 0) || !(kmax > 0)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  if (!gl_ready) gl_init();
  const int nc = ncomp_in(kernel);
  int K1 = (int)floor(kmax * L[0] / (2.0 * M_PI));
#pragma omp parallel for schedule(dynamic, 1)
  for (long m = 0; m < Nt; ++m) {
    double acc[3] = {0, 0, 0};
    double Qre[27], Qim[27];
    for (long n = 0; n < N; ++n) {
      const double* fn = f + n * nc;
      double dx = t[m * 3 + 0] - x[n * 3 + 0];
      double r2 = t[m * 3 + 1] - x[n * 3 + 1];
      double r3 = t[m * 3 + 2] - x[n * 3 + 2];
      double V = xi * xi * (r2 * r2 + r3 * r3);
      for (int a = 1; a <= K1; ++a) {
        /* K_nu(U,V) depends on k1 only through k1^2: shared by +k1 and -k1 */
        double k1 = 2.0 * M_PI * a / L[0];
        double Kn[4];
        knu_all(k1 * k1 / (4.0 * xi * xi), V, Kn);
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          double kk = sgn * k1;
          q1p_from_k(kernel, xi, kk, r2, r3, Kn, Qre, Qim);
          double complex v[3];
          contract_c(kernel, Qre, Qim, fn, v);
          double complex e = cexp(I * kk * dx);
          for (int j = 0; j < 3; ++j) acc[j] += creal(v[j] * e);
        }
      }
      orc_Q1p0(kernel, xi, r2, r3, Qre);
      contract_add(kernel, Qre, fn, acc);
    }
    for (int j = 0; j < 3; ++j) u[m * 3 + j] += acc[j] / L[0];
  }
  return 0;
}

/* ------------------------------------------------------------ free space, direct sum */

int orc_direct0p(int kernel, long N, const double* x, const double* f, long Nt,
                 const double* t, double* u) {
  if (!valid_kernel(kernel)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  const int nc = ncomp_in(kernel);
#pragma omp parallel for schedule(dynamic, 16)
  for (long m = 0; m < Nt; ++m) {
    double acc[3] = {0, 0, 0};
    double G[27];
    for (long n = 0; n < N; ++n) {
      double r[3] = {t[m * 3] - x[n * 3], t[m * 3 + 1] - x[n * 3 + 1], t[m * 3 + 2] - x[n * 3 + 2]};
      if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) continue;
      kernel_full(kernel, r, G);
      contract_add(kernel, G, f + n * nc, acc);
    }
    for (int j = 0; j < 3; ++j) u[m * 3 + j] += acc[j];
  }
  return 0;
}

/* --------------------------------------------------------------------------- self term */

int orc_self(double xi, int kernel, long N, const double* x, const double* f, long Nt,
             const double* t, double* u) {
  if (!valid_kernel(kernel)) return -1;
  if (kernel != ORC_STOKESLET) return 0; /* zero for the rotlet and stresslet */
  const double c = -4.0 * xi / SQRTPI;     /* Eq. (3p-stokeslet-self-term) */
  if (t == NULL) {
    for (long m = 0; m < N; ++m)
      for (int j = 0; j < 3; ++j) u[m * 3 + j] += c * f[m * 3 + j];
    return 0;
  }
  for (long m = 0; m < Nt; ++m)
    for (long n = 0; n < N; ++n)
      if (t[m * 3] == x[n * 3] && t[m * 3 + 1] == x[n * 3 + 1] && t[m * 3 + 2] == x[n * 3 + 2])
        for (int j = 0; j < 3; ++j) u[m * 3 + j] += c * f[n * 3 + j];
  return 0;
}

/* ------------------------------------------ harmonic (Laplace) potential, phi = sum q / r
 *
 * The scalar potential of the harmonic kernel H(r) = 1/|r| (Sec. 2.1) with one strength q
 * per source; one output per target, u[m]. Ewald split with the Ewald screening function
 * (Eq. ewald-screening): real-space kernel erfc(xi r) / r, Fourier-space kernel
 * 4 pi / k^2 exp(-k^2 / 4 xi^2). Zero-mode conventions:
 *   3P: the potential has zero mean over the cell (the k = 0 term of the full kernel is
 *       left out); the Ewald form then carries the constant -pi Q / (xi^2 V), Q = sum q,
 *       which is minus the k -> 0 limit of the real-space kernel's transform over V.
 *   2P: the k^P = 0 mode uses the App. A result for the harmonic, whose kernel in the free
 *       direction is -2 pi |r_3| (no constant).
 *   1P: the k_1 = 0 mode uses the App. B result with gauge l_H = 1, i.e. the kernel
 *       -2 log(rho) in the free plane.
 *   0P: the plain free-space sum. */

int orc_h_real(int D, const double L[3], double xi, double rc, long N, const double* x,
               const double* q, long Nt, const double* t, double* u) {
  if (D < 0 || D > 3 || !(xi > 0) || !(rc > 0) || N < 0) return -1;
  if (t == NULL) { t = x; Nt = N; }
  int pmax[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) pmax[d] = (int)floor(rc / L[d]) + 1;
#pragma omp parallel for schedule(dynamic, 4)
  for (long m = 0; m < Nt; ++m) {
    double acc = 0;
    for (long n = 0; n < N; ++n)
      for (int p0 = -pmax[0]; p0 <= pmax[0]; ++p0)
        for (int p1 = -pmax[1]; p1 <= pmax[1]; ++p1)
          for (int p2 = -pmax[2]; p2 <= pmax[2]; ++p2) {
            double r0 = t[m * 3 + 0] - x[n * 3 + 0] + p0 * L[0];
            double r1 = t[m * 3 + 1] - x[n * 3 + 1] + p1 * L[1];
            double r2 = t[m * 3 + 2] - x[n * 3 + 2] + p2 * L[2];
            double rr = r0 * r0 + r1 * r1 + r2 * r2;
            if (rr == 0.0 || rr >= rc * rc) continue;
            double r = sqrt(rr);
            acc += q[n] * erfc(xi * r) / r;
          }
    u[m] += acc;
  }
  return 0;
}

/* 3P, k != 0, |k| <= kmax: (1/V) sum_k 4 pi / k^2 exp(-k^2/4xi^2) sum_n q_n e^{i k.(x - x_n)} */
int orc_h_fourier3p(const double L[3], double xi, double kmax, long N, const double* x,
                    const double* q, long Nt, const double* t, double* u) {
  if (!(xi > 0) || !(kmax > 0)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  int K[3];
  for (int d = 0; d < 3; ++d) K[d] = (int)floor(kmax * L[d] / (2.0 * M_PI));
  long nmax = (long)(2 * K[0] + 1) * (2 * K[1] + 1) * (2 * K[2] + 1);
  double* kv = (double*)malloc(sizeof(double) * 4 * nmax);
  long nk = 0;
  for (int a = -K[0]; a <= K[0]; ++a)
    for (int b = -K[1]; b <= K[1]; ++b)
      for (int c = -K[2]; c <= K[2]; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        double k0 = 2.0 * M_PI * a / L[0], k1 = 2.0 * M_PI * b / L[1], k2 = 2.0 * M_PI * c / L[2];
        double kk = k0 * k0 + k1 * k1 + k2 * k2;
        if (kk > kmax * kmax) continue;
        kv[nk * 4 + 0] = k0;
        kv[nk * 4 + 1] = k1;
        kv[nk * 4 + 2] = k2;
        kv[nk * 4 + 3] = 4.0 * M_PI / kk * exp(-kk / (4.0 * xi * xi));
        ++nk;
      }
  double complex* S = (double complex*)malloc(sizeof(double complex) * (nk > 0 ? nk : 1));
#pragma omp parallel for schedule(dynamic, 16)
  for (long k = 0; k < nk; ++k) {
    double complex acc = 0;
    for (long n = 0; n < N; ++n)
      acc += q[n] * cexp(-I * (kv[k * 4] * x[n * 3] + kv[k * 4 + 1] * x[n * 3 + 1] + kv[k * 4 + 2] * x[n * 3 + 2]));
    S[k] = acc;
  }
  const double vol = L[0] * L[1] * L[2];
#pragma omp parallel for schedule(dynamic, 16)
  for (long m = 0; m < Nt; ++m) {
    double acc = 0;
    for (long k = 0; k < nk; ++k)
      acc += kv[k * 4 + 3] *
             creal(S[k] * cexp(I * (kv[k * 4] * t[m * 3] + kv[k * 4 + 1] * t[m * 3 + 1] + kv[k * 4 + 2] * t[m * 3 + 2])));
    u[m] += acc / vol;
  }
  free(kv);
  free(S);
  return 0;
}

/* 3P zero-mean constant -pi Q / (xi^2 V), added to every target. */
int orc_h_k0_3p(const double L[3], double xi, long N, const double* q, long Nt, double* u) {
  double Q = 0;
  for (long n = 0; n < N; ++n) Q += q[n];
  const double c = -M_PI * Q / (xi * xi * L[0] * L[1] * L[2]);
  for (long m = 0; m < Nt; ++m) u[m] += c;
  return 0;
}

/* 2P: (1/A) [ sum_{k^P != 0} Q^{H,2P}(k1,k2,r3) e^{i(k1 r1 + k2 r2)} + Q^{H,2P,(0)}(r3) ]
 * per source, with Q^{H,2P} = (pi / alpha) beta^+ (Eq. 2p-QH-integral, auxiliary variables
 * Eq. 2p-aux) and Q^{H,2P,(0)} = -2 pi (r3 erf(xi r3) + exp(-xi^2 r3^2) / (sqrt(pi) xi))
 * (App. A, zero mode of the harmonic). */
int orc_h_fourier2p(const double L[3], double xi, double kmax, long N, const double* x,
                    const double* q, long Nt, const double* t, double* u) {
  if (!(xi > 0) || !(kmax > 0)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  int K1 = (int)floor(kmax * L[0] / (2.0 * M_PI));
  int K2 = (int)floor(kmax * L[1] / (2.0 * M_PI));
  const double area = L[0] * L[1];
#pragma omp parallel for schedule(dynamic, 1)
  for (long m = 0; m < Nt; ++m) {
    double acc = 0;
    for (long n = 0; n < N; ++n) {
      double r1 = t[m * 3 + 0] - x[n * 3 + 0];
      double r2 = t[m * 3 + 1] - x[n * 3 + 1];
      double r3 = t[m * 3 + 2] - x[n * 3 + 2];
      double s = 0;
      for (int a = -K1; a <= K1; ++a)
        for (int b = -K2; b <= K2; ++b) {
          if (a == 0 && b == 0) continue;
          double k1 = 2.0 * M_PI * a / L[0], k2 = 2.0 * M_PI * b / L[1];
          double al2 = k1 * k1 + k2 * k2;
          if (al2 > kmax * kmax) continue;
          double al = sqrt(al2);
          double bp = theta(+1.0, al, xi, r3) + theta(-1.0, al, xi, r3);
          s += M_PI / al * bp * cos(k1 * r1 + k2 * r2);
        }
      s += -2.0 * M_PI * (r3 * erf(xi * r3) + exp(-xi * xi * r3 * r3) / (SQRTPI * xi));
      acc += q[n] * s;
    }
    u[m] += acc / area;
  }
  return 0;
}

/* 1P: (1/L1) [ sum_{k1 != 0} K_0(U,V) e^{i k1 r1} + Q^{H,1P,(0)}(r2,r3) ] per source, with
 * Q^{H,1P} = K_0(U,V) (Eq. 1p-QH-integral, U, V of Eq. 1p-aux, K_nu of Eq. Knu-def) and
 * Q^{H,1P,(0)} = -log(rho^2) - E_1(xi^2 rho^2) (App. B, zero mode of the harmonic, l_H = 1),
 * whose limit at rho = 0 is EULER_GAMMA + log(xi^2). */
int orc_h_fourier1p(const double L[3], double xi, double kmax, long N, const double* x,
                    const double* q, long Nt, const double* t, double* u) {
  if (!(xi > 0) || !(kmax > 0)) return -1;
  if (t == NULL) { t = x; Nt = N; }
  if (!gl_ready) gl_init();
  int K1 = (int)floor(kmax * L[0] / (2.0 * M_PI));
#pragma omp parallel for schedule(dynamic, 1)
  for (long m = 0; m < Nt; ++m) {
    double acc = 0;
    for (long n = 0; n < N; ++n) {
      double r1 = t[m * 3 + 0] - x[n * 3 + 0];
      double r2 = t[m * 3 + 1] - x[n * 3 + 1];
      double r3 = t[m * 3 + 2] - x[n * 3 + 2];
      double rho2 = r2 * r2 + r3 * r3;
      double V = xi * xi * rho2;
      double s = 0;
      for (int a = 1; a <= K1; ++a) {
        double k1 = 2.0 * M_PI * a / L[0];
        double Kn[4];
        knu_all(k1 * k1 / (4.0 * xi * xi), V, Kn);
        s += 2.0 * Kn[1] * cos(k1 * r1);     /* the +k1 and -k1 terms */
      }
      s += rho2 > 0 ? -log(rho2) - orc_En(1, V) : EULER_GAMMA + log(xi * xi);
      acc += q[n] * s;
    }
    u[m] += acc / L[0];
  }
  return 0;
}

/* Free space: sum_n q_n / |t_m - x_n|, pairs at zero separation skipped. */
int orc_h_direct0p(long N, const double* x, const double* q, long Nt, const double* t, double* u) {
  if (t == NULL) { t = x; Nt = N; }
#pragma omp parallel for schedule(dynamic, 16)
  for (long m = 0; m < Nt; ++m) {
    double acc = 0;
    for (long n = 0; n < N; ++n) {
      double r0 = t[m * 3] - x[n * 3], r1 = t[m * 3 + 1] - x[n * 3 + 1], r2 = t[m * 3 + 2] - x[n * 3 + 2];
      double rr = r0 * r0 + r1 * r1 + r2 * r2;
      if (rr == 0.0) continue;
      acc += q[n] / sqrt(rr);
    }
    u[m] += acc;
  }
  return 0;
}

/* Self term of the harmonic: -(2 xi / sqrt(pi)) q (the r -> 0 limit of the Fourier-space
 * kernel erf(xi r) / r, removed for the omitted self pair); for every target coinciding
 * exactly with a source (every target in the star form). */
int orc_h_self(double xi, long N, const double* x, const double* q, long Nt, const double* t,
               double* u) {
  const double c = -2.0 * xi / SQRTPI;
  if (t == NULL) {
    for (long m = 0; m < N; ++m) u[m] += c * q[m];
    return 0;
  }
  for (long m = 0; m < Nt; ++m)
    for (long n = 0; n < N; ++n)
      if (t[m * 3] == x[n * 3] && t[m * 3 + 1] == x[n * 3 + 1] && t[m * 3 + 2] == x[n * 3 + 2])
        u[m] += c * q[n];
  return 0;
}
