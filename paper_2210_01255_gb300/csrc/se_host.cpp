// Host-side parts of libse that launch no GPU work: window functions and their Fourier
// transforms (Sec. 3.3), the error estimates and the parameter-selection procedure
// (Sec. 4), and status strings.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "se_internal.h"

namespace se {

// Modified Bessel function I_0 by its power series sum_k (x^2/4)^k / (k!)^2; every term is
// positive, so the sum is accurate for the arguments used here (x <= 2.5 * 32).
double bessel_i0(double x) {
  double q = 0.25 * x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / ((double)k * k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

static double kb_value(const WindowDesc& w, double r) {
  double t = 1.0 - (r / w.aw) * (r / w.aw);
  if (t < 0) return 0.0;
  return bessel_i0(w.beta * std::sqrt(t)) / w.i0beta;  // Eq. (KB-window)
}

void window_setup(WindowDesc* w, int kind, int P, double h) {
  w->kind = kind;
  w->P = P;
  w->aw = 0.5 * P * h;
  w->alpha = 0.91 * (M_PI / 2.0) * P;  // Eq. (TG-window)
  w->beta = 2.5 * P;                   // Eq. (PKB-parameters)
  w->i0beta = bessel_i0(w->beta);
  w->nu = std::min(P / 2 + 2, 10);
  w->pkb.clear();
  if (kind == SE_WIN_PKB) {
    // On subinterval q (offsets (q - P/2) h .. (q - P/2 + 1) h) interpolate the exact KB
    // window in the nu+1 Chebyshev points of the first kind; store Chebyshev coefficients
    // c_j of p(s) = sum_j c_j T_j(s), s in [-1, 1] (discrete Chebyshev transform).
    const int n = w->nu + 1;
    std::vector<double> s(n), v(n);
    for (int i = 0; i < n; ++i) s[i] = std::cos((2.0 * i + 1.0) * M_PI / (2.0 * n));
    w->pkb.resize((size_t)P * n);
    for (int q = 0; q < P; ++q) {
      double l = q - P / 2;
      for (int i = 0; i < n; ++i) v[i] = kb_value(*w, (l + 0.5 + 0.5 * s[i]) * h);
      for (int j = 0; j < n; ++j) {
        double c = 0;
        for (int i = 0; i < n; ++i) c += v[i] * std::cos(j * std::acos(s[i]));
        w->pkb[(size_t)q * n + j] = (j == 0 ? 1.0 : 2.0) * c / n;
      }
    }
  }
}

double window_value(const WindowDesc& w, double r) {
  if (w.kind == SE_WIN_GAUSSIAN)
    return std::fabs(r) <= w.aw ? std::exp(-w.alpha * (r / w.aw) * (r / w.aw)) : 0.0;
  return kb_value(w, r);
}

// Fourier transform of the 1-D window used in the scaling step: the untruncated Gaussian
// for the truncated-Gaussian window (Sec. 5.3), the exact KB transform otherwise (Eq. KB-window).
double window_hat(const WindowDesc& w, double k) {
  if (w.kind == SE_WIN_GAUSSIAN)
    return std::sqrt(M_PI / w.alpha) * w.aw * std::exp(-k * k * w.aw * w.aw / (4.0 * w.alpha));
  double z2 = w.beta * w.beta - k * k * w.aw * w.aw;
  double val;
  if (z2 > 0) {
    double z = std::sqrt(z2);
    val = std::sinh(z) / z;
  } else if (z2 < 0) {
    double z = std::sqrt(-z2);
    val = std::sin(z) / z;
  } else {
    val = 1.0;
  }
  return 2.0 * w.aw * val / w.i0beta;
}

// ------------------------------------------------------------------ error estimates (Sec. 4)

// Potential rms estimate U(L,Q,xi), Eqs. (pot-mag-est-*) with the mean C_U of Table 3.
double pot_mag(int kernel, double L, double Q, double xi) {
  double t = xi * L;
  if (kernel == SE_STOKESLET) {
    double f = (1.0 + 1.323e-2 * t + 2.469e-4 * t * t) * std::exp(-5.205 / (t * t));
    return 1.8 * std::sqrt(Q) * f / L;
  }
  if (kernel == SE_STRESSLET) return 7.2 * std::sqrt(Q) * std::sqrt(t) / (L * L);
  return 2.4 * std::sqrt(Q) * std::sqrt(t) * std::exp(-11.60 / (t * t)) / (L * L);
}

// Real-space truncation estimates, Eqs. (rs-trunc-est-stokeslet/-stresslet/-rotlet).
double est_real(int kernel, double L, double Q, double xi, double rc) {
  double L3 = L * L * L, e = std::exp(-xi * xi * rc * rc);
  if (kernel == SE_STOKESLET) return std::sqrt(4.0 * Q * rc / L3) * e;
  if (kernel == SE_STRESSLET)
    return std::sqrt(112.0 * Q * std::pow(xi, 4) * rc * rc * rc / (9.0 * L3)) * e;
  return std::sqrt(8.0 * Q / (3.0 * L3 * rc)) * e;
}

// Fourier-space truncation estimates, Eqs. (fs-trunc-est-rotlet/-stokeslet/-stresslet).
double est_fourier(int kernel, double L, double Q, double xi, double kinf) {
  double e = std::exp(-kinf * kinf / (4.0 * xi * xi));
  if (kernel == SE_STOKESLET) return 4.0 / (M_PI * L) * std::sqrt(Q / 3.0) * e;
  if (kernel == SE_STRESSLET) return 4.0 * kinf / (3.0 * M_PI * L) * std::sqrt(7.0 * Q / 2.0) * e;
  return std::sqrt(8.0 * xi * xi * Q / (3.0 * M_PI * L * L * L * kinf)) * e;
}

// Largest x with f(x) = target on the decreasing tail of f (f eventually decreasing).
template <typename F>
static double solve_tail(F f, double target, double lo, double hi) {
  // make sure f(hi) < target
  for (int i = 0; i < 200 && f(hi) >= target; ++i) hi *= 2.0;
  // walk lo up until f(lo) > target, else the tolerance holds for every x >= lo
  if (f(lo) <= target) return lo;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (f(mid) > target) lo = mid; else hi = mid;
  }
  return hi;
}

double rc_from_tol(int kernel, double L, double Q, double xi, double tau) {
  return solve_tail([&](double rc) { return est_real(kernel, L, Q, xi, rc); }, tau, 0.5 / xi, 20.0 / xi);
}
double kinf_from_tol(int kernel, double L, double Q, double xi, double tau) {
  return solve_tail([&](double k) { return est_fourier(kernel, L, Q, xi, k); }, tau, xi, 40.0 * xi);
}
// xi such that the real-space estimate at the given rc equals tau (decreasing in xi for
// xi rc beyond the estimate's maximum)
double xi_from_rc(int kernel, double L, double Q, double rc, double tau) {
  return solve_tail([&](double xi) { return est_real(kernel, L, Q, xi, rc); }, tau, 0.5 / rc, 20.0 / rc);
}

// Upsampling of the K_* class and its threshold, Eqs. (upsampling-factor-sstar) and
// (estimate-kbarstar), with lg = log(U / (2 tau)) / (2 pi). The printed rules are for a cube,
// where M = L/h is both the free extent of the sources and the periodic length. For a cuboid
// the two roles are separated: the aperiodic support along a free direction spans
// M_free = L_free/h grid points, and the slowest-decaying k^P != 0 mode, |k^P| = 2 pi / L_per,
// needs a further M_per lg points (M_per = the longest periodic side over h), so
//   s_* = max_free (M_free + M_per lg) / M',   kbar_* = max_free ceil(M_per lg / (M' - M_free) - 1),
// which reduce to the printed forms when M_free = M_per = M.
void upsampling_rule(int D, const double* box, double h, const int* Mext, double lg, double* s_star,
                     int* kbar_star) {
  double Mper = 0;
  for (int d = 0; d < D; ++d) Mper = std::max(Mper, box[d] / h);
  double ss = 1.0, kb = 0;
  for (int d = D; d < 3; ++d) {
    const double Mf = box[d] / h;
    ss = std::max(ss, (Mf + Mper * lg) / Mext[d]);
    kb = std::max(kb, std::ceil(Mper * lg / (Mext[d] - Mf) - 1.0));
  }
  *s_star = ss;
  *kbar_star = std::max(0, (int)kb);
}

// Average number of neighbours within rc, Table 5 (uniform system).
static double nrc_uniform(int kernel, int D) {
  static const double sr[4] = {2500, 950, 450, 400};  // stokeslet, rotlet, D = 0..3
  static const double st[4] = {6000, 1600, 800, 800}; // stresslet
  return kernel == SE_STRESSLET ? st[D] : sr[D];
}

// Box padding factor lambda, Table 4.
double lambda_table(int kernel, int D) {
  if (D >= 1) return 2.4;
  return kernel == SE_STOKESLET ? 2.2 : (kernel == SE_STRESSLET ? 2.4 : 1.5);
}

}  // namespace se

using namespace se;

namespace se {
// the smallest multiple of fM that is >= x; with smooth, the smallest even number >= x with no
// prime factor above 7 (cuFFT's fastest radices)
int round_extent(int x, int fM, bool smooth) {
  int v = fM * ((std::max(x, 1) + fM - 1) / fM);
  if (!smooth) return v;
  for (v = std::max(2, x + (x & 1));; v += 2) {
    int r = v;
    for (int q : {2, 3, 5, 7})
      while (r % q == 0) r /= q;
    if (r == 1) return v;
  }
}
}  // namespace se

extern "C" se_status se_autotune(int D, const double box[3], int kernel_mask, double Q, long long N,
                                 double tol_rel, se_opts* io, double* xi_io, double* rc_out,
                                 int M_out[3], int* P_out) {
  if (D < 0 || D > 3 || !box || !io || !xi_io || !rc_out || !M_out || !P_out) return SE_ERR_ARG;
  for (int i = 0; i < 3; ++i)
    if (!(box[i] > 0) || !std::isfinite(box[i])) return SE_ERR_ARG;
  if (!(Q > 0)) return SE_ERR_ARG;
  if (kernel_mask & ~31) return SE_ERR_ARG;
  // the harmonic field takes the rotlet's rules (both are first derivatives of H)
  const int rmask = rule_mask(kernel_mask);
  int kernels[3], nk = 0;
  for (int k : {SE_STOKESLET, SE_ROTLET, SE_STRESSLET})
    if (rmask & k) kernels[nk++] = k;
  if (nk == 0) return SE_ERR_ARG;
  const int fM = io->f_M > 0 ? io->f_M : 4;
  const bool smooth = (io->flags & SE_FLAG_FFT_SIZES) != 0;
  // a grid extent >= x: the next multiple of f_M (with SE_FLAG_FFT_SIZES: whose prime factors
  // are 2, 3, 5, 7 only)
  auto extent = [&](double x) { return round_extent((int)std::ceil(x - 1e-9), fM, smooth); };
  // In the estimates a cube of side L is assumed; for a cuboid L^3 -> |B|, L -> |B|^(1/3).
  const double vol = box[0] * box[1] * box[2];
  const double L = std::cbrt(vol);
  const bool absolute = io->tol_abs > 0 && !(tol_rel > 0);

  double xi = *xi_io;
  double tau = 0;
  // tau_abs from the relative tolerance with U of the kernel giving the smallest U
  auto tau_of = [&](double x) {
    if (absolute) return io->tol_abs;
    double t = 1e300;
    for (int i = 0; i < nk; ++i) t = std::min(t, tol_rel * pot_mag(kernels[i], L, Q, x));
    return t;
  };
  if (!(xi > 0)) {
    // Sec. 5.2: choose rc from the average neighbour count, then xi from the real-space
    // estimate at tolerance tau (a fixed point when tau depends on xi through U).
    if (N <= 0) return SE_ERR_ARG;
    double nrc = 0;
    for (int i = 0; i < nk; ++i) nrc = std::max(nrc, nrc_uniform(kernels[i], D));
    if (io->n_rc > 0) nrc = io->n_rc;
    double rc = std::cbrt(3.0 * nrc * vol / (4.0 * M_PI * (double)N));
    xi = 4.0 / rc;
    for (int it = 0; it < 60; ++it) {
      double t = tau_of(xi);
      double xn = 0;
      for (int i = 0; i < nk; ++i) xn = std::max(xn, xi_from_rc(kernels[i], L, Q, rc, t));
      if (std::fabs(xn - xi) < 1e-13 * xi) { xi = xn; break; }
      xi = xn;
    }
  }
  tau = tau_of(xi);
  if (!(tau > 0)) return SE_ERR_ARG;

  // step 1: rc; step 2: h_estimate = pi / k_inf; step 3: P_estimate
  double rc = 0, kinf = 0, Pest = 0;
  for (int i = 0; i < nk; ++i) {
    rc = std::max(rc, rc_from_tol(kernels[i], L, Q, xi, tau));
    kinf = std::max(kinf, kinf_from_tol(kernels[i], L, Q, xi, tau));
    double U = pot_mag(kernels[i], L, Q, xi);
    Pest = std::max(Pest, std::log(10.0 * U / tau) / 2.5);  // Eq. (approximation-estimate)
  }
  double h_est = M_PI / kinf;
  // step 4: error-pollution rule, Eq. (error-pollution-fix), then Eq. (grid-adjustment)
  double h_t = D == 0 ? h_est / 1.1 : h_est / 1.05;
  double P_t = Pest + (io->P_margin >= 0 ? (double)io->P_margin : (D == 0 ? 2.0 : 4.0));
  // isotropic h: the first periodic direction (or direction 0 for D = 0) fixes h
  int M[3] = {0, 0, 0};
  // (for D = 0, M_0 only sets h; the transform extents are the M'_i below)
  M[0] = D > 0 ? extent(box[0] / h_t) : round_extent((int)std::ceil(box[0] / h_t - 1e-9), fM, false);
  double h = box[0] / M[0];
  for (int d = 1; d < 3; ++d) {
    double md = box[d] / h;
    if (d < D) {
      int mi = (int)std::llround(md);
      if (std::fabs(md - mi) > 1e-9 * md) return SE_ERR_UNSUPPORTED;  // non-commensurate box
      M[d] = mi;
    } else {
      M[d] = std::max(2, (int)std::llround(md));  // informational for free directions
    }
  }
  // step 5: P
  int P = 2 * (int)std::ceil(P_t / 2.0);
  P = std::max(2, std::min(P, MAX_P));
  // the window must fit the grid (P <= M): refine the grid where it does not
  if (M[0] < P) {
    M[0] = extent((double)P);
    h = box[0] / M[0];
    for (int d = 1; d < 3; ++d) {
      double md = box[d] / h;
      if (d < D) {
        int mi = (int)std::llround(md);
        if (std::fabs(md - mi) > 1e-9 * md) return SE_ERR_UNSUPPORTED;
        M[d] = mi;
      } else {
        M[d] = std::max(2, (int)std::llround(md));
      }
    }
  }
  for (int d = 0; d < D; ++d)
    if (M[d] < P || (M[d] & 1)) return SE_ERR_UNSUPPORTED;
  // steps 6-7: extended grid, truncation radius and upsampling (free directions)
  if (D < 3) {
    double Mext[3] = {0, 0, 0};
    for (int d = D; d < 3; ++d) {
      double lam = io->lambda > 0 ? io->lambda : 0;
      double Md = 0;
      for (int i = 0; i < nk; ++i) {
        double lm = lam > 0 ? lam : lambda_table(kernels[i], D);
        double theta = kernels[i] == SE_ROTLET ? 0.0 : 8.0;
        double v = box[d] / h + P + (lm - 1.0) * std::max((double)P, theta);  // Eq. (extended-grid-size)
        Md = std::max(Md, (double)extent(v));
      }
      Mext[d] = Md;
      io->Mext[d] = (int)Md;
    }
    double R2 = 0, minLe = 1e300;
    for (int d = D; d < 3; ++d) {
      double Le = h * Mext[d];
      R2 += Le * Le;
      minLe = std::min(minLe, Le);
    }
    double R = std::sqrt(R2);
    double s0 = 1.0 + R / minLe;               // Eq. (upsampling-factor-s0)
    s0 = std::ceil(10.0 * s0 - 1e-9) / 10.0;
    io->s0 = s0;
    if (D > 0) {
      double Umin = 1e300;
      for (int i = 0; i < nk; ++i) Umin = std::min(Umin, pot_mag(kernels[i], L, Q, xi));
      double lg = std::max(0.0, std::log(Umin / (2.0 * tau)) / (2.0 * M_PI));
      int me[3] = {0, 0, 0};
      for (int d = D; d < 3; ++d) me[d] = (int)Mext[d];
      upsampling_rule(D, box, h, me, lg, &io->s_star, &io->kbar_star);
    }
  }
  io->f_M = fM;
  io->tol_abs = tau;
  *xi_io = xi;
  *rc_out = rc;
  M_out[0] = M[0];
  M_out[1] = M[1];
  M_out[2] = M[2];
  *P_out = P;
  return SE_OK;
}

extern "C" const char* se_status_str(se_status s) {
  switch (s) {
    case SE_OK: return "ok";
    case SE_ERR_ARG: return "invalid argument";
    case SE_ERR_RANGE: return "coordinate out of range";
    case SE_ERR_NOMEM: return "out of memory";
    case SE_ERR_CUDA: return "CUDA error";
    case SE_ERR_CUFFT: return "cuFFT error";
    case SE_ERR_TIMEOUT: return "device wait timed out";
    case SE_ERR_UNSUPPORTED: return "unsupported request";
    case SE_ERR_CAPACITY: return "request exceeds a fixed capacity";
  }
  return "unknown status";
}

extern "C" se_status se_opts_default(se_opts* o) {
  if (!o) return SE_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->prec = SE_FP64;
  o->f_M = 4;
  o->kbar_star = -1;
  o->P_margin = -1;
  return SE_OK;
}
