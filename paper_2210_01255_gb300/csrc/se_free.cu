// libse: the Fourier-space steps (ii)-(iv) of Alg. 1 for reduced periodicity (D = 2, 1, 0):
// the adaptive FFT of Sec. 3.4 with the modified kernels of Sec. 3.1 for D = 2 and D = 1,
// and the zero-padded transform with the precomputed truncated kernel of Sec. 3.5 for D = 0.
//
// Layouts (component-major, direction 2 contiguous):
//   D = 2: grid [C][M0][M1][M'2] -> 2-D R2C over (0,1) -> spec [C][M0][M1/2+1][M'2]; the
//          columns along direction 2 are transformed per class: k^P = 0 (zero-padded to n0),
//          K_* (|kbar_i| <= kbar_*, padded to n_*), K_inf (length M'2, in place).
//   D = 1: grid [C][M0][M'1][M'2] -> 1-D R2C over 0 -> spec [C][M0/2+1][M'1][M'2]; the planes
//          along (1,2) are transformed per class in the same way.
//   D = 0: grid [C][M'0][2M'1][2M'2] (points spread into the first M' of each direction, the
//          rest zero) -> 2-D R2C over (1,2) into [C][2M'0][2M'1][M'2+1] (planes >= M'0 zero)
//          -> 1-D C2C over 0 -> scaled by the precomputed kernel -> the inverse steps.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "se_device.cuh"

namespace se {

// ----------------------------------------------------------- modified kernels (host, FP64)

// 1 - cos t - t sin t by its series for small t
static double s_1mcos_tsin(double t) {
  double out = 0, term = 1;
  for (int m = 1; m < 25; ++m) {
    term *= -t * t / ((2.0 * m - 1) * (2.0 * m));
    out += term * (2.0 * m - 1);
  }
  return out;
}
// H^_R^{2P}(kappa), below Eq. (2p-vico-H-kernel); -2 pi R^2 at 0
static double hat_H2p(double kap, double R) {
  double t = R * std::fabs(kap);
  if (t == 0) return -2.0 * M_PI * R * R;
  if (t < 0.5) return 4.0 * M_PI * R * R * s_1mcos_tsin(t) / (t * t);
  return 4.0 * M_PI / (kap * kap) * (1.0 - std::cos(t) - t * std::sin(t));
}
// Im Z^_R^{2P}(kappa) = -8 pi sin^2(R kappa/2)/kappa; 0 at 0
static double hat_Z2p_im(double kap, double R) {
  if (kap == 0) return 0.0;
  double s = std::sin(R * kap / 2);
  return -8.0 * M_PI * s * s / kap;
}
// 1 - J0(t) (which = 0) or 1 - J0(t) - t J1(t)/2 (which = 1) by their power series
static double s_bessel(double t, int which) {
  double q = 0.25 * t * t, term = 1, out = 0;
  for (int m = 1; m < 40; ++m) {
    term *= q / ((double)m * m);
    double sgn = (m % 2 == 0) ? -1.0 : 1.0;
    out += which == 0 ? sgn * term : sgn * term * (1.0 - m);
  }
  return out;
}
// Eq. (optimal-1p-harmonic), pi R^2 at 0
static double hat_H1p(double kap, double R) {
  double t = R * kap;
  if (t == 0) return M_PI * R * R;
  if (t < 2.0) return 4.0 * M_PI * R * R * s_bessel(t, 0) / (t * t);
  return 4.0 * M_PI / (kap * kap) * (1.0 - std::cyl_bessel_j(0.0, t));
}
// Eq. (optimal-1p-biharmonic), -pi R^4 / 8 at 0
static double hat_B1p(double kap, double R) {
  double t = R * kap;
  if (t == 0) return -M_PI * R * R * R * R / 8.0;
  if (t < 2.0) return -8.0 * M_PI * std::pow(R, 4) * s_bessel(t, 1) / std::pow(t, 4);
  return -8.0 * M_PI / std::pow(kap, 4) * (1.0 - std::cyl_bessel_j(0.0, t) - 0.5 * t * std::cyl_bessel_j(1.0, t));
}

// ---------------------------------------------------------------- device: 0P precompute

// Eq. (vico-harmonic-0p) and Eq. (optimal-biharmonic-0p) with the series for small R kappa
__device__ inline double dev_hat0p(int biharm, double kap, double R) {
  const double pi = 3.14159265358979323846;
  if (!biharm) {
    if (kap == 0) return 2.0 * pi * R * R;
    double s = sin(R * kap / 2);
    return 8.0 * pi * s * s / (kap * kap);
  }
  double t = R * kap;
  if (t < 1.0) {
    // -8 pi R^4 sum_{m>=2} (-1)^m (m-1) t^{2m-4} / (2m+1)!
    double sum = 0, tp = 1, fact = 120.0;  // t^{2m-4}, (2m+1)! at m = 2
    for (int m = 2; m < 20; ++m) {
      sum += ((m & 1) ? -1.0 : 1.0) * (m - 1) * tp / fact;
      tp *= t * t;
      fact *= (2.0 * m + 2) * (2.0 * m + 3);
    }
    return -8.0 * pi * R * R * R * R * sum;
  }
  return -8.0 * pi / (kap * kap * kap * kap) * (1.0 + 0.5 * cos(t) - 1.5 * sin(t) / t);
}

// A^_R on the half spectrum of the upsampled grid (complex, imaginary part 0)
__global__ void k_fill_ahat(int n0, int n1, int n2, double h, double R, int biharm, double* out) {
  const int h2 = n2 / 2 + 1;
  const size_t N = (size_t)n0 * n1 * h2;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int i2 = (int)(i % h2), i1 = (int)((i / h2) % n1), i0 = (int)(i / ((size_t)h2 * n1));
  const int b0 = i0 < (n0 + 1) / 2 ? i0 : i0 - n0, b1 = i1 < (n1 + 1) / 2 ? i1 : i1 - n1, b2 = i2;
  const double pi = 3.14159265358979323846;
  const double k0 = 2 * pi * b0 / (n0 * h), k1 = 2 * pi * b1 / (n1 * h), k2 = 2 * pi * b2 / (n2 * h);
  out[2 * i] = dev_hat0p(biharm, sqrt(k0 * k0 + k1 * k1 + k2 * k2), R);
  out[2 * i + 1] = 0.0;
}

// Least-squares fit of the truncated kernel by an even polynomial of degree 6 in r
// (SE_FLAG_SPLIT_POLY): over the 2M' box of offsets o (FFT order, r^2 = h^2 |o|^2,
// t = r^2 / R^2), the sums sums[k] = sum t^k (k = 0..6) and sums[7 + j] = sum A(o) t^j
// (j = 0..3) of the normal equations, accumulated in FP64 (block partials added atomically).
constexpr int PS_NB = 4;                   // basis 1, t, t^2, t^3
constexpr int PS_NSUM = 2 * PS_NB - 1 + PS_NB;
__global__ void k_poly_fit_sums(const double* A, int u0, int u1, int u2, int m0, int m1, int m2, double scale,
                                double h2R2, double* sums) {
  const int n0 = 2 * m0, n1 = 2 * m1, n2 = 2 * m2;
  const size_t N = (size_t)n0 * n1 * n2;
  double acc[PS_NSUM];
  for (int k = 0; k < PS_NSUM; ++k) acc[k] = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(i % n2), i1 = (int)((i / n2) % n1), i0 = (int)(i / ((size_t)n2 * n1));
    const int o0 = i0 < m0 ? i0 : i0 - n0, o1 = i1 < m1 ? i1 : i1 - n1, o2 = i2 < m2 ? i2 : i2 - n2;
    const int s0 = ((o0 % u0) + u0) % u0, s1 = ((o1 % u1) + u1) % u1, s2 = ((o2 % u2) + u2) % u2;
    const double v = A[((size_t)s0 * u1 + s1) * u2 + s2] * scale;
    const double t = h2R2 * ((double)o0 * o0 + (double)o1 * o1 + (double)o2 * o2);
    double tk = 1.0;
    for (int k = 0; k < 2 * PS_NB - 1; ++k) {
      acc[k] += tk;
      if (k < PS_NB) acc[2 * PS_NB - 1 + k] += v * tk;
      tk *= t;
    }
  }
  __shared__ double red[PS_NSUM][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < PS_NSUM; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < PS_NSUM) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    atomicAdd(&sums[threadIdx.x], v);
  }
}

// truncate A_R to the 2M' offsets around the origin (FFT order), normalise the inverse
// transform, take out the fitted polynomial (SE_FLAG_SPLIT_POLY: pa0 + pa1 r^2 + pa2 r^4 +
// pa3 r^6, in the units of the normalised samples; zero otherwise) and mollify the biharmonic
// (Sec. 3.5)
__global__ void k_trunc_moll(const double* A, int u0, int u1, int u2, int m0, int m1, int m2, int biharm,
                             double scale, double h, double pa0, double pa1, double pa2, double pa3, double* At) {
  const int n0 = 2 * m0, n1 = 2 * m1, n2 = 2 * m2;
  const size_t N = (size_t)n0 * n1 * n2;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int i2 = (int)(i % n2), i1 = (int)((i / n2) % n1), i0 = (int)(i / ((size_t)n2 * n1));
  const int o0 = i0 < m0 ? i0 : i0 - n0, o1 = i1 < m1 ? i1 : i1 - n1, o2 = i2 < m2 ? i2 : i2 - n2;
  const int s0 = ((o0 % u0) + u0) % u0, s1 = ((o1 % u1) + u1) % u1, s2 = ((o2 % u2) + u2) % u2;
  double v = A[((size_t)s0 * u1 + s1) * u2 + s2] * scale;
  if (biharm) {
    const double r2 = h * h * ((double)o0 * o0 + (double)o1 * o1 + (double)o2 * o2);
    v -= pa0 + r2 * (pa1 + r2 * (pa2 + r2 * pa3));
    // mu = (f(3), f(2), f(1), f(0), 1, ..., 1, f(0), f(1), f(2), f(3)) in natural order
    const double a = 2.0 / 7.0 * sqrt(log(100.0));
    const int nat[3] = {o0 + m0, o1 + m1, o2 + m2};
    const int len[3] = {n0, n1, n2};
    for (int d = 0; d < 3; ++d) {
      int t = -1;
      if (nat[d] < 4) t = 3 - nat[d];
      else if (nat[d] >= len[d] - 4) t = nat[d] - (len[d] - 4);
      if (t >= 0) v *= exp(-a * a * t * t) + exp(-a * a * (t - 7.0) * (t - 7.0));
    }
  }
  At[i] = v;
}

template <typename T>
__global__ void k_real_part(const double* z, size_t n, T* out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)z[2 * i];
}

// ----------------------------------------------------------- device: AFT copies and scaling

// column / plane selection: mode 0 = the k^P = 0 class, 1 = K_*, 2 = every column in place
struct ColMap {
  int D;        // 2 or 1
  int mode;
  int M0, M1;   // periodic grid sizes (D = 2: M0, M1; D = 1: M0)
  int H;        // stored extent of the halved periodic direction (M1/2+1 for D = 2, M0/2+1 for D = 1)
  int kstar;
  int xm;       // D = 1: component slots per x wavenumber of the spectrum [H][xm][planes]
};

// periodic indices of column j of a class (FFT order); returns false for a slot that is not a
// real column
__device__ inline void colmap_idx(const ColMap& m, int j, int* i0, int* i1) {
  if (m.D == 2) {
    if (m.mode == 0) { *i0 = 0; *i1 = 0; return; }
    if (m.mode == 2) { *i0 = j / m.H; *i1 = j % m.H; return; }
    // K_*: a in [-k*, k*], b in [0, k*], (a, b) != (0, 0)
    const int w = m.kstar + 1;
    int jj = j + (j >= m.kstar * w ? 1 : 0);
    const int a = jj / w - m.kstar, b = jj % w;
    *i0 = a < 0 ? a + m.M0 : a;
    *i1 = b;
    return;
  }
  // D = 1: planes indexed by the x wavenumber (half spectrum 0..M0/2)
  if (m.mode == 0) *i0 = 0;
  else if (m.mode == 1) *i0 = 1 + j;
  else *i0 = j;
  *i1 = 0;
}

__device__ inline bool in_class(const ColMap& m, int i0, int i1, int cls) {
  // class of the periodic wavenumber (i0, i1): 0, 1 (K_*) or 2 (K_inf)
  if (m.D == 2) {
    const int a = i0 < m.M0 / 2 ? i0 : i0 - m.M0, b = i1;
    int c = (a == 0 && b == 0) ? 0 : ((abs(a) <= m.kstar && b <= m.kstar) ? 1 : 2);
    return c == cls;
  }
  int c = i0 == 0 ? 0 : (i0 <= m.kstar ? 1 : 2);
  return c == cls;
}

// copy class columns (D = 2: length Mz along direction 2; D = 1: planes Mf1 x Mf2) from spec
// into a zero-padded class buffer, or back (truncated) for the output components
struct Ext2 {
  int v[2];
};
template <typename T>
__global__ void k_aft_copy(ColMap m, int ncomp, int ncols, Ext2 fm, Ext2 fn, bool to_buffer, T* spec, T* bufp) {
  // fm: extents in spec of the free directions (1 or 2 values), fn: padded extents
  const int* f_m = fm.v;
  const int* f_n = fn.v;
  const int nf = m.D == 2 ? 1 : 2;
  // 32-bit index arithmetic (the launcher checks ncomp ncols plane_n < 2^31)
  const unsigned plane_n = nf == 1 ? (unsigned)f_n[0] : (unsigned)f_n[0] * f_n[1];
  const size_t plane_m = nf == 1 ? (size_t)f_m[0] : (size_t)f_m[0] * f_m[1];
  const unsigned N = (unsigned)ncomp * ncols * plane_n;
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned q = i / plane_n;
  const unsigned e = i - q * plane_n;
  const int j = (int)(q % (unsigned)ncols);
  const int c = (int)(q / (unsigned)ncols);
  int a0, a1;
  if (nf == 1) {
    a0 = (int)e;
    a1 = 0;
  } else {
    a0 = (int)(e / (unsigned)f_n[1]);
    a1 = (int)(e - (unsigned)a0 * f_n[1]);
  }
  const bool inside = nf == 1 ? a0 < f_m[0] : (a0 < f_m[0] && a1 < f_m[1]);
  int i0, i1;
  colmap_idx(m, j, &i0, &i1);
  size_t so;
  if (m.D == 2) so = (((size_t)c * m.M0 + i0) * m.H + i1) * plane_m + (inside ? a0 : 0);
  else so = ((size_t)i0 * m.xm + c) * plane_m + (inside ? (size_t)a0 * f_m[1] + a1 : 0);
  const size_t bo = (size_t)i;
  if (to_buffer) {
    bufp[2 * bo] = inside ? spec[2 * so] : T(0);
    bufp[2 * bo + 1] = inside ? spec[2 * so + 1] : T(0);
  } else if (inside) {
    spec[2 * so] = bufp[2 * bo];
    spec[2 * so + 1] = bufp[2 * bo + 1];
  }
}

struct FreeScale {
  ColMap m;
  int cls;        // 0, 1, 2
  int ncols;
  int fn[2];      // transform lengths in the free directions (one for D = 2)
  double h;
  double kf0, kf1;  // 2 pi / L_0, 2 pi / L_1 (periodic)
  double inv4xi2;
  long long cstr, jstr;  // complex elements between components and between columns of the buffer
};

// One kernel's operator on one mode (Eq. SE-scaling-disc): the regular symbol for
// k^P != 0 (scalar s), the modified kernels of Eqs. (mod-*-2p) / (mod-*-1p) for the k^P = 0
// class (scalars mr + i mi, and tb = B^ for D = 1). Writes the 3 output components (1 for
// the harmonic potential).
template <typename T>
__device__ __forceinline__ void free_mode(const FreeScale& a, int kernel, T s, T k0, T k1, T k2, T mr, T mi, T tb,
                                          const T* re, const T* im, T* ore, T* oim) {
  if (a.cls != 0) {
    apply_regular<T>(kernel, s, k0, k1, k2, re, im, ore, oim);
  } else if (a.m.D == 2) {
    // modified column: scalar (mr + i mi) times D^S, D^Omega or D^T; the harmonic field's
    // column has only the direction-2 derivative: the rotlet's scalar (the same derivative of
    // the modified harmonic kernel) times (0, 0, q)
    T vr[3], vi[3];
    if (kernel == SE_HARMONIC) {
      // the truncated harmonic kernel itself (its table holds H^_R^{2P} gamma^)
      vr[0] = re[0]; vi[0] = im[0];
      vr[1] = 0; vi[1] = 0;
      vr[2] = 0; vi[2] = 0;
    } else if (kernel == SE_HARMONIC_FIELD) {
      vr[0] = 0; vi[0] = 0;
      vr[1] = 0; vi[1] = 0;
      vr[2] = re[0]; vi[2] = im[0];
    } else if (kernel == SE_STOKESLET) {
      vr[0] = 2 * re[0]; vi[0] = 2 * im[0];
      vr[1] = 2 * re[1]; vi[1] = 2 * im[1];
      vr[2] = 0; vi[2] = 0;
    } else if (kernel == SE_ROTLET) {
      vr[0] = re[1]; vi[0] = im[1];
      vr[1] = -re[0]; vi[1] = -im[0];
      vr[2] = 0; vi[2] = 0;
    } else {
      // D^T_1lm F_lm = -2 (F13 + F31), D^T_2lm F_lm = -2 (F23 + F32), D^T_3lm F_lm = -2 tr F
      vr[0] = -4 * re[4]; vi[0] = -4 * im[4];
      vr[1] = -4 * re[5]; vi[1] = -4 * im[5];
      vr[2] = -2 * (re[0] + re[1] + re[2]); vi[2] = -2 * (im[0] + im[1] + im[2]);
    }
    for (int q = 0; q < 3; ++q) {
      ore[q] = mr * vr[q] - mi * vi[q];
      oim[q] = mr * vi[q] + mi * vr[q];
    }
  } else {
    // modified plane (D = 1), k = (0, kappa2, kappa3)
    const T q2 = k1, q3 = k2;
    if (harmonic_family(kernel)) {
      apply_regular<T>(kernel, mr, T(0), q2, q3, re, im, ore, oim);
    } else if (kernel == SE_STOKESLET) {
      ore[0] = 2 * mr * re[0];
      oim[0] = 2 * mr * im[0];
      ore[1] = tb * (-q3 * q3 * re[1] + q2 * q3 * re[2]);
      oim[1] = tb * (-q3 * q3 * im[1] + q2 * q3 * im[2]);
      ore[2] = tb * (q2 * q3 * re[1] - q2 * q2 * re[2]);
      oim[2] = tb * (q2 * q3 * im[1] - q2 * q2 * im[2]);
    } else {
      // 2i C^TH H^ - i C^TB B^ with symmetric F: 11,22,33,12,13,23 = 0..5
      const T kk = q2 * q2 + q3 * q3;
      T chr[3], chi[3], cbr[3], cbi[3];
      chr[0] = 2 * q2 * re[3] + 2 * q3 * re[4];
      chi[0] = 2 * q2 * im[3] + 2 * q3 * im[4];
      chr[1] = q2 * re[0];
      chi[1] = q2 * im[0];
      chr[2] = q3 * re[0];
      chi[2] = q3 * im[0];
      cbr[0] = 0;
      cbi[0] = 0;
      const T c22 = q2 * (3 * kk - 2 * q2 * q2), c23 = q3 * (kk - 2 * q2 * q2), c33 = q2 * (kk - 2 * q3 * q3);
      cbr[1] = c22 * re[1] + 2 * c23 * re[5] + c33 * re[2];
      cbi[1] = c22 * im[1] + 2 * c23 * im[5] + c33 * im[2];
      const T d22 = q3 * (kk - 2 * q2 * q2), d23 = q2 * (kk - 2 * q3 * q3), d33 = q3 * (3 * kk - 2 * q3 * q3);
      cbr[2] = d22 * re[1] + 2 * d23 * re[5] + d33 * re[2];
      cbi[2] = d22 * im[1] + 2 * d23 * im[5] + d33 * im[2];
      for (int q = 0; q < 3; ++q) {
        const T vr = 2 * mr * chr[q] - tb * cbr[q];
        const T vi = 2 * mr * chi[q] - tb * cbi[q];
        ore[q] = -vi;  // i (vr + i vi)
        oim[q] = vr;
      }
    }
  }
}

// Scaling step, Eq. (SE-scaling-disc), on a class buffer [C][ncols][free...] in place:
// regular kernel for k^P != 0; the modified kernels of Eqs. (mod-*-2p) / (mod-*-1p) for the
// k^P = 0 class. Tables (plan precision): tp0/tp1 periodic factors, tf0/tf1 free factors
// (exp(-k^2/4xi^2) / w^2 / n each); for the k^P = 0 class mod0 / mod1 hold the modified-
// kernel scalars (D = 2: complex scalar of the kernel, and of the stresslet for S|T in mod1;
// D = 1: H^ and B^). S|T sums the stokeslet operator on components 0..2 and the stresslet
// operator on components 3..8.
template <typename T>
__global__ void k_scale_free(FreeScale a, int kernel, int n_rhs, const T* __restrict__ tp0,
                             const T* __restrict__ tp1, const T* __restrict__ tf0, const T* __restrict__ tf1,
                             const T* __restrict__ mod0, const T* __restrict__ mod1, T* __restrict__ spec) {
  const int nf = a.m.D == 2 ? 1 : 2;
  const size_t plane = nf == 1 ? (size_t)a.fn[0] : (size_t)a.fn[0] * a.fn[1];
  const size_t per = (size_t)a.ncols * plane;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= per) return;
  const int j = (int)(idx / plane);
  const size_t e = idx % plane;
  int i0, i1;
  colmap_idx(a.m, j, &i0, &i1);
  // skip columns of other classes when running in place over every column
  if (a.cls == 2 && !in_class(a.m, i0, i1, 2)) return;
  int f0 = nf == 1 ? (int)e : (int)(e / a.fn[1]);
  int f1 = nf == 1 ? 0 : (int)(e % a.fn[1]);
  const int cin = kernel_comps(kernel), no = out_comps(kernel);
  // wavenumbers
  bool zero = false;
  T k0, k1, k2;
  const double pi2 = 2.0 * 3.14159265358979323846;
  const int kb_f0 = f0 < a.fn[0] / 2 ? f0 : f0 - a.fn[0];
  if (f0 == a.fn[0] / 2) zero = true;
  int kb_f1 = 0;
  if (nf == 2) {
    kb_f1 = f1 < a.fn[1] / 2 ? f1 : f1 - a.fn[1];
    if (f1 == a.fn[1] / 2) zero = true;
  }
  T s = 0;
  T mr = 0, mi = 0, tb = 0, mr2 = 0, mi2 = 0;  // mr2, mi2: stresslet scalar of S|T
  if (a.m.D == 2) {
    const int kb0 = i0 < a.m.M0 / 2 ? i0 : i0 - a.m.M0;
    if (i0 == a.m.M0 / 2 || i1 == a.m.M1 / 2) zero = true;
    k0 = (T)(a.kf0 * kb0);
    k1 = (T)(a.kf1 * i1);
    k2 = (T)(pi2 * kb_f0 / (a.fn[0] * a.h));
    if (a.cls == 0) {
      mr = mod0[2 * f0];
      mi = mod0[2 * f0 + 1];
      if (kernel == SE_KERNEL_ST) {
        mr2 = mod1[2 * f0];
        mi2 = mod1[2 * f0 + 1];
      }
    } else {
      const T kk = k0 * k0 + k1 * k1 + k2 * k2;
      s = regular_scalar<T>(kernel, kk, (T)a.inv4xi2) * tp0[i0] * tp1[i1] * tf0[f0];
    }
  } else {
    if (i0 == a.m.M0 / 2) zero = true;
    k0 = (T)(a.kf0 * i0);
    k1 = (T)(pi2 * kb_f0 / (a.fn[0] * a.h));
    k2 = (T)(pi2 * kb_f1 / (a.fn[1] * a.h));
    if (a.cls == 0) {
      mr = mod0[e];       // H^-type table for this kernel
      tb = mod1 ? mod1[e] : T(0);  // B^ table (stokeslet, stresslet)
      mr2 = mr;           // the stresslet of S|T uses the same H^ and B^
    } else {
      const T kk = k0 * k0 + k1 * k1 + k2 * k2;
      s = regular_scalar<T>(kernel, kk, (T)a.inv4xi2) * tp0[i0] * tf0[f0] * tf1[f1];
    }
  }
  const size_t H = (size_t)a.cstr;  // component stride in this buffer
  const size_t jo = (size_t)j * a.jstr + e;
  // in place, in the order that never overwrites an input still to be read (see k_scale3p)
  for (int rr = 0; rr < n_rhs; ++rr) {
    const int r = cin >= no ? rr : n_rhs - 1 - rr;
    T re[9], im[9];
    for (int c = 0; c < cin; ++c) {
      const size_t o = (((size_t)(cin * r + c)) * H + jo) * 2;
      re[c] = spec[o];
      im[c] = spec[o + 1];
    }
    T ore[3] = {0, 0, 0}, oim[3] = {0, 0, 0};
    if (!zero) {
      if (kernel == SE_KERNEL_ST) {
        T tre[3], tim[3];
        free_mode<T>(a, SE_STOKESLET, s, k0, k1, k2, mr, mi, tb, re, im, ore, oim);
        free_mode<T>(a, SE_STRESSLET, s, k0, k1, k2, mr2, mi2, tb, re + 3, im + 3, tre, tim);
        for (int q = 0; q < 3; ++q) {
          ore[q] += tre[q];
          oim[q] += tim[q];
        }
      } else {
        free_mode<T>(a, kernel, s, k0, k1, k2, mr, mi, tb, re, im, ore, oim);
      }
    }
    for (int q = 0; q < no; ++q) {
      const size_t o = (((size_t)(no * r + q)) * H + jo) * 2;
      spec[o] = ore[q];
      spec[o + 1] = oim[q];
    }
  }
}

// gauge constants: u[r][i][j] += c_j sum_n f[r][n][j] (f the first nc <= 3 of stride
// components, u with nc components per target)
template <typename T>
__global__ void k_fsum(const T* f, int stride, int nc, int n, int n_rhs, double* sums) {
  __shared__ double red[3][256];
  for (int r = 0; r < n_rhs; ++r) {
    double a[3] = {0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      for (int j = 0; j < nc; ++j) a[j] += (double)f[((size_t)r * n + i) * stride + j];
    for (int j = 0; j < 3; ++j) red[j][threadIdx.x] = a[j];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
      if (threadIdx.x < off)
        for (int j = 0; j < 3; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0)
      for (int j = 0; j < 3; ++j) atomicAdd(&sums[r * 3 + j], red[j][0]);
    __syncthreads();
  }
}

template <typename T>
__global__ void k_add_const(int nt, int n_rhs, int nc, const double* sums, double c0, double c1, double c2, T* u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const double c[3] = {c0, c1, c2};
  for (int r = 0; r < n_rhs; ++r)
    for (int j = 0; j < nc; ++j) u[((size_t)r * nt + i) * nc + j] += (T)(c[j] * sums[r * 3 + j]);
}

// ----------------------------------------------------------------------- host side

template <typename T>
static se_status upload_tab(const std::vector<double>& v, DevBuf* b) {
  std::vector<T> h(v.begin(), v.end());
  if (b->p) cudaFree(b->p);
  b->p = nullptr;
  size_t bytes = sizeof(T) * std::max<size_t>(1, h.size());
  if (cudaMalloc(&b->p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SE_ERR_NOMEM;
  }
  b->bytes = bytes;
  if (!h.empty()) SE_CUDA(cudaMemcpy(b->p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return SE_OK;
}

static se_status upload_any(se_plan_t* p, const std::vector<double>& v, DevBuf* b) {
  return p->prec == SE_FP32 ? upload_tab<float>(v, b) : upload_tab<double>(v, b);
}

// exp(-k^2/4xi^2) / w^_0(k)^2 / n at the FFT-order wavenumbers of a length-n direction
static std::vector<double> sep_table(const se_plan_t* p, int n, int count) {
  std::vector<double> g(count);
  for (int i = 0; i < count; ++i) {
    int kb = i < (n + 1) / 2 ? i : i - n;
    if (i == n / 2) kb = -n / 2;
    double k = 2.0 * M_PI * kb / (p->geom.h * n);
    double wh = window_hat(p->win, k);
    g[i] = std::exp(-k * k / (4.0 * p->xi * p->xi)) / (wh * wh) / n;
  }
  return g;
}

static se_status precompute_0p(se_plan_t* p, int biharm, DevBuf* out) {
  const GridGeom& g = p->geom;
  int u[3];
  const int fM = p->opts.f_M > 0 ? p->opts.f_M : 4;
  for (int d = 0; d < 3; ++d) u[d] = fM * (int)std::ceil(p->s0 * g.m[d] / fM - 1e-9);
  const size_t hu = (size_t)u[0] * u[1] * (u[2] / 2 + 1);
  const size_t nu = (size_t)u[0] * u[1] * u[2];
  const size_t nt = (size_t)(2 * g.m[0]) * (2 * g.m[1]) * (2 * g.m[2]);
  const size_t ht = (size_t)(2 * g.m[0]) * (2 * g.m[1]) * (g.m[2] + 1);
  double *ahat = nullptr, *areal = nullptr, *at = nullptr, *atr = nullptr;
  se_status st = SE_OK;
  cufftHandle h1 = 0, h2 = 0;
  bool h1ok = false, h2ok = false;
  do {
    if (cudaMalloc(&ahat, sizeof(double) * 2 * hu) != cudaSuccess) { st = SE_ERR_NOMEM; break; }
    if (cudaMalloc(&areal, sizeof(double) * nu) != cudaSuccess) { st = SE_ERR_NOMEM; break; }
    k_fill_ahat<<<grid1d((long long)hu, 256), 256, 0, p->stream>>>(u[0], u[1], u[2], g.h, p->R, biharm, ahat);
    if (cufftPlan3d(&h1, u[0], u[1], u[2], CUFFT_Z2D) != CUFFT_SUCCESS) { st = SE_ERR_CUFFT; break; }
    h1ok = true;
    cufftSetStream(h1, p->stream);
    if (cufftExecZ2D(h1, (cufftDoubleComplex*)ahat, areal) != CUFFT_SUCCESS) { st = SE_ERR_CUFFT; break; }
    cudaStreamSynchronize(p->stream);
    cudaFree(ahat);
    ahat = nullptr;
    cufftDestroy(h1);
    h1ok = false;
    if (cudaMalloc(&at, sizeof(double) * nt) != cudaSuccess) { st = SE_ERR_NOMEM; break; }
    // SE_FLAG_SPLIT_POLY: fit c0 + c1 r^2 + c2 r^4 + c3 r^6 to the biharmonic samples (normal
    // equations in t = r^2 / R^2, solved in FP64 with partial pivoting)
    double pa[PS_NB] = {0, 0, 0, 0};
    p->poly_on = false;
    if (biharm && (p->flags & SE_FLAG_SPLIT_POLY)) {
      double* sums = nullptr;
      if (cudaMalloc(&sums, sizeof(double) * PS_NSUM) != cudaSuccess) { st = SE_ERR_NOMEM; break; }
      cudaMemsetAsync(sums, 0, sizeof(double) * PS_NSUM, p->stream);
      const double R2 = p->R * p->R;
      k_poly_fit_sums<<<std::min(grid1d((long long)nt, 256), 152 * 8), 256, 0, p->stream>>>(
          areal, u[0], u[1], u[2], g.m[0], g.m[1], g.m[2], 1.0 / (double)nu, g.h * g.h / R2, sums);
      double hs[PS_NSUM];
      const bool ok = cudaMemcpyAsync(hs, sums, sizeof hs, cudaMemcpyDeviceToHost, p->stream) == cudaSuccess &&
                      cudaStreamSynchronize(p->stream) == cudaSuccess;
      cudaFree(sums);
      if (!ok) { st = SE_ERR_CUDA; break; }
      double Mx[PS_NB][PS_NB + 1];
      for (int a = 0; a < PS_NB; ++a) {
        for (int b = 0; b < PS_NB; ++b) Mx[a][b] = hs[a + b];
        Mx[a][PS_NB] = hs[2 * PS_NB - 1 + a];
      }
      for (int c = 0; c < PS_NB; ++c) {
        int piv = c;
        for (int a = c + 1; a < PS_NB; ++a)
          if (std::fabs(Mx[a][c]) > std::fabs(Mx[piv][c])) piv = a;
        for (int b = 0; b <= PS_NB; ++b) std::swap(Mx[c][b], Mx[piv][b]);
        if (!(std::fabs(Mx[c][c]) > 0)) { st = SE_ERR_UNSUPPORTED; break; }
        for (int a = c + 1; a < PS_NB; ++a) {
          const double f = Mx[a][c] / Mx[c][c];
          for (int b = c; b <= PS_NB; ++b) Mx[a][b] -= f * Mx[c][b];
        }
      }
      if (st != SE_OK) break;
      double b[PS_NB];
      for (int a = PS_NB - 1; a >= 0; --a) {
        double v = Mx[a][PS_NB];
        for (int c = a + 1; c < PS_NB; ++c) v -= Mx[a][c] * b[c];
        b[a] = v / Mx[a][a];
      }
      // from the t basis to r^2 powers, in the units of the samples (h^3 B_R)
      double rp = 1.0;
      const double h3 = g.h * g.h * g.h;
      for (int k = 0; k < PS_NB; ++k) {
        pa[k] = b[k] / rp;
        p->poly_c[k] = pa[k] / h3;
        rp *= R2;
      }
      p->poly_on = true;
    }
    k_trunc_moll<<<grid1d((long long)nt, 256), 256, 0, p->stream>>>(areal, u[0], u[1], u[2], g.m[0], g.m[1],
                                                                   g.m[2], biharm, 1.0 / (double)nu, g.h, pa[0],
                                                                   pa[1], pa[2], pa[3], at);
    cudaStreamSynchronize(p->stream);
    cudaFree(areal);
    areal = nullptr;
    if (cudaMalloc(&atr, sizeof(double) * 2 * ht) != cudaSuccess) { st = SE_ERR_NOMEM; break; }
    if (cufftPlan3d(&h2, 2 * g.m[0], 2 * g.m[1], 2 * g.m[2], CUFFT_D2Z) != CUFFT_SUCCESS) { st = SE_ERR_CUFFT; break; }
    h2ok = true;
    cufftSetStream(h2, p->stream);
    if (cufftExecD2Z(h2, at, (cufftDoubleComplex*)atr) != CUFFT_SUCCESS) { st = SE_ERR_CUFFT; break; }
    size_t es = p->prec == SE_FP32 ? 4 : 8;
    if (cudaMalloc(&out->p, es * ht) != cudaSuccess) { st = SE_ERR_NOMEM; break; }
    out->bytes = es * ht;
    if (p->prec == SE_FP32)
      k_real_part<float><<<grid1d((long long)ht, 256), 256, 0, p->stream>>>(atr, ht, (float*)out->p);
    else
      k_real_part<double><<<grid1d((long long)ht, 256), 256, 0, p->stream>>>(atr, ht, (double*)out->p);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) st = SE_ERR_CUDA;
  } while (0);
  if (h1ok) cufftDestroy(h1);
  if (h2ok) cufftDestroy(h2);
  if (ahat) cudaFree(ahat);
  if (areal) cudaFree(areal);
  if (at) cudaFree(at);
  if (atr) cudaFree(atr);
  cudaGetLastError();
  return st;
}

// Tables and precomputation of a D < 3 plan (called by se_plan_create after the geometry).
se_status free_plan_setup(se_plan_t* p) {
  const GridGeom& g = p->geom;
  const int D = p->D;
  const double h = g.h;
  if (D == 0) {
    for (int d = 0; d < 3; ++d) {
      int n = g.n[d];
      SE_TRY(upload_any(p, sep_table(p, n, d == 2 ? n / 2 + 1 : n), &p->ptab[d]));
    }
    int mask = rule_mask(p->opts.kernel_mask ? p->opts.kernel_mask : 7);
    if (mask & SE_ROTLET) SE_TRY(precompute_0p(p, 0, &p->atr[0]));
    if (mask & (SE_STOKESLET | SE_STRESSLET)) SE_TRY(precompute_0p(p, 1, &p->atr[1]));
    return SE_OK;
  }
  if (D == 2) {
    SE_TRY(upload_any(p, sep_table(p, g.m[0], g.m[0]), &p->ptab[0]));
    SE_TRY(upload_any(p, sep_table(p, g.m[1], g.m[1] / 2 + 1), &p->ptab[1]));
    for (int c = 0; c < 3; ++c) {
      int n = p->ncls[c][2];
      SE_TRY(upload_any(p, sep_table(p, n, n), &p->ftab[c][2]));
    }
    // k^P = 0 column: modified scalar times gamma^ / w^2 and the normalisation, complex
    const int n0 = p->ncls[0][2];
    const double w00 = window_hat(p->win, 0.0);
    // 0: stokeslet, 1: stresslet, 2: rotlet and harmonic field, 3: harmonic potential
    for (int kind = 0; kind < 4; ++kind) {
      std::vector<double> t(2 * n0);
      for (int i = 0; i < n0; ++i) {
        int kb = i < n0 / 2 ? i : i - n0;
        double kap = 2.0 * M_PI * kb / (n0 * h);
        double wh = window_hat(p->win, kap);
        double e = std::exp(-kap * kap / (4.0 * p->xi * p->xi));
        double scr = kind >= 2 ? e : e * (1.0 + kap * kap / (4.0 * p->xi * p->xi));
        double norm = scr / (w00 * w00 * w00 * w00 * wh * wh) / ((double)g.m[0] * g.m[1] * n0);
        if (i == n0 / 2) norm = 0;
        if (kind == 0 || kind == 3) {
          t[2 * i] = hat_H2p(kap, p->R) * norm;
          t[2 * i + 1] = 0;
        } else {
          t[2 * i] = 0;
          t[2 * i + 1] = hat_Z2p_im(kap, p->R) * norm;
        }
      }
      SE_TRY(upload_any(p, t, &p->mod0[kind]));
    }
    return SE_OK;
  }
  // D = 1
  SE_TRY(upload_any(p, sep_table(p, g.m[0], g.m[0] / 2 + 1), &p->ptab[0]));
  for (int c = 0; c < 3; ++c)
    for (int d = 1; d < 3; ++d) {
      int n = p->ncls[c][d];
      SE_TRY(upload_any(p, sep_table(p, n, n), &p->ftab[c][d]));
    }
  const int n1 = p->ncls[0][1], n2 = p->ncls[0][2];
  const double w00 = window_hat(p->win, 0.0);
  std::vector<double> TH_H((size_t)n1 * n2), TB_H((size_t)n1 * n2), TH_E((size_t)n1 * n2);
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b) {
      int ka = a < n1 / 2 ? a : a - n1, kb = b < n2 / 2 ? b : b - n2;
      double k2 = 2.0 * M_PI * ka / (n1 * h), k3 = 2.0 * M_PI * kb / (n2 * h);
      double kap = std::sqrt(k2 * k2 + k3 * k3);
      double w2 = window_hat(p->win, k2), w3 = window_hat(p->win, k3);
      double e = std::exp(-kap * kap / (4.0 * p->xi * p->xi));
      double scrH = e * (1.0 + kap * kap / (4.0 * p->xi * p->xi));
      double base = 1.0 / (w00 * w00 * w2 * w2 * w3 * w3) / ((double)g.m[0] * n1 * n2);
      if (a == n1 / 2 || b == n2 / 2) base = 0;
      double Hr = hat_H1p(kap, p->R), Br = hat_B1p(kap, p->R);
      size_t i = (size_t)a * n2 + b;
      TH_H[i] = Hr * scrH * base;
      TB_H[i] = Br * scrH * base;
      TH_E[i] = Hr * e * base;
    }
  SE_TRY(upload_any(p, TH_H, &p->mod0[0]));
  SE_TRY(upload_any(p, TB_H, &p->mod0[1]));
  SE_TRY(upload_any(p, TH_E, &p->mod0[2]));
  return SE_OK;
}

namespace {

// cached cuFFT plans for the free-direction transforms, keyed by a small integer tag
se_status free_fft(se_plan_t* p, int tag, int batch, int rank, const int* n, int* inembed, int istride,
                   int idist, int* onembed, int ostride, int odist, cufftType type, cufftHandle* out) {
  // the key holds every argument: plans of the same tag and batch can differ in their strides
  std::vector<long long> key = {tag, batch, rank, istride, idist, ostride, odist, (long long)type};
  for (int d = 0; d < rank; ++d) {
    key.push_back(n[d]);
    key.push_back(inembed ? inembed[d] : -1);
    key.push_back(onembed ? onembed[d] : -1);
  }
  auto it = p->ffree->find(key);
  if (it != p->ffree->end()) {
    SE_CUFFT(cufftSetStream(it->second, p->stream));  // the stream the caller issues on now
    *out = it->second;
    return SE_OK;
  }
  cufftHandle h;
  int nn[3] = {n[0], rank > 1 ? n[1] : 0, rank > 2 ? n[2] : 0};
  SE_CUFFT(cufftPlanMany(&h, rank, nn, inembed, istride, idist, onembed, ostride, odist, type, batch));
  SE_CUFFT(cufftSetStream(h, p->stream));
  (*p->ffree)[key] = h;
  *out = h;
  return SE_OK;
}

template <typename T> struct FT;
template <> struct FT<float> {
  static constexpr cufftType R2C = CUFFT_R2C, C2R = CUFFT_C2R, C2C = CUFFT_C2C;
  static cufftResult r2c(cufftHandle h, float* i, float* o) { return cufftExecR2C(h, i, (cufftComplex*)o); }
  static cufftResult c2r(cufftHandle h, float* i, float* o) { return cufftExecC2R(h, (cufftComplex*)i, o); }
  static cufftResult c2c(cufftHandle h, float* i, float* o, int dir) {
    return cufftExecC2C(h, (cufftComplex*)i, (cufftComplex*)o, dir);
  }
};
template <> struct FT<double> {
  static constexpr cufftType R2C = CUFFT_D2Z, C2R = CUFFT_Z2D, C2C = CUFFT_Z2Z;
  static cufftResult r2c(cufftHandle h, double* i, double* o) { return cufftExecD2Z(h, i, (cufftDoubleComplex*)o); }
  static cufftResult c2r(cufftHandle h, double* i, double* o) { return cufftExecZ2D(h, (cufftDoubleComplex*)i, o); }
  static cufftResult c2c(cufftHandle h, double* i, double* o, int dir) {
    return cufftExecZ2Z(h, (cufftDoubleComplex*)i, (cufftDoubleComplex*)o, dir);
  }
};

}  // namespace

// SE_FLAG_FFT_TIMED (D = 0): among the even extents M'_d >= mmin[d] whose transform lengths
// 2 M'_d have no prime factor above 7, up to 25 % above the minimum, the ones whose transforms
// take the least time. A candidate's cost is that of one evaluation's transforms and scaling:
// cin forward (2-D R2C over directions 1, 2 of the M'_0 planes, 1-D C2C along direction 0)
// and no inverse transforms, timed on scratch buffers with CUDA events (best of 3), plus the
// scaling pass estimated from its bytes. Equal minima (a cube) are searched together, others
// one direction at a time. Results are kept per (precision, minima, cin, no) for the process.
namespace {
std::mutex fft0_mu;
std::map<std::vector<int>, std::array<int, 3>> fft0_cache;

bool smooth7(int v) {
  for (int q : {2, 3, 5, 7})
    while (v % q == 0) v /= q;
  return v == 1;
}

template <typename T>
double fft0_cost(const int me[3], int cin, int no, cudaStream_t st) {
  const int n0 = 2 * me[0], n1 = 2 * me[1], n2 = 2 * me[2], h2 = n2 / 2 + 1, m0 = me[0];
  if ((double)n0 * n1 * n2 >= 2147483647.0) return -1;
  const size_t lines = (size_t)n1 * h2, GS = (size_t)m0 * n1 * n2, H = (size_t)n0 * lines;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const size_t need = sizeof(T) * (GS + 4 * H);
  if (need * 2 > fr) return -1;  // leave room: the plan's own buffers come later
  T *grid = nullptr, *tmp = nullptr, *spec = nullptr;
  cufftHandle hA = 0, hB = 0, hAi = 0;
  bool okA = false, okB = false, okAi = false;
  double cost = -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  do {
    if (cudaMalloc(&grid, sizeof(T) * GS) != cudaSuccess || cudaMalloc(&tmp, sizeof(T) * 2 * H) != cudaSuccess ||
        cudaMalloc(&spec, sizeof(T) * 2 * H) != cudaSuccess)
      break;
    cudaMemsetAsync(grid, 0, sizeof(T) * GS, st);
    cudaMemsetAsync(tmp, 0, sizeof(T) * 2 * H, st);
    int nA[2] = {n1, n2}, nB[1] = {n0}, eB[1] = {n0};
    okA = cufftPlanMany(&hA, 2, nA, nullptr, 1, n1 * n2, nullptr, 1, (int)lines, FT<T>::R2C, m0) == CUFFT_SUCCESS;
    okB = okA && cufftPlanMany(&hB, 1, nB, eB, (int)lines, 1, eB, (int)lines, 1, FT<T>::C2C, (int)lines) ==
                     CUFFT_SUCCESS;
    okAi = okB && cufftPlanMany(&hAi, 2, nA, nullptr, 1, (int)lines, nullptr, 1, n1 * n2, FT<T>::C2R, m0) ==
                      CUFFT_SUCCESS;
    if (!okAi) break;
    cufftSetStream(hA, st);
    cufftSetStream(hB, st);
    cufftSetStream(hAi, st);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    double best_f = 1e30, best_i = 1e30;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {
      cudaEventRecord(e0, st);
      ok = FT<T>::r2c(hA, grid, tmp) == CUFFT_SUCCESS && FT<T>::c2c(hB, tmp, spec, CUFFT_FORWARD) == CUFFT_SUCCESS;
      cudaEventRecord(e1, st);
      ok = ok && FT<T>::c2c(hB, spec, spec, CUFFT_INVERSE) == CUFFT_SUCCESS && FT<T>::c2r(hAi, spec, grid) == CUFFT_SUCCESS;
      cudaEventRecord(e2, st);
      float tf = 0, ti = 0;
      ok = ok && cudaEventSynchronize(e2) == cudaSuccess && cudaEventElapsedTime(&tf, e0, e1) == cudaSuccess &&
           cudaEventElapsedTime(&ti, e1, e2) == cudaSuccess;
      if (ok && rep > 0) {  // the first round warms up
        best_f = std::min(best_f, (double)tf);
        best_i = std::min(best_i, (double)ti);
      }
    }
    if (!ok) break;
    const double scale_ms = (double)(cin + no) * 2 * sizeof(T) * H / 5e12 * 1e3;
    cost = cin * best_f + no * best_i + scale_ms;
  } while (0);
  if (okA) cufftDestroy(hA);
  if (okB) cufftDestroy(hB);
  if (okAi) cufftDestroy(hAi);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  cudaFree(grid);
  cudaFree(tmp);
  cudaFree(spec);
  cudaGetLastError();
  return cost;
}
}  // namespace

se_status fft0_timed_extents(int prec, cudaStream_t st, const int mmin[3], int cin, int no, int out[3]) {
  std::lock_guard<std::mutex> lk(fft0_mu);
  const std::vector<int> key = {prec, mmin[0], mmin[1], mmin[2], cin, no};
  auto it = fft0_cache.find(key);
  if (it != fft0_cache.end()) {
    for (int d = 0; d < 3; ++d) out[d] = it->second[d];
    return SE_OK;
  }
  auto cost = [&](const int me[3]) {
    return prec == SE_FP32 ? fft0_cost<float>(me, cin, no, st) : fft0_cost<double>(me, cin, no, st);
  };
  auto cands = [](int lo) {
    std::vector<int> c;
    for (int v = lo + (lo & 1); v <= lo + lo / 4 && c.size() < 8; v += 2)
      if (smooth7(2 * v)) c.push_back(v);
    if (c.empty()) c.push_back(lo);
    return c;
  };
  int best[3] = {mmin[0], mmin[1], mmin[2]};
  if (mmin[0] == mmin[1] && mmin[1] == mmin[2]) {
    double bc = -1;
    for (int v : cands(mmin[0])) {
      const int me[3] = {v, v, v};
      const double c = cost(me);
      if (c >= 0 && (bc < 0 || c < bc)) {
        bc = c;
        best[0] = best[1] = best[2] = v;
      }
    }
  } else {
    for (int d = 0; d < 3; ++d) {
      double bc = -1;
      int bv = best[d];
      for (int v : cands(mmin[d])) {
        int me[3] = {best[0], best[1], best[2]};
        me[d] = v;
        const double c = cost(me);
        if (c >= 0 && (bc < 0 || c < bc)) {
          bc = c;
          bv = v;
        }
      }
      best[d] = bv;
    }
  }
  fft0_cache[key] = {best[0], best[1], best[2]};
  for (int d = 0; d < 3; ++d) out[d] = best[d];
  return SE_OK;
}

// Steps (ii)-(iv) for D = 2, 1 (adaptive FFT) and D = 0 (padded FFT with the precomputed
// kernel). grid: C spread components; ugrid: receives the 3 n_rhs inverse-transformed
// components on the spread grid.
template <typename T>
se_status fourier_free(se_plan_t* p, int kernel, int n_rhs, T* grid, int C, T* ugrid, int NC) {
  const GridGeom& g = p->geom;
  cudaStream_t st = p->stream;
  const int D = p->D;
  // k^P = 0 tables of D = 2 per kernel: 0 stokeslet, 1 stresslet, 2 rotlet and harmonic
  // field, 3 harmonic potential (S|T: 0 and 1)
  const int kidx = kernel == SE_HARMONIC ? 3 : ((kernel & SE_STOKESLET) ? 0 : (kernel == SE_STRESSLET ? 1 : 2));
  // spectrum and class buffers hold the C inputs and, after the in-place scaling, the NC
  // outputs (C < NC for the harmonic field)
  const int CS = std::max(C, NC);
  if (D == 0) {
    // the 3-D R2C of the 2M' grid, scaling by A^_{R,tr} (Sec. 3.5), the C2R. The grid holds
    // only the first M'_0 planes along direction 0 ([C][M'0][2M'1][2M'2], zero beyond M' along
    // directions 1 and 2): the transform is done as 2-D R2C over (1, 2) of those M'_0 planes
    // into a buffer [C][2M'0][2M'1][M'2+1] whose other planes stay zero, then 1-D C2C along
    // direction 0 into the spectrum; the inverse runs the same steps backwards and keeps the
    // first M'_0 planes. Same transform as the 3-D one, without its passes over zero planes.
    const int biharm = !harmonic_family(kernel);
    if (!p->atr[biharm].p) return SE_ERR_UNSUPPORTED;  // kernel not in the plan's kernel_mask
    const int m0 = g.m[0], n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], h2 = n2 / 2 + 1;
    const size_t GS = (size_t)g.cs;               // real elements per grid component
    const size_t H = (size_t)n0 * n1 * h2;        // complex elements per spectrum component
    void *spec, *tmp;
    SE_TRY(buf(p, "spec", sizeof(T) * 2 * CS * H, &spec));
    SE_TRY(buf(p, "tmp0p", sizeof(T) * 2 * C * H, &tmp));
    if (p->zeroed_tmp != tmp || p->zeroed_tmp_C != C) {
      SE_CUDA(cudaMemsetAsync(tmp, 0, sizeof(T) * 2 * C * H, st));
      p->zeroed_tmp = tmp;
      p->zeroed_tmp_C = C;
    }
    int nA[2] = {n1, n2};
    int nB[1] = {n0}, eB[1] = {n0};
    const int lines = n1 * h2;
    cufftHandle hA, hB, hAi;
    SE_TRY(free_fft(p, 30, m0, 2, nA, nullptr, 1, n1 * n2, nullptr, 1, lines, FT<T>::R2C, &hA));
    SE_TRY(free_fft(p, 31, lines, 1, nB, eB, lines, 1, eB, lines, 1, FT<T>::C2C, &hB));
    SE_TRY(free_fft(p, 32, m0, 2, nA, nullptr, 1, lines, nullptr, 1, n1 * n2, FT<T>::C2R, &hAi));
    for (int c = 0; c < C; ++c) {
      SE_CUFFT(FT<T>::r2c(hA, grid + c * GS, (T*)tmp + 2 * c * H));
      SE_CUFFT(FT<T>::c2c(hB, (T*)tmp + 2 * c * H, (T*)spec + 2 * c * H, CUFFT_FORWARD));
    }
    stage_event(p, 3);
    ScaleTables<T> tb{(const T*)p->ptab[0].p, (const T*)p->ptab[1].p, (const T*)p->ptab[2].p,
                      (const T*)p->atr[biharm].p};
    SE_TRY(launch_scale3p<T>(p, kernel, n_rhs, (T*)spec, tb));
    p->scale_modes = (long long)H;
    stage_event(p, 4);
    for (int c = 0; c < NC; ++c) {
      SE_CUFFT(FT<T>::c2c(hB, (T*)spec + 2 * c * H, (T*)spec + 2 * c * H, CUFFT_INVERSE));
      SE_CUFFT(FT<T>::c2r(hAi, (T*)spec + 2 * c * H, ugrid + c * GS));
    }
    return SE_OK;
  }
  const int M0 = g.m[0];
  if (D == 2) {
    const int M1 = g.m[1], Mz = g.m[2];
    const int H1 = M1 / 2 + 1;
    const size_t G = (size_t)M0 * M1 * Mz;
    const size_t S = (size_t)M0 * H1 * Mz;  // complex elements per component
    void* spec;
    SE_TRY(buf(p, "spec", sizeof(T) * 2 * CS * S, &spec));
    // (ii-a) 2-D R2C over (0, 1) for every z, one execution per component
    int n2[2] = {M0, M1};
    int in2[2] = {M0, M1}, on2[2] = {M0, H1};
    cufftHandle h2f, h2i;
    SE_TRY(free_fft(p, 10, Mz, 2, n2, in2, Mz, 1, on2, Mz, 1, FT<T>::R2C, &h2f));
    SE_TRY(free_fft(p, 11, Mz, 2, n2, on2, Mz, 1, in2, Mz, 1, FT<T>::C2R, &h2i));
    for (int c = 0; c < C; ++c) SE_CUFFT(FT<T>::r2c(h2f, grid + (size_t)c * G, (T*)spec + 2 * (size_t)c * S));
    // class buffers for k^P = 0 and K_*
    ColMap cm{2, 0, M0, M1, H1, p->kbar_star, 0};
    const int ncolS = (2 * p->kbar_star + 1) * (p->kbar_star + 1) - 1;
    const int n0 = p->ncls[0][2], nS = p->ncls[1][2];
    if ((double)CS * std::max(ncolS, 1) * nS >= 2147483647.0 || (double)CS * n0 >= 2147483647.0)
      return SE_ERR_UNSUPPORTED;  // class buffers are indexed with 32-bit offsets
    void *b0, *bS;
    SE_TRY(buf(p, "aft.b0", sizeof(T) * 2 * CS * (size_t)n0, &b0));
    SE_TRY(buf(p, "aft.bS", sizeof(T) * 2 * CS * (size_t)std::max(ncolS, 1) * nS, &bS));
    const Ext2 em{{Mz, 0}}, e0{{n0, 0}}, eS{{nS, 0}};
    cm.mode = 0;
    k_aft_copy<T><<<grid1d((long long)C * n0, 256), 256, 0, st>>>(cm, C, 1, em, e0, true, (T*)spec, (T*)b0);
    if (ncolS > 0) {
      cm.mode = 1;
      k_aft_copy<T><<<grid1d((long long)C * ncolS * nS, 256), 256, 0, st>>>(cm, C, ncolS, em, eS, true,
                                                                            (T*)spec, (T*)bS);
    }
    // (ii-b) 1-D transforms along direction 2 per class
    int nz[1] = {Mz}, nz0[1] = {n0}, nzS[1] = {nS};
    cufftHandle hz, hzi, hz0, hz0i, hzS, hzSi;
    SE_TRY(free_fft(p, 12, C * M0 * H1, 1, nz, nullptr, 1, Mz, nullptr, 1, Mz, FT<T>::C2C, &hz));
    SE_TRY(free_fft(p, 13, NC * M0 * H1, 1, nz, nullptr, 1, Mz, nullptr, 1, Mz, FT<T>::C2C, &hzi));
    SE_TRY(free_fft(p, 14, C, 1, nz0, nullptr, 1, n0, nullptr, 1, n0, FT<T>::C2C, &hz0));
    SE_TRY(free_fft(p, 15, NC, 1, nz0, nullptr, 1, n0, nullptr, 1, n0, FT<T>::C2C, &hz0i));
    SE_CUFFT(FT<T>::c2c(hz, (T*)spec, (T*)spec, CUFFT_FORWARD));
    SE_CUFFT(FT<T>::c2c(hz0, (T*)b0, (T*)b0, CUFFT_FORWARD));
    if (ncolS > 0) {
      SE_TRY(free_fft(p, 16, C * ncolS, 1, nzS, nullptr, 1, nS, nullptr, 1, nS, FT<T>::C2C, &hzS));
      SE_TRY(free_fft(p, 17, NC * ncolS, 1, nzS, nullptr, 1, nS, nullptr, 1, nS, FT<T>::C2C, &hzSi));
      SE_CUFFT(FT<T>::c2c(hzS, (T*)bS, (T*)bS, CUFFT_FORWARD));
    }
    // (iii) scaling per class
    stage_event(p, 3);
    FreeScale fs;
    fs.h = g.h;
    fs.kf0 = 2.0 * M_PI / g.L[0];
    fs.kf1 = 2.0 * M_PI / g.L[1];
    fs.inv4xi2 = 1.0 / (4.0 * p->xi * p->xi);
    const T* tp0 = (const T*)p->ptab[0].p;
    const T* tp1 = (const T*)p->ptab[1].p;
    fs.m = cm;
    fs.m.mode = 2;
    fs.cls = 2;
    fs.ncols = M0 * H1;
    fs.fn[0] = Mz;
    fs.fn[1] = 1;
    fs.cstr = (long long)M0 * H1 * Mz;
    fs.jstr = Mz;
    k_scale_free<T><<<grid1d((long long)M0 * H1 * Mz, 256), 256, 0, st>>>(
        fs, kernel, n_rhs, tp0, tp1, (const T*)p->ftab[2][2].p, nullptr, nullptr, nullptr, (T*)spec);
    fs.m.mode = 0;
    fs.cls = 0;
    fs.ncols = 1;
    fs.fn[0] = n0;
    fs.cstr = n0;
    fs.jstr = n0;
    k_scale_free<T><<<grid1d(n0, 256), 256, 0, st>>>(
        fs, kernel, n_rhs, tp0, tp1, (const T*)p->ftab[0][2].p, nullptr, (const T*)p->mod0[kidx].p,
        kernel == SE_KERNEL_ST ? (const T*)p->mod0[1].p : nullptr, (T*)b0);
    if (ncolS > 0) {
      fs.m.mode = 1;
      fs.cls = 1;
      fs.ncols = ncolS;
      fs.fn[0] = nS;
      fs.cstr = (long long)ncolS * nS;
      fs.jstr = nS;
      k_scale_free<T><<<grid1d((long long)ncolS * nS, 256), 256, 0, st>>>(
          fs, kernel, n_rhs, tp0, tp1, (const T*)p->ftab[1][2].p, nullptr, nullptr, nullptr, (T*)bS);
    }
    p->scale_modes = (long long)M0 * H1 * Mz + n0 + (long long)std::max(ncolS, 0) * nS;
    stage_event(p, 4);
    // (iv) inverse per class, truncate and merge, inverse over (0, 1)
    SE_CUFFT(FT<T>::c2c(hzi, (T*)spec, (T*)spec, CUFFT_INVERSE));
    SE_CUFFT(FT<T>::c2c(hz0i, (T*)b0, (T*)b0, CUFFT_INVERSE));
    cm.mode = 0;
    k_aft_copy<T><<<grid1d((long long)NC * n0, 256), 256, 0, st>>>(cm, NC, 1, em, e0, false, (T*)spec, (T*)b0);
    if (ncolS > 0) {
      SE_CUFFT(FT<T>::c2c(hzSi, (T*)bS, (T*)bS, CUFFT_INVERSE));
      cm.mode = 1;
      k_aft_copy<T><<<grid1d((long long)NC * ncolS * nS, 256), 256, 0, st>>>(cm, NC, ncolS, em, eS, false,
                                                                             (T*)spec, (T*)bS);
    }
    for (int c = 0; c < NC; ++c) SE_CUFFT(FT<T>::c2r(h2i, (T*)spec + 2 * (size_t)c * S, ugrid + (size_t)c * G));
    SE_CUDA(cudaGetLastError());
    return SE_OK;
  }
  // D = 1: 1-D R2C along direction 0, planes along (1, 2) per class. The grid is direction-0-
  // major, [M0][C][My][Mz], and the spectrum [M0/2+1][CS][My][Mz] (CS component slots per x
  // wavenumber, the scaling writes its NC outputs over the C inputs): the transforms along
  // direction 0 take every component in one call each way, and the planes of every x
  // wavenumber and component are contiguous for the 2-D transforms.
  const int My = g.m[1], Mz = g.m[2];
  const int H0 = M0 / 2 + 1;
  const size_t PL = (size_t)My * Mz;
  const size_t S = (size_t)H0 * PL;
  void* spec;
  SE_TRY(buf(p, "spec", sizeof(T) * 2 * CS * S, &spec));
  int n1[1] = {M0}, in1[1] = {M0}, on1[1] = {H0};
  cufftHandle h1f, h1i;
  SE_TRY(free_fft(p, 20, C * (int)PL, 1, n1, in1, C * (int)PL, 1, on1, CS * (int)PL, 1, FT<T>::R2C, &h1f));
  SE_TRY(free_fft(p, 21, NC * (int)PL, 1, n1, on1, CS * (int)PL, 1, in1, NC * (int)PL, 1, FT<T>::C2R, &h1i));
  SE_CUFFT(FT<T>::r2c(h1f, grid, (T*)spec));
  ColMap cm{1, 0, M0, 0, H0, std::min(p->kbar_star, H0 - 2), CS};
  const int kst = std::max(0, cm.kstar);
  const int n0y = p->ncls[0][1], n0z = p->ncls[0][2], nSy = p->ncls[1][1], nSz = p->ncls[1][2];
  if ((double)CS * std::max(kst, 1) * nSy * nSz >= 2147483647.0 || (double)CS * n0y * n0z >= 2147483647.0)
    return SE_ERR_UNSUPPORTED;  // class buffers are indexed with 32-bit offsets
  void *b0, *bS;
  SE_TRY(buf(p, "aft.b0", sizeof(T) * 2 * CS * (size_t)n0y * n0z, &b0));
  SE_TRY(buf(p, "aft.bS", sizeof(T) * 2 * CS * (size_t)std::max(kst, 1) * nSy * nSz, &bS));
  const Ext2 em{{My, Mz}}, e0{{n0y, n0z}}, eS{{nSy, nSz}};
  cm.mode = 0;
  k_aft_copy<T><<<grid1d((long long)C * n0y * n0z, 256), 256, 0, st>>>(cm, C, 1, em, e0, true, (T*)spec, (T*)b0);
  if (kst > 0) {
    cm.mode = 1;
    k_aft_copy<T><<<grid1d((long long)C * kst * nSy * nSz, 256), 256, 0, st>>>(cm, C, kst, em, eS, true,
                                                                               (T*)spec, (T*)bS);
  }
  int np[2] = {My, Mz}, np0[2] = {n0y, n0z}, npS[2] = {nSy, nSz};
  cufftHandle hp, hpi, hp0, hp0i, hpS, hpSi;
  // every (x wavenumber, component slot) plane: the K_inf class transformed in place (the other
  // classes are taken from their own upsampled buffers; unused slots are transformed harmlessly)
  SE_TRY(free_fft(p, 22, CS * H0, 2, np, nullptr, 1, (int)PL, nullptr, 1, (int)PL, FT<T>::C2C, &hp));
  hpi = hp;
  SE_TRY(free_fft(p, 24, C, 2, np0, nullptr, 1, n0y * n0z, nullptr, 1, n0y * n0z, FT<T>::C2C, &hp0));
  SE_TRY(free_fft(p, 25, NC, 2, np0, nullptr, 1, n0y * n0z, nullptr, 1, n0y * n0z, FT<T>::C2C, &hp0i));
  SE_CUFFT(FT<T>::c2c(hp, (T*)spec, (T*)spec, CUFFT_FORWARD));
  SE_CUFFT(FT<T>::c2c(hp0, (T*)b0, (T*)b0, CUFFT_FORWARD));
  if (kst > 0) {
    SE_TRY(free_fft(p, 26, C * kst, 2, npS, nullptr, 1, nSy * nSz, nullptr, 1, nSy * nSz, FT<T>::C2C, &hpS));
    SE_TRY(free_fft(p, 27, NC * kst, 2, npS, nullptr, 1, nSy * nSz, nullptr, 1, nSy * nSz, FT<T>::C2C, &hpSi));
    SE_CUFFT(FT<T>::c2c(hpS, (T*)bS, (T*)bS, CUFFT_FORWARD));
  }
  stage_event(p, 3);
  FreeScale fs;
  fs.h = g.h;
  fs.kf0 = 2.0 * M_PI / g.L[0];
  fs.kf1 = 0;
  fs.inv4xi2 = 1.0 / (4.0 * p->xi * p->xi);
  const T* tp0 = (const T*)p->ptab[0].p;
  fs.m = cm;
  fs.m.mode = 2;
  fs.cls = 2;
  fs.ncols = H0;
  fs.fn[0] = My;
  fs.fn[1] = Mz;
  fs.cstr = (long long)PL;
  fs.jstr = (long long)CS * PL;
  k_scale_free<T><<<grid1d((long long)H0 * PL, 256), 256, 0, st>>>(
      fs, kernel, n_rhs, tp0, nullptr, (const T*)p->ftab[2][1].p, (const T*)p->ftab[2][2].p, nullptr, nullptr,
      (T*)spec);
  fs.m.mode = 0;
  fs.cls = 0;
  fs.ncols = 1;
  fs.fn[0] = n0y;
  fs.fn[1] = n0z;
  fs.cstr = (long long)n0y * n0z;
  fs.jstr = (long long)n0y * n0z;
  const T* modH = (const T*)(harmonic_family(kernel) ? p->mod0[2].p : p->mod0[0].p);
  const T* modB = (const T*)(harmonic_family(kernel) ? nullptr : p->mod0[1].p);
  k_scale_free<T><<<grid1d((long long)n0y * n0z, 256), 256, 0, st>>>(fs, kernel, n_rhs, tp0, nullptr, nullptr,
                                                                     nullptr, modH, modB, (T*)b0);
  if (kst > 0) {
    fs.m.mode = 1;
    fs.cls = 1;
    fs.ncols = kst;
    fs.fn[0] = nSy;
    fs.fn[1] = nSz;
    fs.cstr = (long long)kst * nSy * nSz;
    fs.jstr = (long long)nSy * nSz;
    k_scale_free<T><<<grid1d((long long)kst * nSy * nSz, 256), 256, 0, st>>>(
        fs, kernel, n_rhs, tp0, nullptr, (const T*)p->ftab[1][1].p, (const T*)p->ftab[1][2].p, nullptr, nullptr,
        (T*)bS);
  }
  p->scale_modes = (long long)H0 * PL + (long long)n0y * n0z + (long long)kst * nSy * nSz;
  stage_event(p, 4);
  SE_CUFFT(FT<T>::c2c(hpi, (T*)spec, (T*)spec, CUFFT_INVERSE));
  SE_CUFFT(FT<T>::c2c(hp0i, (T*)b0, (T*)b0, CUFFT_INVERSE));
  cm.mode = 0;
  k_aft_copy<T><<<grid1d((long long)NC * n0y * n0z, 256), 256, 0, st>>>(cm, NC, 1, em, e0, false, (T*)spec,
                                                                       (T*)b0);
  if (kst > 0) {
    SE_CUFFT(FT<T>::c2c(hpSi, (T*)bS, (T*)bS, CUFFT_INVERSE));
    cm.mode = 1;
    k_aft_copy<T><<<grid1d((long long)NC * kst * nSy * nSz, 256), 256, 0, st>>>(cm, NC, kst, em, eS, false,
                                                                                (T*)spec, (T*)bS);
  }
  SE_CUFFT(FT<T>::c2r(h1i, (T*)spec, ugrid));
  SE_CUDA(cudaGetLastError());
  return SE_OK;
}

long long free_class_elems(const se_plan_t* p) {
  const int k = p->kbar_star;
  if (p->D == 2) {
    const long long ncolS = (2LL * k + 1) * (k + 1) - 1;
    return std::max<long long>(p->ncls[0][2], std::max<long long>(ncolS, 1) * p->ncls[1][2]);
  }
  if (p->D == 1) {
    const int H0 = p->geom.m[0] / 2 + 1;
    const long long kst = std::max(0, std::min(k, H0 - 2));
    return std::max<long long>((long long)p->ncls[0][1] * p->ncls[0][2],
                               std::max<long long>(kst, 1) * p->ncls[1][1] * p->ncls[1][2]);
  }
  return 0;
}

// Gauge constants of the 0P and 1P stokeslet (Eqs. 0p-stokeslet-extra-contribution and
// 1p-stokeslet-extra-contribution): 0P adds (2/R) sum f; 1P subtracts
// diag(4 ln R + 4, 2 ln R + 1, 2 ln R + 1) sum f / L_0.
template <typename T>
se_status gauge_correction(se_plan_t* p, const T* f, int stride, int n, int n_rhs, int nt, T* u) {
  if (!((p->D == 0 || p->D == 1) && n > 0 && nt > 0)) return SE_OK;
  void* sums;
  SE_TRY(buf(p, "gauge.sums", sizeof(double) * 3 * n_rhs, &sums));
  SE_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * 3 * n_rhs, p->stream));
  ++p->launches;
  k_fsum<T><<<std::min(grid1d(n, 256), 152), 256, 0, p->stream>>>(f, stride, 3, n, n_rhs, (double*)sums);
  double c[3];
  if (p->D == 0) {
    c[0] = c[1] = c[2] = 2.0 / p->R;
  } else {
    const double lr = std::log(p->R);
    c[0] = -(4.0 * lr + 4.0) / p->L[0];
    c[1] = c[2] = -(2.0 * lr + 1.0) / p->L[0];
  }
  ++p->launches;
  k_add_const<T><<<grid1d(nt, 256), 256, 0, p->stream>>>(nt, n_rhs, 3, (double*)sums, c[0], c[1], c[2], u);
  SE_CUDA(cudaGetLastError());
  return SE_OK;
}

// The potential of the polynomial p = sum_n c_n r^(2n) (n = 0..3) taken out of the truncated
// biharmonic (SE_FLAG_SPLIT_POLY), added back exactly. For a source at y, the stokeslet and
// stresslet operators map r^(2n), r = x - y, to polynomials in r (the constant c0 to zero);
// expanded in monomials x^a of the target and y^b of the source (tables of se_poly_split.h,
// generated symbolically), the summed potential is a polynomial of degree <= 4 in x:
//   u_j(x) = sum_a C_ja x^a,  C_ja = sum_n c_n sum_(b,k) T_n[j][a][b][k] M[b][k],
//   M[b][k] = sum_sources y^b s_k,  s = f (k = 0..2) or the products q_l nu_m (k = 3 l + m).
// The Fourier part sees p through the Hasimoto screening: convolving a polynomial with the
// radial screening function applies its transform at k^2 = -Lap, 1 - Lap^2/(32 xi^4) -
// Lap^3/(192 xi^6) + ..., so r^2 and r^4 pass unchanged up to constants (annihilated by both
// operators) and r^6 gains -840/(32 xi^4) r^2, which is added to c1. Three kernels: the
// moments (one thread per (b, k), points staged with their monomials in shared memory), the
// coefficients C, and the evaluation at the targets (FP64).
#define SE_PS_STORAGE static __constant__
#include "se_poly_split.h"

constexpr int PS_MS = SE_PS_NMONO * 3;     // stokeslet moments
constexpr int PS_MT = SE_PS_NMONO3 * 9;    // stresslet moments (degree <= 3)
constexpr int PS_NM = PS_MS + PS_MT;       // per RHS
constexpr int PS_TP = 64;                  // points per shared-memory tile

template <typename T>
__global__ void __launch_bounds__(320) k_poly_moments(const double* __restrict__ x, const T* __restrict__ f, int n,
                                                      int cin, int soff, int toff, double* __restrict__ sums) {
  __shared__ T mono[PS_TP][SE_PS_NMONO];
  __shared__ T str[PS_TP][12];
  const int r = blockIdx.y;
  const int t = threadIdx.x;
  // this thread's moment: (b, k) of the stokeslet or of the stresslet part
  const bool ms = t < PS_MS, mt = t >= PS_MS && t < PS_NM;
  const int b = ms ? t / 3 : (t - PS_MS) / 9, kk = ms ? t % 3 : 3 + (t - PS_MS) % 9;
  const bool active = (ms && soff >= 0) || (mt && toff >= 0);
  double acc = 0.0;
  for (int base = blockIdx.x * PS_TP; base < n; base += gridDim.x * PS_TP) {
    __syncthreads();
    for (int e = t; e < PS_TP * (SE_PS_NMONO + 12); e += blockDim.x) {
      const int pnt = e / (SE_PS_NMONO + 12), c = e % (SE_PS_NMONO + 12);
      const int i = base + pnt;
      T v = T(0);
      if (i < n) {
        if (c < SE_PS_NMONO) {
          const T y0 = (T)x[3 * i], y1 = (T)x[3 * i + 1], y2 = (T)x[3 * i + 2];
          v = T(1);
          for (int q = 0; q < se_ps_mono[c][0]; ++q) v *= y0;
          for (int q = 0; q < se_ps_mono[c][1]; ++q) v *= y1;
          for (int q = 0; q < se_ps_mono[c][2]; ++q) v *= y2;
          mono[pnt][c] = v;
          continue;
        }
        const int s = c - SE_PS_NMONO;
        const T* fi = f + ((size_t)r * n + i) * cin;
        if (s < 3) v = soff >= 0 ? fi[soff + s] : T(0);
        else v = toff >= 0 ? fi[toff + (s - 3) / 3] * fi[toff + 3 + (s - 3) % 3] : T(0);
      } else if (c < SE_PS_NMONO) {
        mono[pnt][c] = T(0);
        continue;
      }
      str[pnt][c - SE_PS_NMONO] = v;
    }
    __syncthreads();
    if (active) {
      const int np = min(PS_TP, n - base);
      T part = T(0);
      for (int pnt = 0; pnt < np; ++pnt) part += mono[pnt][b] * str[pnt][kk];
      acc += (double)part;
    }
  }
  if (active && acc != 0.0) atomicAdd(&sums[(size_t)r * PS_NM + t], acc);
}

// C[r][j][a] = sum over the table rows of c_n T M (one thread per (RHS, j, a))
__global__ void k_poly_coeffs(const double* __restrict__ sums, int n_rhs, int has_s, int has_t, double c1,
                              double c2, double c3, double* __restrict__ C) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_rhs * 3 * SE_PS_NMONO) return;
  const int r = id / (3 * SE_PS_NMONO), j = (id / SE_PS_NMONO) % 3, a = id % SE_PS_NMONO;
  const double cn[4] = {0.0, c1, c2, c3};
  const double* M = sums + (size_t)r * PS_NM;
  double v = 0.0;
  if (has_s)
    for (int q = 0; q < SE_PS_NS; ++q) {
      const SePsTerm& e = se_ps_stokeslet[q];
      if (e.j == j && e.a == a) v += cn[e.n] * e.c * M[e.b * 3 + e.k];
    }
  if (has_t)
    for (int q = 0; q < SE_PS_NT; ++q) {
      const SePsTerm& e = se_ps_stresslet[q];
      if (e.j == j && e.a == a) v += cn[e.n] * e.c * M[PS_MS + e.b * 9 + e.k];
    }
  C[id] = v;
}

template <typename T>
__global__ void k_poly_apply(const double* __restrict__ t, int nt, int n_rhs, const double* __restrict__ C,
                             T* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nt) return;
  const double x0 = t[3 * i], x1 = t[3 * i + 1], x2 = t[3 * i + 2];
  double xm[SE_PS_NMONO];
#pragma unroll
  for (int a = 0; a < SE_PS_NMONO; ++a) {
    double v = 1.0;
    for (int q = 0; q < se_ps_mono[a][0]; ++q) v *= x0;
    for (int q = 0; q < se_ps_mono[a][1]; ++q) v *= x1;
    for (int q = 0; q < se_ps_mono[a][2]; ++q) v *= x2;
    xm[a] = v;
  }
  for (int r = 0; r < n_rhs; ++r)
    for (int j = 0; j < 3; ++j) {
      const double* c = C + ((size_t)r * 3 + j) * SE_PS_NMONO;
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < SE_PS_NMONO; ++a) v += c[a] * xm[a];
      u[((size_t)r * nt + i) * 3 + j] += (T)v;
    }
}

template <typename T>
se_status poly_correction(se_plan_t* p, int kernel, const double* x, const T* f, int n, int n_rhs, const double* t,
                          int nt, T* u) {
  if (!p->poly_on || p->D != 0 || n <= 0 || nt <= 0) return SE_OK;
  const int has_s = (kernel & SE_STOKESLET) ? 1 : 0, has_t = (kernel & SE_STRESSLET) ? 1 : 0;
  if (!has_s && !has_t) return SE_OK;
  void *sums, *coef;
  SE_TRY(buf(p, "poly.sums", sizeof(double) * PS_NM * n_rhs, &sums));
  SE_TRY(buf(p, "poly.coef", sizeof(double) * 3 * SE_PS_NMONO * n_rhs, &coef));
  SE_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * PS_NM * n_rhs, p->stream));
  const int cin = kernel_comps(kernel);
  const int soff = has_s ? 0 : -1, toff = has_t ? (has_s ? 3 : 0) : -1;
  const double xi2 = p->xi * p->xi;
  const double c1 = p->poly_c[1] - 840.0 / 32.0 * p->poly_c[3] / (xi2 * xi2);
  ++p->launches;
  dim3 gr(std::min(std::max((n + PS_TP - 1) / PS_TP, 1), 152 * 2), n_rhs);
  k_poly_moments<T><<<gr, 320, 0, p->stream>>>(x, f, n, cin, soff, toff, (double*)sums);
  ++p->launches;
  k_poly_coeffs<<<grid1d(3LL * SE_PS_NMONO * n_rhs, 128), 128, 0, p->stream>>>(
      (const double*)sums, n_rhs, has_s, has_t, c1, p->poly_c[2], p->poly_c[3], (double*)coef);
  ++p->launches;
  k_poly_apply<T><<<grid1d(nt, 256), 256, 0, p->stream>>>(t, nt, n_rhs, (const double*)coef, u);
  SE_CUDA(cudaGetLastError());
  return SE_OK;
}

// Constants of the harmonic potential: 3P adds -pi Q / (xi^2 V) (the zero-mean potential: the
// real-space kernel erfc(xi r)/r carries pi / xi^2 of k = 0 content per charge); 1P subtracts
// 2 log(R) Q / L_0 (the k_1 = 0 class used -2 log(rho / R), the reported gauge is l_H = 1);
// Q = sum q per right-hand side. 2P and 0P need none.
template <typename T>
se_status harmonic_constant(se_plan_t* p, const T* q, int n, int n_rhs, int nt, T* u) {
  if (!((p->D == 3 || p->D == 1) && n > 0 && nt > 0)) return SE_OK;
  void* sums;
  SE_TRY(buf(p, "gauge.sums", sizeof(double) * 3 * n_rhs, &sums));
  SE_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * 3 * n_rhs, p->stream));
  ++p->launches;
  k_fsum<T><<<std::min(grid1d(n, 256), 152), 256, 0, p->stream>>>(q, 1, 1, n, n_rhs, (double*)sums);
  const double c = p->D == 3 ? -M_PI / (p->xi * p->xi * p->L[0] * p->L[1] * p->L[2])
                             : -2.0 * std::log(p->R) / p->L[0];
  ++p->launches;
  k_add_const<T><<<grid1d(nt, 256), 256, 0, p->stream>>>(nt, n_rhs, 1, (double*)sums, c, 0.0, 0.0, u);
  SE_CUDA(cudaGetLastError());
  return SE_OK;
}

template se_status fourier_free<float>(se_plan_t*, int, int, float*, int, float*, int);
template se_status fourier_free<double>(se_plan_t*, int, int, double*, int, double*, int);
template se_status gauge_correction<float>(se_plan_t*, const float*, int, int, int, int, float*);
template se_status gauge_correction<double>(se_plan_t*, const double*, int, int, int, int, double*);
template se_status harmonic_constant<float>(se_plan_t*, const float*, int, int, int, float*);
template se_status poly_correction<float>(se_plan_t*, int, const double*, const float*, int, int, const double*, int,
                                          float*);
template se_status poly_correction<double>(se_plan_t*, int, const double*, const double*, int, int, const double*,
                                           int, double*);
template se_status harmonic_constant<double>(se_plan_t*, const double*, int, int, int, double*);

}  // namespace se
