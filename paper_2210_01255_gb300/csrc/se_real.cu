// libse real-space part, Eq. (real-space-potential-Dp) with the kernels of Eqs.
// (stokeslet-real), (rotlet-real), (stresslet-real) and the self term of Eq. (self-term):
// the sum over sources within r_c of each target (periodic images in the periodic
// directions), on a cell list of sorted points. Two kernels:
//   k_real      a warp per target (sparse neighbourhoods): candidate columns of the cell list
//               walked by the lanes, pairs inside r_c compacted into a per-warp ring;
//   k_real_blk  a warp per block of 32 spatially close targets (dense neighbourhoods): the
//               candidates of the whole block are staged in shared memory 32 at a time and
//               every lane tests and evaluates them against its own target.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "se_device.cuh"
#include "se_erfc_fit.h"

namespace se {

// ====================================== real-space sum, Eq. (real-space-potential-Dp)
//
// Cell list of cells with side >= rc / S (S = range); one thread per target looping over
// the (2S+1)^3 neighbour cells with periodic images in the periodic directions. A pair at
// exactly zero separation is the omitted self interaction of the star sum: it contributes
// the self term -G^F(0) . f (Eq. self-term) instead, so the star form and explicit
// coincident targets agree.


// erfc(x), x >= 0, given g = exp(-x^2) (computed anyway for the Gaussian terms).
// FP32: erfc(x) = g t R(t), t = 1 / (1 + a x), R the degree-10 polynomial of se_erfc_fit.h
// (relative error of the fit < 1e-8; a few FP32 ulp after rounding). FP64: the library erfc.
template <typename T>
__device__ inline T dev_erfc_g(T x, T g);
template <> __device__ __forceinline__ float dev_erfc_g<float>(float x, float g) {
  const float t = __fdividef(1.0f, fmaf(float(SE_ERFC_FIT_A), x, 1.0f));  // fast reciprocal, ~1 ulp
  float r = float(SE_ERFC_FIT_C10);
  r = fmaf(r, t, float(SE_ERFC_FIT_C9));
  r = fmaf(r, t, float(SE_ERFC_FIT_C8));
  r = fmaf(r, t, float(SE_ERFC_FIT_C7));
  r = fmaf(r, t, float(SE_ERFC_FIT_C6));
  r = fmaf(r, t, float(SE_ERFC_FIT_C5));
  r = fmaf(r, t, float(SE_ERFC_FIT_C4));
  r = fmaf(r, t, float(SE_ERFC_FIT_C3));
  r = fmaf(r, t, float(SE_ERFC_FIT_C2));
  r = fmaf(r, t, float(SE_ERFC_FIT_C1));
  r = fmaf(r, t, float(SE_ERFC_FIT_C0));
  return g * (t * r);
}
template <> __device__ __forceinline__ double dev_erfc_g<double>(double x, double) { return erfc(x); }

// exp(a) for the Gaussian factor exp(-xi^2 r^2), a in [-xi^2 r_c^2, 0]: FP32 takes the hardware
// exponential (a few ulp on this range, far below the FP32 path's tolerance), FP64 the library
__device__ __forceinline__ float gauss(float a) { return __expf(a); }
__device__ __forceinline__ double gauss(double a) { return exp(a); }

// One pair (target, source image): accumulate G^R(r) . f into acc, or the self term when
// the separation is exactly zero (the omitted n = m, p = 0 term of the star sum).
template <typename T, int KERNEL, int RMAX>
__device__ __forceinline__ void real_pair(T r0, T r1, T r2, T rr2, T xi, T xi2, T c2pi, const T* __restrict__ f,
                                          int n_rhs, T* acc) {
  if (rr2 == T(0)) {
    if (KERNEL == SE_HARMONIC) {
#pragma unroll
      for (int r = 0; r < RMAX; ++r)
        if (r < n_rhs) acc[r] -= c2pi * f[r];  // -2 xi / sqrt(pi) q
    }
    if (KERNEL == SE_STOKESLET || KERNEL == SE_KERNEL_ST) {
      const T cs = -T(2) * c2pi;  // -4 xi / sqrt(pi), Eq. (3p-stokeslet-self-term)
      constexpr int STRIDE = KERNEL == SE_KERNEL_ST ? 9 : 3;
#pragma unroll
      for (int r = 0; r < RMAX; ++r)
        if (r < n_rhs)
          for (int q = 0; q < 3; ++q) acc[3 * r + q] += cs * f[STRIDE * r + q];
    }
    return;
  }
  const T inv = rsqrt(rr2);
  const T rn = rr2 * inv;
  const T inv2 = inv * inv;
  const T e = gauss(-xi2 * rr2);
  const T ec = dev_erfc_g(xi * rn, e) * inv;
  if (KERNEL == SE_HARMONIC) {
    // the Ewald-screened harmonic kernel erfc(xi r) / r times q (one output per RHS)
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < n_rhs) acc[r] += ec * f[r];
  } else if (KERNEL == SE_STOKESLET) {
    // Eq. (stokeslet-real): (delta + r r / r^2)(erfc/r + 2 xi e/sqrt pi) - delta 4 xi e/sqrt pi
    const T c1 = ec + c2pi * e;
    const T c0 = c1 - T(2) * c2pi * e;
    const T c1i = c1 * inv2;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        const T* fr = f + 3 * r;
        const T rf = (r0 * fr[0] + r1 * fr[1] + r2 * fr[2]) * c1i;
        acc[3 * r + 0] += c0 * fr[0] + r0 * rf;
        acc[3 * r + 1] += c0 * fr[1] + r1 * rf;
        acc[3 * r + 2] += c0 * fr[2] + r2 * rf;
      }
    }
  } else if (KERNEL == SE_HARMONIC_FIELD) {
    // -grad of the screened harmonic kernel erfc(xi r)/r: r_j / r^2 (erfc/r + 2 xi e/sqrt pi) q
    // (the rotlet's radial factor, Eq. rotlet-real, with the gradient in place of the curl)
    const T c1 = (ec + c2pi * e) * inv2;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        const T cq = c1 * f[r];
        acc[3 * r + 0] += cq * r0;
        acc[3 * r + 1] += cq * r1;
        acc[3 * r + 2] += cq * r2;
      }
    }
  } else if (KERNEL == SE_ROTLET) {
    // Eq. (rotlet-real): eps_jlm r_m / r^2 (erfc/r + 2 xi e/sqrt pi) f_l = (f x r)_j c
    const T c1 = (ec + c2pi * e) * inv2;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        const T* fr = f + 3 * r;
        acc[3 * r + 0] += c1 * (fr[1] * r2 - fr[2] * r1);
        acc[3 * r + 1] += c1 * (fr[2] * r0 - fr[0] * r2);
        acc[3 * r + 2] += c1 * (fr[0] * r1 - fr[1] * r0);
      }
    }
  } else {
    // Eq. (stresslet-real): -2 r_j r_l r_m / r^4 (3 erfc/r + (3 + 2 xi^2 r^2) 2 xi e/sqrt pi)
    //   + (delta_jl r_m + delta_mj r_l + delta_lm r_j) 4 xi^3 e / sqrt pi
    // (S|T: the stokeslet term of Eq. stokeslet-real on f as above, then this on (q, nu))
    constexpr int STRIDE = KERNEL == SE_KERNEL_ST ? 9 : 6;
    constexpr int QOFF = KERNEL == SE_KERNEL_ST ? 3 : 0;
    if (KERNEL == SE_KERNEL_ST) {
      const T c1 = ec + c2pi * e;
      const T c0 = c1 - T(2) * c2pi * e;
      const T c1i = c1 * inv2;
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        if (r < n_rhs) {
          const T* fr = f + STRIDE * r;
          const T rf = (r0 * fr[0] + r1 * fr[1] + r2 * fr[2]) * c1i;
          acc[3 * r + 0] += c0 * fr[0] + r0 * rf;
          acc[3 * r + 1] += c0 * fr[1] + r1 * rf;
          acc[3 * r + 2] += c0 * fr[2] + r2 * rf;
        }
      }
    }
    const T A = T(3) * ec + (T(3) + T(2) * xi2 * rr2) * c2pi * e;
    const T B = T(2) * xi2 * c2pi * e;
    const T Ai = -T(2) * A * inv2 * inv2;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        const T* q = f + STRIDE * r + QOFF;
        const T* nu = q + 3;
        const T rq = r0 * q[0] + r1 * q[1] + r2 * q[2];
        const T rnu = r0 * nu[0] + r1 * nu[1] + r2 * nu[2];
        const T qn = q[0] * nu[0] + q[1] * nu[1] + q[2] * nu[2];
        const T c3 = Ai * rq * rnu + qn * B;
        const T bq = B * rnu, bn = B * rq;
        acc[3 * r + 0] += c3 * r0 + bq * q[0] + bn * nu[0];
        acc[3 * r + 1] += c3 * r1 + bq * q[1] + bn * nu[1];
        acc[3 * r + 2] += c3 * r2 + bq * q[2] + bn * nu[2];
      }
    }
  }
}

// The pair terms of real_pair without branches, for a pair that may or may not count: the
// radial coefficients are formed from a safe r^2 and then kept (a pair inside r_c at r > 0),
// replaced by the self term (r = 0, the omitted star-sum term: the stokeslet's -4 xi/sqrt(pi)
// f, the harmonic potential's -2 xi/sqrt(pi) q, nothing for the other kernels) or zeroed
// (outside r_c). Same arithmetic as real_pair for
// a pair that counts; with no branch, the terms of two candidates interleave (k_real_blk).
// QNPRE: the stresslet's q . nu of RHS r is staged at f[STRIDE RMAX + r] (k_real_blk).
template <typename T, int KERNEL, int RMAX, bool QNPRE = false>
__device__ __forceinline__ void real_pair_m(T r0, T r1, T r2, T rr2, bool inside, T xi, T xi2, T c2pi,
                                            const T* __restrict__ f, int n_rhs, T* acc) {
  const bool reg = inside && rr2 > T(0);
  const bool self = inside && rr2 == T(0);
  const T q2 = reg ? rr2 : T(1);
  const T inv = rsqrt(q2);
  const T rn = q2 * inv;
  const T inv2 = inv * inv;
  const T e = gauss(-xi2 * q2);
  const T ec = dev_erfc_g(xi * rn, e) * inv;
  if (KERNEL == SE_STOKESLET || KERNEL == (SE_STOKESLET | SE_STRESSLET)) {
    constexpr int STRIDE = KERNEL == SE_STOKESLET ? 3 : 9;
    const T c1 = ec + c2pi * e;
    T c0 = c1 - T(2) * c2pi * e;
    c0 = reg ? c0 : (self ? -T(2) * c2pi : T(0));
    const T c1i = reg ? c1 * inv2 : T(0);
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        const T* fr = f + STRIDE * r;
        const T rf = (r0 * fr[0] + r1 * fr[1] + r2 * fr[2]) * c1i;
        acc[3 * r + 0] += c0 * fr[0] + r0 * rf;
        acc[3 * r + 1] += c0 * fr[1] + r1 * rf;
        acc[3 * r + 2] += c0 * fr[2] + r2 * rf;
      }
    }
  }
  if (KERNEL == SE_HARMONIC) {
    const T c0 = reg ? ec : (self ? -c2pi : T(0));
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < n_rhs) acc[r] += c0 * f[r];
  }
  if (KERNEL == SE_HARMONIC_FIELD || KERNEL == SE_ROTLET) {
    const T c1 = reg ? (ec + c2pi * e) * inv2 : T(0);
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        if (KERNEL == SE_HARMONIC_FIELD) {
          const T cq = c1 * f[r];
          acc[3 * r + 0] += cq * r0;
          acc[3 * r + 1] += cq * r1;
          acc[3 * r + 2] += cq * r2;
        } else {
          const T* fr = f + 3 * r;
          acc[3 * r + 0] += c1 * (fr[1] * r2 - fr[2] * r1);
          acc[3 * r + 1] += c1 * (fr[2] * r0 - fr[0] * r2);
          acc[3 * r + 2] += c1 * (fr[0] * r1 - fr[1] * r0);
        }
      }
    }
  }
  if (KERNEL == SE_STRESSLET || KERNEL == (SE_STOKESLET | SE_STRESSLET)) {
    constexpr int STRIDE = KERNEL == SE_STRESSLET ? 6 : 9;
    constexpr int QOFF = KERNEL == SE_STRESSLET ? 0 : 3;
    const T A = T(3) * ec + (T(3) + T(2) * xi2 * q2) * c2pi * e;
    const T B = reg ? T(2) * xi2 * c2pi * e : T(0);
    const T Ai = reg ? -T(2) * A * inv2 * inv2 : T(0);
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < n_rhs) {
        const T* q = f + STRIDE * r + QOFF;
        const T* nu = q + 3;
        const T rq = r0 * q[0] + r1 * q[1] + r2 * q[2];
        const T rnu = r0 * nu[0] + r1 * nu[1] + r2 * nu[2];
        const T qn = QNPRE ? f[STRIDE * RMAX + r] : q[0] * nu[0] + q[1] * nu[1] + q[2] * nu[2];
        const T c3 = Ai * rq * rnu + qn * B;
        const T bq = B * rnu, bn = B * rq;
        acc[3 * r + 0] += c3 * r0 + bq * q[0] + bn * nu[0];
        acc[3 * r + 1] += c3 * r1 + bq * q[1] + bn * nu[1];
        acc[3 * r + 2] += c3 * r2 + bq * q[2] + bn * nu[2];
      }
    }
  }
}

// Real-space sum: one warp per target.
// (1) Column table: the neighbour columns of the target's cell (along direction 2, trimmed to
//     the cells that can hold sources within rc, split at periodic images into contiguous
//     source ranges, "segments") are set up one column per lane, all cstart loads in flight
//     at once; a warp scan lays the segments out as one flat candidate list.
// (2) Candidates: the warp walks the flat list U x 32 at a time (U = 2 independent loads per
//     lane), tests them on the hi parts and compacts the ones inside rc (ballot + popc) into a
//     per-warp ring of pairs.
// (3) Pairs: whenever 32 are queued they are evaluated one per lane with the exact hi + lo
//     separation. Lane partial sums are combined by shuffles.
// More than 32 columns (or more segments than the table holds) are done in rounds.
constexpr int RS_WARPS = 4;    // warps per CTA
constexpr int RS_SEGCAP = 64;  // column segments per round
constexpr int RS_RING = 256;   // pair ring entries (power of two, >= 32 (RS_U + 1))
template <typename T>
struct RsU {  // candidate chunks of 32 in flight per lane
  static constexpr int value = 2;  // 4 in FP32 measured 5 % slower (registers, occupancy)
};

template <typename T>
struct RealSmem {
  typename Vec4<T>::type seg[RS_SEGCAP];  // image shift (x, y, z); w: first source - flat start
  int start[RS_SEGCAP + 1];              // flat start of each segment (+ total)
  int len[RS_SEGCAP];
  int pk[RS_SEGCAP];                     // packed image numbers (3 x 8 bits, biased by 128)
  int ring_j[RS_RING];
  int ring_pk[RS_RING];
};

__device__ __forceinline__ float ipack(int v, float) { return __int_as_float(v); }
__device__ __forceinline__ double ipack(int v, double) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int iunpack(float v) { return __float_as_int(v); }
__device__ __forceinline__ int iunpack(double v) { return (int)__double_as_longlong(v); }

// wrap an unwrapped cell index into [0, n) and return the image number
__device__ __forceinline__ int wrap_cell(int u, int n, int* im) {
  int k = 0;
  while (u < 0) { u += n; --k; }
  while (u >= n) { u -= n; ++k; }
  *im = k;
  return u;
}

// outputs per target and RHS (the harmonic potential is a scalar)
template <int KERNEL>
struct RsOut {
  static constexpr int value = KERNEL == SE_HARMONIC ? 1 : 3;
};

template <typename T, int KERNEL, int RMAX>
__global__ void __launch_bounds__(32 * RS_WARPS) k_real(RealArgs<T> a) {
  constexpr int NO = RsOut<KERNEL>::value;
  __shared__ RealSmem<T> sm_all[RS_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int s = blockIdx.x * RS_WARPS + warp;
  if (a.tlist) {  // a list of the sorted targets to evaluate (the others go to k_real_blk)
    if (s >= *a.tcount) return;  // warp-uniform
    s = a.tlist[s];
  } else if (s >= a.ntgt) {
    return;  // warp-uniform
  }
  RealSmem<T>& sm = sm_all[warp];
  typedef typename Vec4<T>::type V4;
  const V4 xt = a.xt[s];
  V4 xtl;
  xtl.x = xtl.y = xtl.z = xtl.w = T(0);
  if (sizeof(T) == 4) xtl = a.xtl[s];
  const int cx = a.tcell[3 * s], cy = a.tcell[3 * s + 1], cz = a.tcell[3 * s + 2];
  // a group evaluation: the cells of this target's configuration (sorted by configuration first)
  const int cfgcell = group_of(a.cg.gr, s) * (a.cg.nc[0] * a.cg.nc[1] * a.cg.nc[2]);
  const int nc = kernel_comps(KERNEL);
  const int C = nc * a.n_rhs;
  T acc[NO * RMAX];
#pragma unroll
  for (int k = 0; k < NO * RMAX; ++k) acc[k] = T(0);
  const T xi = a.xi;
  const T xi2 = xi * xi;
  const T c2pi = T(2.0 / 1.7724538509055160273) * xi;  // 2 xi / sqrt(pi)
  const CellGeom& g = a.cg;
  // candidate pre-test on the hi parts with a slightly larger radius; the exact test runs
  // on the hi + lo separation when the pair is evaluated
  const T cs0 = a.Lhi[0] / T(g.nc[0]), cs1 = a.Lhi[1] / T(g.nc[1]), cs2 = a.Lhi[2] / T(g.nc[2]);
  const T rcp2 = a.rc2 * T(1.0001) + T(1e-12);
  const T tx = xt.x, ty = xt.y, tz = xt.z;
  const T inv_cs2 = T(g.nc[2]) / a.Lhi[2];
  unsigned head = 0, tail = 0;  // pair ring [head, tail)
  // evaluate the pairs ring[head .. head + cnt) (cnt <= 32), one per lane
  // evaluate the queued pairs [0, cnt) (cnt <= 32), one per lane
  auto flush = [&](int cnt) {
    __syncwarp();
    if (lane < cnt) {
      const int e = (head + lane) & (RS_RING - 1);
      const int j = sm.ring_j[e], pk = sm.ring_pk[e];
      const T i0 = T((pk & 255) - 128), i1 = T(((pk >> 8) & 255) - 128), i2 = T(((pk >> 16) & 255) - 128);
      const V4 xs = a.xs[j];
      T r0, r1, r2;
      if (sizeof(T) == 4) {
        // r = x_target - (x_source + p): hi + lo parts, x_source_hi + shift split exactly
        const V4 xl = a.xsl[j];
        const T shx = i0 * a.Lhi[0], shy = i1 * a.Lhi[1], shz = i2 * a.Lhi[2];
        const T ax = xs.x + shx, ay = xs.y + shy, az = xs.z + shz;
        const T ex = xs.x - (ax - shx), ey = xs.y - (ay - shy), ez = xs.z - (az - shz);
        r0 = (xt.x - ax) + ((xtl.x - xl.x) - (i0 * a.Llo[0] + ex));
        r1 = (xt.y - ay) + ((xtl.y - xl.y) - (i1 * a.Llo[1] + ey));
        r2 = (xt.z - az) + ((xtl.z - xl.z) - (i2 * a.Llo[2] + ez));
      } else {
        r0 = xt.x - (xs.x + i0 * a.Lhi[0]);
        r1 = xt.y - (xs.y + i1 * a.Lhi[1]);
        r2 = xt.z - (xs.z + i2 * a.Lhi[2]);
      }
      const T rr2 = r0 * r0 + r1 * r1 + r2 * r2;
      if (rr2 < a.rc2)
        real_pair<T, KERNEL, RMAX>(r0, r1, r2, rr2, xi, xi2, c2pi, a.fs + (size_t)j * C, a.n_rhs, acc);
    }
    __syncwarp();
  };
  const unsigned FULL = 0xffffffffu;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int rx = g.range[0], ry = g.range[1];
  const int ncy = 2 * ry + 1, ncol = (2 * rx + 1) * ncy;
  const int maxseg = a.maxseg, cpr = a.cols_per_round;
  for (int c0 = 0; c0 < ncol; c0 += cpr) {
    // ---- (1) segments of columns c0 .. c0 + cpr - 1, column c0 + lane on this lane
    __syncwarp();
    const int slot0 = lane * maxseg;
    int nseg = 0, tot = 0;
    const int k = c0 + lane;
    if (lane < cpr && k < ncol) {
      const int kx = k / ncy;
      const int dx = kx - rx, dy = k - kx * ncy - ry;
      int imx = 0, imy = 0, ux = cx + dx, uy = cy + dy;
      bool ok = true;
      if (g.periodic[0]) ux = wrap_cell(ux, g.nc[0], &imx);
      else ok = ux >= 0 && ux < g.nc[0];
      if (g.periodic[1]) uy = wrap_cell(uy, g.nc[1], &imy);
      else ok = ok && uy >= 0 && uy < g.nc[1];
      if (ok) {
        // distance from the target to this image of the column, directions 0 and 1
        const T x0 = T(cx + dx) * cs0, x1 = x0 + cs0;
        const T ddx = tx < x0 ? x0 - tx : (tx > x1 ? tx - x1 : T(0));
        const T y0 = T(cy + dy) * cs1, y1 = y0 + cs1;
        const T ddy = ty < y0 ? y0 - ty : (ty > y1 ? ty - y1 : T(0));
        const T rem = rcp2 - ddx * ddx - ddy * ddy;
        if (rem > T(0)) {
          // cells along direction 2 that can hold sources within rc: |z - tz| < sqrt(rem)
          const T zr = sqrt(rem);
          int zlo = (int)floor((tz - zr) * inv_cs2), zend = (int)floor((tz + zr) * inv_cs2);
          zlo = max(zlo, cz - g.range[2]);
          zend = min(zend, cz + g.range[2]);
          if (!g.periodic[2]) {
            zlo = max(zlo, 0);
            zend = min(zend, g.nc[2] - 1);
          }
          const T shx = T(imx) * a.Lhi[0], shy = T(imy) * a.Lhi[1];
          const int colbase = cfgcell + (ux * g.nc[1] + uy) * g.nc[2];
          while (zlo <= zend && nseg < maxseg) {
            int imz = 0, w0 = zlo;
            if (g.periodic[2]) w0 = wrap_cell(zlo, g.nc[2], &imz);
            const int w1 = min(g.nc[2] - 1, w0 + (zend - zlo));  // up to the end of this image
            const int beg = a.cstart[colbase + w0], end = a.cstart[colbase + w1 + 1];
            V4 sg;
            sg.x = shx;
            sg.y = shy;
            sg.z = T(imz) * a.Lhi[2];
            sg.w = ipack(beg, T());
            sm.seg[slot0 + nseg] = sg;
            sm.len[slot0 + nseg] = end - beg;
            sm.pk[slot0 + nseg] = (imx + 128) | ((imy + 128) << 8) | ((imz + 128) << 16);
            tot += end - beg;
            ++nseg;
            zlo += w1 - w0 + 1;
          }
        }
      }
    }
    if (lane < cpr)
      for (int i = nseg; i < maxseg; ++i) sm.len[slot0 + i] = 0;
    int inc = tot;  // inclusive warp scan of the per-column candidate counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(FULL, inc, off);
      if (lane >= off) inc += v;
    }
    const int total = __shfl_sync(FULL, inc, 31);
    __syncwarp();
    if (lane < cpr) {
      int run = inc - tot;
      for (int i = 0; i < maxseg; ++i) {
        const int sl = slot0 + i;
        sm.start[sl] = run;
        if (i < nseg) sm.seg[sl].w = ipack(iunpack(sm.seg[sl].w) - run, T());
        run += sm.len[sl];
      }
    }
    if (lane == 0) sm.start[cpr * maxseg] = total;
    __syncwarp();
    // ---- (2) candidates of the flat list, RS_U x 32 per pass
    int sp = 0;  // this lane's segment (monotone along the list)
    constexpr int RS_U = RsU<T>::value;
    for (int b0 = 0; b0 < total; b0 += 32 * RS_U) {
      int jj[RS_U], sv[RS_U];
      V4 xv[RS_U];
      T sx[RS_U], sy[RS_U], sz[RS_U];
#pragma unroll
      for (int u = 0; u < RS_U; ++u) {
        const int f = b0 + 32 * u + lane;
        sv[u] = -1;
        if (f < total) {
          while (sm.start[sp + 1] <= f) ++sp;
          const V4 sg = sm.seg[sp];
          sv[u] = sp;
          jj[u] = iunpack(sg.w) + f;
          sx[u] = sg.x;
          sy[u] = sg.y;
          sz[u] = sg.z;
          xv[u] = a.xs[jj[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < RS_U; ++u) {
        bool in = false;
        if (sv[u] >= 0) {
          const T r0 = tx - (xv[u].x + sx[u]), r1 = ty - (xv[u].y + sy[u]), r2 = tz - (xv[u].z + sz[u]);
          in = r0 * r0 + r1 * r1 + r2 * r2 < rcp2;
        }
        const unsigned bal = __ballot_sync(FULL, in);
        if (in) {
          const int e = (tail + __popc(bal & lt_mask)) & (RS_RING - 1);
          sm.ring_j[e] = jj[u];
          sm.ring_pk[e] = sm.pk[sv[u]];
        }
        tail += __popc(bal);
      }
      // ---- (3) pairs, 32 at a time
      while (tail - head >= 32u) {
        flush(32);
        head += 32;
      }
    }
  }
  if (tail != head) flush((int)(tail - head));
#pragma unroll
  for (int k = 0; k < NO * RMAX; ++k) {
    T v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    acc[k] = v;
  }
  if (lane == 0) {
    const int i = a.tperm[s];
    for (int r = 0; r < a.n_rhs && r < RMAX; ++r)
      for (int qq = 0; qq < NO; ++qq) {
        T* o = a.u + out_index(a.cg.gr, a.n_rhs, NO, a.ntgt, i, r, qq);
        *o = a.overwrite ? acc[NO * r + qq] : *o + acc[NO * r + qq];
      }
  }
}

// Segment-table layout of a real-space launch: segments per column (periodic direction 2
// splits a column at each image boundary) and columns per round.
template <typename T>
se_status real_seg_setup(RealArgs<T>& ra) {
  const CellGeom& g = ra.cg;
  int maxseg = 1;
  if (g.periodic[2]) maxseg = (2 * g.range[2] + 1 + g.nc[2] - 1) / g.nc[2] + 1;
  if (maxseg > RS_SEGCAP) return SE_ERR_UNSUPPORTED;
  ra.maxseg = maxseg;
  ra.cols_per_round = std::min(32, RS_SEGCAP / maxseg);
  return SE_OK;
}

// ================================================== dense neighbourhoods: k_real_blk
//
// A warp owns a block of up to 32 consecutive cell-sorted targets (lane = target) whose
// positions lie in a small box. Its candidate sources are the cells within r_c of that box:
// columns along direction 2 trimmed to the box's r_c neighbourhood, one lane per column, laid
// out as one flat list by a warp scan (as in k_real). The list is streamed in chunks of 32:
// each lane loads one candidate (position and strengths) into registers one chunk ahead and
// stores it into the warp's staging area, then every lane runs over the staged chunk,
// reading each source as a shared-memory broadcast, and adds the pairs within r_c of its
// own target into a chunk partial that is folded into the target's sum with Kahan
// compensation (FP32), so that sums over 1e5 neighbours keep FP32 accuracy.
// Separations are formed as in k_real: a staged source holds its image position a = x_hi +
// shift (FP32) and the remainder lo = x_lo + shift_lo + (the rounding of that addition), so
// r = (t_hi - a) + (t_lo - lo), whose leading difference is exact for nearby points: FP32
// separations carry a few ulp of relative error however close the points are. A source that
// coincides with a target gives exactly r = 0: the self term, as in k_real.

constexpr int RB_WARPS = 4;    // warps per CTA
constexpr int RB_SEGCAP = 64;  // column segments per round

template <typename T, int CP>
struct BlkSmem {
  typename Vec4<T>::type pos[32];  // staged chunk: image positions (hi parts)
  typename Vec4<T>::type low[32];  // staged chunk: the remainders
  T str[32][CP];                   // staged chunk: strengths
  int beg[RB_SEGCAP];              // first sorted source of each segment
  int start[RB_SEGCAP + 1];        // flat start of each segment (+ total)
  int len[RB_SEGCAP];
  int pk[RB_SEGCAP];               // packed image numbers (3 x 8 bits, biased by 128)
};

// strengths per source: c (kernel) x n_rhs, padded to a multiple of 4 for the staging area
template <int KERNEL, int RMAX>
struct BlkComps {
  static constexpr int c = KERNEL == SE_STRESSLET ? 6 : (KERNEL == (SE_STOKESLET | SE_STRESSLET) ? 9
                           : ((KERNEL == SE_HARMONIC_FIELD || KERNEL == SE_HARMONIC) ? 1 : 3));
  static constexpr bool t = KERNEL == SE_STRESSLET || KERNEL == (SE_STOKESLET | SE_STRESSLET);
  static constexpr int cp = (c * RMAX + (t ? RMAX : 0) + 3) & ~3;  // + the staged q . nu per RHS
};

// one listed block of 32 targets, evaluated by one warp (sm: the warp's own staging area)
template <typename T, int KERNEL, int RMAX>
__device__ __forceinline__ void real_blk_one(const RealArgs<T>& a, int blk,
                                             BlkSmem<T, BlkComps<KERNEL, RMAX>::cp>& sm) {
  constexpr int CP = BlkComps<KERNEL, RMAX>::cp;
  constexpr int NO = RsOut<KERNEL>::value;
  typedef typename Vec4<T>::type V4;
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const CellGeom& g = a.cg;
  const int s0 = blk * 32;
  const int nt = min(32, a.ntgt - s0);
  const bool tv = lane < nt;
  const int s = s0 + (tv ? lane : 0);
  const int C = BlkComps<KERNEL, RMAX>::c * a.n_rhs;
  // a group evaluation: every target of a listed block is in one configuration (k_real_classify)
  const int cfgcell = group_of(a.cg.gr, s0) * (a.cg.nc[0] * a.cg.nc[1] * a.cg.nc[2]);
  const V4 th = a.xt[s];
  V4 tl;
  tl.x = tl.y = tl.z = tl.w = T(0);
  if (sizeof(T) == 4) tl = a.xtl[s];
  // the block's box (hi parts)
  T bl[3] = {th.x, th.y, th.z}, bh[3] = {th.x, th.y, th.z};
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      bl[d] = min(bl[d], __shfl_xor_sync(FULL, bl[d], off));
      bh[d] = max(bh[d], __shfl_xor_sync(FULL, bh[d], off));
    }
  }
  const T rc = sqrt(a.rc2);
  const T rcp2 = a.rc2 * T(1.0001) + T(1e-12);  // column trimming, slightly larger than r_c^2
  // unwrapped cells that can hold sources within rc of the box
  int ulo[3], uhi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ulo[d] = (int)floor((bl[d] - rc) / a.cs[d]);
    uhi[d] = (int)floor((bh[d] + rc) / a.cs[d]);
    if (!g.periodic[d]) {
      ulo[d] = max(ulo[d], 0);
      uhi[d] = min(uhi[d], g.nc[d] - 1);
    }
  }
  const int ncx = uhi[0] - ulo[0] + 1, ncy = uhi[1] - ulo[1] + 1;
  const int ncol = max(0, ncx) * max(0, ncy);
  const int maxseg = a.maxseg, cpr = a.cols_per_round;
  T acc[NO * RMAX], cmp[NO * RMAX];
#pragma unroll
  for (int k = 0; k < NO * RMAX; ++k) acc[k] = cmp[k] = T(0);
  const T xi = a.xi, xi2 = xi * xi;
  const T c2pi = T(2.0 / 1.7724538509055160273) * xi;  // 2 xi / sqrt(pi)
  for (int c0 = 0; c0 < ncol; c0 += cpr) {
    // ---- segments of the columns c0 .. c0 + cpr - 1 (column c0 + lane on this lane)
    __syncwarp();
    const int slot0 = lane * maxseg;
    int nseg = 0, tot = 0;
    const int k = c0 + lane;
    if (lane < cpr && k < ncol) {
      const int ux = ulo[0] + k / ncy, uy = ulo[1] + k % ncy;
      // distance between the column (cells ux, uy) and the box, directions 0 and 1
      const T x0 = T(ux) * a.cs[0], x1 = x0 + a.cs[0];
      const T y0 = T(uy) * a.cs[1], y1 = y0 + a.cs[1];
      const T ddx = max(T(0), max(x0 - bh[0], bl[0] - x1));
      const T ddy = max(T(0), max(y0 - bh[1], bl[1] - y1));
      const T rem = rcp2 - ddx * ddx - ddy * ddy;
      if (rem > T(0)) {
        const T zr = sqrt(rem);
        int zlo = max((int)floor((bl[2] - zr) / a.cs[2]), ulo[2]);
        const int zhi = min((int)floor((bh[2] + zr) / a.cs[2]), uhi[2]);
        int imx = 0, imy = 0;
        const int wx = g.periodic[0] ? wrap_cell(ux, g.nc[0], &imx) : ux;
        const int wy = g.periodic[1] ? wrap_cell(uy, g.nc[1], &imy) : uy;
        const int colbase = cfgcell + (wx * g.nc[1] + wy) * g.nc[2];
        while (zlo <= zhi && nseg < maxseg) {
          int imz = 0, w0 = zlo;
          if (g.periodic[2]) w0 = wrap_cell(zlo, g.nc[2], &imz);
          const int w1 = min(g.nc[2] - 1, w0 + (zhi - zlo));
          const int beg = a.cstart[colbase + w0], end = a.cstart[colbase + w1 + 1];
          const int sl = slot0 + nseg;
          sm.beg[sl] = beg;
          sm.len[sl] = end - beg;
          sm.pk[sl] = (imx + 128) | ((imy + 128) << 8) | ((imz + 128) << 16);
          tot += end - beg;
          ++nseg;
          zlo += w1 - w0 + 1;
        }
      }
    }
    if (lane < cpr)
      for (int i = nseg; i < maxseg; ++i) sm.len[slot0 + i] = 0;
    int inc = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(FULL, inc, off);
      if (lane >= off) inc += v;
    }
    const int total = __shfl_sync(FULL, inc, 31);
    __syncwarp();
    if (lane < cpr) {
      int run = inc - tot;
      for (int i = 0; i < maxseg; ++i) {
        sm.start[slot0 + i] = run;
        run += sm.len[slot0 + i];
      }
    }
    if (lane == 0) sm.start[cpr * maxseg] = total;
    __syncwarp();
    // ---- stream the flat list: candidate b0 + lane loaded one chunk ahead
    int sp = 0;
    V4 pv, lv;
    T fv[CP];
    auto fetch = [&](int b0) {
      const int f = b0 + lane;
      pv.x = pv.y = pv.z = pv.w = T(0);
      lv = pv;
      pv.x = T(3e30);  // an unused slot is never within rc
#pragma unroll
      for (int c = 0; c < CP; ++c) fv[c] = T(0);
      if (f < total) {
        while (sm.start[sp + 1] <= f) ++sp;
        const int j = sm.beg[sp] + (f - sm.start[sp]);
        const int pk = sm.pk[sp];
        const T i0 = T((pk & 255) - 128), i1 = T(((pk >> 8) & 255) - 128), i2 = T(((pk >> 16) & 255) - 128);
        const V4 xh = a.xs[j];
        V4 xl;
        xl.x = xl.y = xl.z = xl.w = T(0);
        if (sizeof(T) == 4) xl = a.xsl[j];
        // image position a = x_hi + i L_hi and the rest x_lo + i L_lo + (a's rounding)
        const T shx = i0 * a.Lhi[0], shy = i1 * a.Lhi[1], shz = i2 * a.Lhi[2];
        pv.x = xh.x + shx;
        pv.y = xh.y + shy;
        pv.z = xh.z + shz;
        lv.x = xl.x + (i0 * a.Llo[0] + (xh.x - (pv.x - shx)));
        lv.y = xl.y + (i1 * a.Llo[1] + (xh.y - (pv.y - shy)));
        lv.z = xl.z + (i2 * a.Llo[2] + (xh.z - (pv.z - shz)));
        const T* fj = a.fs + (size_t)j * C;
#pragma unroll
        for (int c = 0; c < CP; ++c)
          if (c < C) fv[c] = fj[c];
        if (BlkComps<KERNEL, RMAX>::t) {  // q . nu of each RHS, after the strengths
          constexpr int ST_ = BlkComps<KERNEL, RMAX>::c, QO = KERNEL == SE_STRESSLET ? 0 : 3;
#pragma unroll
          for (int r = 0; r < RMAX; ++r) {
            const T* qv = fv + ST_ * r + QO;
            fv[ST_ * RMAX + r] = qv[0] * qv[3] + qv[1] * qv[4] + qv[2] * qv[5];
          }
        }
      }
    };
    if (total > 0) fetch(0);
    for (int b0 = 0; b0 < total; b0 += 32) {
      __syncwarp();
      sm.pos[lane] = pv;
      sm.low[lane] = lv;
#pragma unroll
      for (int c = 0; c < CP; ++c) sm.str[lane][c] = fv[c];
      __syncwarp();
      if (b0 + 32 < total) fetch(b0 + 32);  // in flight while this chunk is evaluated
      const int cnt = min(32, total - b0);
      T part[NO * RMAX];
#pragma unroll
      for (int q = 0; q < NO * RMAX; ++q) part[q] = T(0);
      // two staged candidates at a time, their pair terms without branches (real_pair_m)
      // so that the two evaluations interleave; a pair of candidates that no lane needs is
      // skipped (warp-uniform). Unused staging slots hold a far position (never inside).
      for (int jj = 0; jj < cnt; jj += 2) {
        const V4 sa = sm.pos[jj], sb = sm.pos[jj + 1];
        const V4 la = sm.low[jj], lb = sm.low[jj + 1];
        // exact separations (hi parts and remainders) directly: a pre-test on the hi parts alone
        // cost more than it saved, since in a dense block almost every candidate is needed
        const T a0 = (th.x - sa.x) + (tl.x - la.x), a1 = (th.y - sa.y) + (tl.y - la.y),
                a2 = (th.z - sa.z) + (tl.z - la.z);
        const T b0 = (th.x - sb.x) + (tl.x - lb.x), b1 = (th.y - sb.y) + (tl.y - lb.y),
                b2 = (th.z - sb.z) + (tl.z - lb.z);
        const T ra = a0 * a0 + a1 * a1 + a2 * a2, rb = b0 * b0 + b1 * b1 + b2 * b2;
        const bool ina = tv && ra < a.rc2;
        const bool inb = tv && jj + 1 < cnt && rb < a.rc2;
        if (!__any_sync(FULL, ina || inb)) continue;
        real_pair_m<T, KERNEL, RMAX, BlkComps<KERNEL, RMAX>::t>(a0, a1, a2, ra, ina, xi, xi2, c2pi, sm.str[jj],
                                                               a.n_rhs, part);
        real_pair_m<T, KERNEL, RMAX, BlkComps<KERNEL, RMAX>::t>(b0, b1, b2, rb, inb, xi, xi2, c2pi,
                                                               sm.str[jj + 1], a.n_rhs, part);
      }
      // fold the chunk into the sums (compensated in FP32)
#pragma unroll
      for (int q = 0; q < NO * RMAX; ++q) {
        if (sizeof(T) == 4) {
          const T y = part[q] - cmp[q];
          const T t = acc[q] + y;
          cmp[q] = (t - acc[q]) - y;
          acc[q] = t;
        } else {
          acc[q] += part[q];
        }
      }
    }
  }
  if (tv) {
    const int i = a.tperm[s];
    for (int r = 0; r < a.n_rhs && r < RMAX; ++r)
      for (int q = 0; q < NO; ++q) {
        T* o = a.u + out_index(a.cg.gr, a.n_rhs, NO, a.ntgt, i, r, q);
        *o = a.overwrite ? acc[NO * r + q] : *o + acc[NO * r + q];
      }
  }
}

// The listed blocks, a warp each: with next == nullptr one warp per listed block (grid over
// all of them); otherwise a grid of a few CTAs per SM whose warps take the next block from the
// counter *next until the list is done, leaving the rest of each SM to the kernels of the
// Fourier part running concurrently on the other stream.
template <typename T, int KERNEL, int RMAX>
__global__ void __launch_bounds__(32 * RB_WARPS) k_real_blk(RealArgs<T> a, const int* __restrict__ blist,
                                                            const int* __restrict__ bcount, int* next) {
  __shared__ __align__(16) BlkSmem<T, BlkComps<KERNEL, RMAX>::cp> sm_all[RB_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = *bcount;
  if (next == nullptr) {
    const int bi = blockIdx.x * RB_WARPS + warp;
    if (bi < nb) real_blk_one<T, KERNEL, RMAX>(a, blist[bi], sm_all[warp]);  // warp-uniform
    return;
  }
  for (;;) {
    int bi = 0;
    if (lane == 0) bi = atomicAdd(next, 1);
    bi = __shfl_sync(0xffffffffu, bi, 0);
    if (bi >= nb) break;
    real_blk_one<T, KERNEL, RMAX>(a, blist[bi], sm_all[warp]);
    __syncwarp();
  }
}

// Blocks of 32 consecutive sorted targets: a block whose targets lie in a box of side <= thr
// (block-relative coordinates) is listed for k_real_blk, the targets of any other block for
// k_real. One warp per block; the list order depends on the atomics, the results do not
// (every target is summed by exactly one warp).
template <typename T>
__global__ void k_real_classify(RealArgs<T> a, T thr, int nblk, int* __restrict__ blist, int* __restrict__ tlist,
                                int* __restrict__ counts) {
  typedef typename Vec4<T>::type V4;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nblk) return;
  const unsigned FULL = 0xffffffffu;
  const int s0 = warp * 32;
  const int nt = min(32, a.ntgt - s0);
  const bool tv = lane < nt;
  const int s = s0 + (tv ? lane : 0);
  const V4 th = a.xt[s];
  const T p[3] = {th.x, th.y, th.z};
  bool dense = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T lo = p[d], hi = p[d];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo = min(lo, __shfl_xor_sync(FULL, lo, off));
      hi = max(hi, __shfl_xor_sync(FULL, hi, off));
    }
    dense = dense && (hi - lo <= thr);
  }
  // a block across two configurations of a group goes to k_real
  if (a.cg.gr.ncfg > 1 && group_of(a.cg.gr, s0) != group_of(a.cg.gr, s0 + nt - 1)) dense = false;
  if (dense) {
    if (lane == 0) blist[atomicAdd(&counts[0], 1)] = warp;
  } else {
    int base = 0;
    if (lane == 0) base = atomicAdd(&counts[1], nt);
    base = __shfl_sync(FULL, base, 0);
    if (tv) tlist[base + lane] = s;
  }
}

template <typename T, int K, int R>
static void launch_sparse_k(cudaStream_t st, const RealArgs<T>& a) {
  k_real<T, K, R><<<grid1d(a.ntgt, RS_WARPS), 32 * RS_WARPS, 0, st>>>(a);
}
template <typename T, int R>
static void launch_sparse(cudaStream_t st, const RealArgs<T>& a) {
  if (a.kernel == SE_STOKESLET) launch_sparse_k<T, SE_STOKESLET, R>(st, a);
  else if (a.kernel == SE_ROTLET) launch_sparse_k<T, SE_ROTLET, R>(st, a);
  else if (a.kernel == SE_STRESSLET) launch_sparse_k<T, SE_STRESSLET, R>(st, a);
  else if (a.kernel == SE_HARMONIC_FIELD) launch_sparse_k<T, SE_HARMONIC_FIELD, R>(st, a);
  else if (a.kernel == SE_HARMONIC) launch_sparse_k<T, SE_HARMONIC, R>(st, a);
  else launch_sparse_k<T, SE_STOKESLET | SE_STRESSLET, R>(st, a);
}

template <typename T>
int real_launch(cudaStream_t st, const RealArgs<T>& a) {
  if (a.n_rhs <= 1) launch_sparse<T, 1>(st, a);
  else if (a.n_rhs <= 4) launch_sparse<T, 4>(st, a);
  else if (a.n_rhs <= 8) launch_sparse<T, 8>(st, a);
  else launch_sparse<T, 16>(st, a);
  return 1;
}

template <typename T, int K, int R>
static void launch_blk_k(cudaStream_t st, const RealArgs<T>& a, const int* blist, const int* bcount, int nblk,
                         int* next, int leave) {
  // persistent: as many CTAs per SM as fit, less `leave`, on every SM
  static int per_sm = -1, sms = 0;
  if (per_sm < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_real_blk<T, K, R>, 32 * RB_WARPS, 0) != cudaSuccess)
      per_sm = 0;
    cudaGetLastError();
  }
  const int ctas = std::max(1, per_sm - leave) * std::max(sms, 1);
  if (per_sm <= 0) next = nullptr;
  k_real_blk<T, K, R><<<next ? ctas : grid1d(nblk, RB_WARPS), 32 * RB_WARPS, 0, st>>>(a, blist, bcount, next);
}
template <typename T, int R>
static void launch_blk(cudaStream_t st, const RealArgs<T>& a, const int* blist, const int* bcount, int nblk,
                       int* next, int leave) {
  if (a.kernel == SE_STOKESLET) launch_blk_k<T, SE_STOKESLET, R>(st, a, blist, bcount, nblk, next, leave);
  else if (a.kernel == SE_ROTLET) launch_blk_k<T, SE_ROTLET, R>(st, a, blist, bcount, nblk, next, leave);
  else if (a.kernel == SE_STRESSLET) launch_blk_k<T, SE_STRESSLET, R>(st, a, blist, bcount, nblk, next, leave);
  else if (a.kernel == SE_HARMONIC_FIELD) launch_blk_k<T, SE_HARMONIC_FIELD, R>(st, a, blist, bcount, nblk, next, leave);
  else if (a.kernel == SE_HARMONIC) launch_blk_k<T, SE_HARMONIC, R>(st, a, blist, bcount, nblk, next, leave);
  else launch_blk_k<T, SE_STOKESLET | SE_STRESSLET, R>(st, a, blist, bcount, nblk, next, leave);
}

template <typename T>
se_status real_launch_blocks(cudaStream_t st, RealArgs<T> a, const RealArgs<T>& sparse, int* work, double thr,
                             int leave, int* launches) {
  if (a.ntgt <= 0) return SE_OK;
  if (a.n_rhs > 4) {  // the block kernel keeps 3 x 3 n_rhs sums per lane: many RHS use k_real
    *launches += real_launch(st, sparse);
    return SE_OK;
  }
  const int nblk = (a.ntgt + 31) / 32;
  // segment table of the block kernel: a column spans the box (<= thr) plus r_c on either side
  // along direction 2, i.e. up to 2 range + ceil(thr / cs) + 2 cells; periodic wrapping splits
  // it once per image boundary
  RealArgs<T> ab = a;
  {
    const CellGeom& g = a.cg;
    const int span = 2 * g.range[2] + (int)std::ceil(thr * g.inv_cs[2]) + 2;
    int maxseg = 1;
    if (g.periodic[2]) maxseg = (span + g.nc[2] - 1) / g.nc[2] + 1;
    if (maxseg > RB_SEGCAP) return SE_ERR_UNSUPPORTED;
    ab.maxseg = maxseg;
    ab.cols_per_round = std::min(32, RB_SEGCAP / maxseg);
  }
  int* counts = work;  // listed blocks, sparse targets, the persistent grid's next block
  int* blist = work + 3;
  int* tlist = blist + nblk;
  SE_CUDA(cudaMemsetAsync(counts, 0, 3 * sizeof(int), st));
  k_real_classify<T><<<grid1d(nblk, 4), 128, 0, st>>>(a, (T)thr, nblk, blist, tlist, counts);
  if (a.n_rhs <= 1) launch_blk<T, 1>(st, ab, blist, counts, nblk, counts + 2, leave);
  else launch_blk<T, 4>(st, ab, blist, counts, nblk, counts + 2, leave);
  RealArgs<T> b = sparse;  // the targets of the other blocks, on the sparse path's own cell list
  b.tlist = tlist;
  b.tcount = counts + 1;
  real_launch(st, b);
  *launches += 3;
  SE_CUDA(cudaGetLastError());
  return SE_OK;
}

template se_status real_seg_setup<float>(RealArgs<float>&);
template se_status real_seg_setup<double>(RealArgs<double>&);
template int real_launch<float>(cudaStream_t, const RealArgs<float>&);
template int real_launch<double>(cudaStream_t, const RealArgs<double>&);
template se_status real_launch_blocks<float>(cudaStream_t, RealArgs<float>, const RealArgs<float>&, int*, double,
                                             int, int*);
template se_status real_launch_blocks<double>(cudaStream_t, RealArgs<double>, const RealArgs<double>&, int*, double,
                                              int, int*);

}  // namespace se
