// Device helpers shared by the CUDA translation units of libse (private).
#pragma once

#include <cuda_runtime.h>

#include "se_internal.h"

namespace se {

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4 type; };

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// floor division for possibly negative a, b > 0
__host__ __device__ inline int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

inline int grid1d(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : g);
}

// Apply the operator symbol K^(k) of Eqs. (diffop-rel-fourier-1..3) times the real scalar s
// to the transformed components F (re, im), writing the 3 output components (ore, oim).
// Stresslet components are the symmetric ones in the order 11,22,33,12,13,23.
template <typename T>
__device__ __forceinline__ void apply_regular(int kernel, T s, T k0, T k1, T k2, const T* re, const T* im,
                                              T* ore, T* oim) {
  const T kk = k0 * k0 + k1 * k1 + k2 * k2;
  const T kv[3] = {k0, k1, k2};
  if (kernel == SE_STOKESLET) {
    // (-delta k^2 + k k) F
    const T kfr = k0 * re[0] + k1 * re[1] + k2 * re[2];
    const T kfi = k0 * im[0] + k1 * im[1] + k2 * im[2];
    for (int j = 0; j < 3; ++j) {
      ore[j] = s * (-kk * re[j] + kv[j] * kfr);
      oim[j] = s * (-kk * im[j] + kv[j] * kfi);
    }
  } else if (kernel == SE_HARMONIC_FIELD) {
    // gradient of the harmonic kernel: -i k_j q (one input component)
    for (int j = 0; j < 3; ++j) {
      ore[j] = s * kv[j] * im[0];
      oim[j] = -s * kv[j] * re[0];
    }
  } else if (kernel == SE_ROTLET) {
    // -i eps_jlm k_m F_l = -i (F x k)_j
    const T cr[3] = {re[1] * k2 - re[2] * k1, re[2] * k0 - re[0] * k2, re[0] * k1 - re[1] * k0};
    const T ci[3] = {im[1] * k2 - im[2] * k1, im[2] * k0 - im[0] * k2, im[0] * k1 - im[1] * k0};
    for (int j = 0; j < 3; ++j) {
      ore[j] = s * ci[j];
      oim[j] = -s * cr[j];
    }
  } else {
    // K^T_jlm F_lm = i [ -k^2 (2 (F k)_j + k_j tr F) + 2 k_j (k F k) ], F symmetric
    T Fkr[3], Fki[3];
    Fkr[0] = re[0] * k0 + re[3] * k1 + re[4] * k2;
    Fkr[1] = re[3] * k0 + re[1] * k1 + re[5] * k2;
    Fkr[2] = re[4] * k0 + re[5] * k1 + re[2] * k2;
    Fki[0] = im[0] * k0 + im[3] * k1 + im[4] * k2;
    Fki[1] = im[3] * k0 + im[1] * k1 + im[5] * k2;
    Fki[2] = im[4] * k0 + im[5] * k1 + im[2] * k2;
    const T trr = re[0] + re[1] + re[2], tri = im[0] + im[1] + im[2];
    const T kFkr = k0 * Fkr[0] + k1 * Fkr[1] + k2 * Fkr[2];
    const T kFki = k0 * Fki[0] + k1 * Fki[1] + k2 * Fki[2];
    for (int j = 0; j < 3; ++j) {
      const T vr = -kk * (T(2) * Fkr[j] + kv[j] * trr) + T(2) * kv[j] * kFkr;
      const T vi = -kk * (T(2) * Fki[j] + kv[j] * tri) + T(2) * kv[j] * kFki;
      ore[j] = -s * vi;
      oim[j] = s * vr;
    }
  }
}

// Scalar of the regular (unmodified) kernel without the separable factors:
// H^ = 4 pi / k^2 (rotlet and harmonic field, Ewald screening) or
// B^ (1 + k^2/4xi^2) = -8 pi/k^4 (1 + k^2/4xi^2)
// (stokeslet, stresslet, Hasimoto screening); the exp(-k^2/4xi^2) and 1/w^2 factors are
// separable and come from the per-direction tables.
template <typename T>
__device__ __forceinline__ T regular_scalar(int kernel, T kk, T inv4xi2) {
  if (harmonic_family(kernel)) return T(4.0 * 3.14159265358979323846) / kk;
  return T(-8.0 * 3.14159265358979323846) / (kk * kk) * (T(1) + kk * inv4xi2);
}

// ---------------------------------------------------------------- gridding source lists

constexpr int SP_MAXB = 12;  // max (bin, image) pairs per direction (E <= 16, P <= 32: <= 8)

// The source tiles (TS cells per direction, the bins of the point sort) whose points can
// reach the output tile starting at o with extent E along one direction, as (wrapped tile
// index, grid shift) pairs: a point in cell c reaches the tile iff
// c in [o - P/2, o + E - 2 + P/2]. In a periodic direction that cell range is
// split at multiples of m into one segment per image; each segment maps to whole tiles of
// the wrapped grid, so no tile is visited twice for the same image.
__device__ inline int tile_list(const GridGeom& g, int d, int o, int E, int* bins, int* shift) {
  const int P = g.P, m = g.m[d];
  int clo = o - P / 2, chi = o + E - 2 + P / 2;
  int nb = 0;
  if (!g.periodic[d]) {
    clo = max(clo, 0);
    chi = min(chi, m - 1);
    for (int b = clo / TS; b <= chi / TS && nb < SP_MAXB; ++b) {
      bins[nb] = b;
      shift[nb] = 0;
      ++nb;
    }
    return nb;
  }
  int c = clo;
  while (c <= chi && nb < SP_MAXB) {
    const int im = fdiv(c, m);
    const int seg_hi = min(chi, (im + 1) * m - 1);
    const int a = c - im * m, e = seg_hi - im * m;  // wrapped cells a..e
    for (int b = a / TS; b <= e / TS && nb < SP_MAXB; ++b) {
      bins[nb] = b;
      shift[nb] = im * m;
      ++nb;
    }
    c = seg_hi + 1;
  }
  return nb;
}

}  // namespace se
