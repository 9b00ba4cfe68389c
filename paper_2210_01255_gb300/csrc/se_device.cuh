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
// to the transformed components F (re, im), writing the 3 output components (ore, oim); the
// harmonic potential's symbol is 1 (one component in, one out).
// Stresslet components are the symmetric ones in the order 11,22,33,12,13,23.
template <typename T>
__device__ __forceinline__ void apply_regular(int kernel, T s, T k0, T k1, T k2, const T* re, const T* im,
                                              T* ore, T* oim) {
  const T kk = k0 * k0 + k1 * k1 + k2 * k2;
  const T kv[3] = {k0, k1, k2};
  if (kernel == SE_HARMONIC) {
    ore[0] = s * re[0];
    oim[0] = s * im[0];
  } else if (kernel == SE_STOKESLET) {
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
// H^ = 4 pi / k^2 (rotlet, harmonic field and potential, Ewald screening) or
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


// ---------------------------------------------------------------- real-space cell list

// Wrap a coordinate of a periodic direction into [0, L); flag a free coordinate outside
// [0, L) or a non-finite one.
__device__ inline double wrap_coord(double x, double L, int periodic, int* status) {
  if (!isfinite(x)) {
    atomicOr(status, 1);
    return 0.0;
  }
  if (periodic) {
    double w = x - floor(x / L) * L;
    if (w >= L) w -= L;
    if (w < 0) w = 0;
    return w;
  }
  if (x < 0.0 || x >= L) atomicOr(status, 1);
  return fmin(fmax(x, 0.0), nextafter(L, 0.0));
}

// key of the real-space cell of each point (cells of side >= rc / S)
struct CellGeom {
  int nc[3];
  int range[3];
  int periodic[3];
  double L[3];
  double inv_cs[3];
  GroupDev gr;  // configurations of a group evaluation: cell keys and cell starts per configuration
};

// index of output q of RHS r of original target i in u: [n_rhs][nt][no], per configuration of a
// group ([n_rhs][N_c][no] blocks one after the other)
__device__ inline size_t out_index(const GroupDev& gr, int n_rhs, int no, int nt, int i, int r, int q) {
  if (gr.ncfg <= 1) return ((size_t)r * nt + i) * no + q;
  const int c = group_of(gr, i);
  const int b = gr.off[c], nl = gr.off[c + 1] - b;
  return (size_t)b * n_rhs * no + ((size_t)r * nl + (i - b)) * no + q;
}

// Arguments of the real-space kernels (Eq. real-space-potential-Dp), se_real.cu.
template <typename T>
struct RealArgs {
  CellGeom cg;
  T xi, rc2;
  int kernel, n_rhs, nsrc, ntgt;
  T Lhi[3], Llo[3];                  // box lengths as hi + lo parts (image shifts)
  int overwrite;                     // 1: u = sum, 0: u += sum
  int maxseg, cols_per_round;        // segment-table layout (real_seg_setup)
  const typename Vec4<T>::type* xs;  // sorted sources (wrapped), by cell
  const typename Vec4<T>::type* xsl; // low parts x - (T)x of the sorted sources (FP32 only)
  const T* fs;                       // sorted strengths [ns][c * n_rhs]
  const int* cstart;                 // cell starts [ncell+1]
  const typename Vec4<T>::type* xt;  // sorted targets
  const typename Vec4<T>::type* xtl; // low parts of the sorted targets (FP32 only)
  const int* tperm;                  // sorted target -> original index
  const int* tcell;                  // cell of each sorted target ([3] ints)
  T* u;
  // dense-block path (k_real_blk) and target lists
  T cs[3];                           // cell sides L_d / nc_d
  const int* tlist;                  // k_real: sorted targets to evaluate (NULL: all ntgt)
  const int* tcount;                 // k_real: number of entries of tlist (device)
};

// segment-table layout of a sparse real-space launch (se_real.cu)
template <typename T>
se_status real_seg_setup(RealArgs<T>& ra);
// the sparse real-space kernel over a.ntgt targets (or the a.tlist entries, grid for at most
// a.ntgt); returns the kernels launched
template <typename T>
int real_launch(cudaStream_t st, const RealArgs<T>& a);
// the dense-block path: targets grouped in blocks of 32 consecutive (cell-sorted) targets;
// blocks whose targets lie within a box of side <= thr go to the block kernel, the others'
// targets to the sparse kernel, which runs with `sparse` (the same targets, its own cell list
// of coarser cells, or `a` itself). work: int scratch of >= ceil(ntgt / 32) + ntgt + 3 entries.
// leave: CTAs per SM that the persistent block kernel leaves free for kernels running
// concurrently on another stream.
template <typename T>
se_status real_launch_blocks(cudaStream_t st, RealArgs<T> a, const RealArgs<T>& sparse, int* work, double thr,
                             int leave, int* launches);

}  // namespace se
