// Internal declarations of libse: the plan object, launch helpers and kernel entry points.
// Everything here is private to the shared library; the public interface is include/se.h.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/se.h"

namespace se {

constexpr int TS = 8;          // spread/gather tile edge (grid points)
constexpr int MAX_P = 32;      // largest window support
constexpr int MAX_COMP = 48;   // largest number of spread components (16 RHS x 3)

// Stokeslet and stresslet in one evaluation: strengths (f, q, nu) per point, one spread of
// 3 + 6 components, the two k-space operators summed into one velocity.
constexpr int SE_KERNEL_ST = SE_STOKESLET | SE_STRESSLET;

// strength components per point and right-hand side, which is also the number of spread
// components: f (3); (q, nu) (6, spread as the 6 symmetric q nu^T entries); (f, q, nu) (9)
__host__ __device__ inline int kernel_comps(int kernel) {
  return kernel == SE_STRESSLET ? 6
         : (kernel == SE_KERNEL_ST ? 9 : ((kernel == SE_HARMONIC_FIELD || kernel == SE_HARMONIC) ? 1 : 3));
}

// output components per target and right-hand side: the harmonic potential is a scalar
__host__ __device__ inline int out_comps(int kernel) { return kernel == SE_HARMONIC ? 1 : 3; }

// the harmonic field (a first derivative of the harmonic kernel like the rotlet) and the
// harmonic potential take the rotlet's parameter rules (Sec. 4), the Ewald screening and the
// harmonic modified-kernel tables
__host__ __device__ inline bool harmonic_family(int kernel) {
  return kernel == SE_ROTLET || kernel == SE_HARMONIC_FIELD || kernel == SE_HARMONIC;
}

// a kernel mask with the harmonic field's and potential's rules entered as the rotlet's
__host__ __device__ inline int rule_mask(int mask) {
  return (mask & 7) | ((mask & (SE_HARMONIC_FIELD | SE_HARMONIC)) ? SE_ROTLET : 0);
}

// A group of independent configurations evaluated together on one plan (se_eval_group):
// configuration c owns the points off[c] .. off[c+1] - 1 of the concatenated inputs, and the
// same range of every sorted order (the sort keys start with the configuration), its own
// block of grid components and its own block of outputs. ncfg = 1 with off = nullptr is the
// ordinary single evaluation.
struct GroupDev {
  int ncfg = 1;
  const int* off = nullptr;  // device [ncfg + 1]
};
// configuration of point i (original or sorted index): the largest c with off[c] <= i
__host__ __device__ inline int group_of(const GroupDev& gr, int i) {
  if (gr.ncfg <= 1) return 0;
  int lo = 0, hi = gr.ncfg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gr.off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Geometry of the grid that gridding writes and gathering reads (Sec. 3.2).
struct GridGeom {
  int m[3];         // extent of the spread grid per direction (M_i periodic, M'_i free)
  int n[3];         // allocated extent of the (possibly zero-padded) FFT grid
  int periodic[3];  // 1 for the first D directions
  int ntile[3];     // tiles of TS grid points covering [0, m)
  double origin[3]; // grid origin o_i: 0 periodic, -dL_i/2 free (Eq. extended-box)
  double h, inv_h;
  double L[3];
  int P;
  long long cs;     // elements per component of the spread and output grids: n0 n1 n2, or for
                    // D = 0 m0 n1 n2 (only the first M'_0 planes along direction 0 are stored)
};

// Host-side description of the window (Sec. 3.3).
struct WindowDesc {
  int kind;      // SE_WIN_*
  int P;
  double aw;     // a_w = P h / 2
  double alpha;  // Gaussian shape (Eq. TG-window)
  double beta;   // KB shape (Eq. PKB-parameters)
  double i0beta; // I_0(beta)
  int nu;        // PKB degree
  std::vector<double> pkb;  // P x (nu+1) Chebyshev coefficients in the local variable s in [-1,1]
};

// A growable device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Timers {
  cudaEvent_t ev[12] = {};
  bool on = false;
};

}  // namespace se

struct se_plan_t {
  int D = 3;
  double L[3] = {1, 1, 1};
  double xi = 0, rc = 0;
  int P = 0;
  int window = SE_WIN_PKB;
  se_opts opts{};
  int prec = SE_FP64;
  int flags = 0;  // se_opts.flags
  cudaStream_t stream = nullptr;
  int device = 0;

  se::GridGeom geom{};
  se::WindowDesc win{};
  double R = 0, s0 = 0, s_star = 0;
  int kbar_star = 0;
  double dL[3] = {0, 0, 0};

  // device tables
  se::DevBuf pkb_coef;     // P*(nu+1) in the plan precision
  se::DevBuf gtab[3];      // per-direction exp(-k^2/4xi^2) / w^(k)^2, FFT order (plan precision)

  // growable scratch
  std::map<std::string, se::DevBuf>* bufs = nullptr;

  // cuFFT plans keyed by batch count (forward R2C and inverse C2R)
  std::map<int, cufftHandle>* fwd = nullptr;
  std::map<int, cufftHandle>* inv = nullptr;
  // cuFFT plans of the free-direction transforms, keyed by every parameter of the plan
  std::map<std::vector<long long>, cufftHandle>* ffree = nullptr;

  // pinned host staging for se_eval_host
  void* pin = nullptr;
  size_t pin_bytes = 0;

  // device status word (range errors, timeouts)
  int* d_status = nullptr;

  // reduced periodicity (D < 3)
  int ncls[3][3] = {};     // [class][direction] transform lengths in the free directions
  se::DevBuf ptab[3];      // periodic-direction factors exp(-k^2/4xi^2) / w^2 / n
  se::DevBuf ftab[3][3];   // [class][direction] free-direction factors
  se::DevBuf mod0[4];      // k^P = 0 modified-kernel tables
  se::DevBuf atr[2];       // D = 0 precomputed kernels: 0 harmonic, 1 biharmonic
  double poly_c[4] = {0, 0, 0, 0};  // SE_FLAG_SPLIT_POLY: c0 + c1 r^2 + c2 r^4 + c3 r^6 taken out of B_R
  bool poly_on = false;
  std::vector<std::vector<int>> group_off;  // se_eval_group: point offsets last uploaded, per sub-group

  se::Timers timers;
  float times_ms[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  int last_grid_comps = 0;
  bool timed_pending = false;
  bool real_timed = false;
  // side stream for the real-space part (forked from and joined to the plan's stream)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the Fourier chain's stream while the real space runs beside it: the greatest priority
  cudaStream_t hi = nullptr;
  cudaEvent_t ev_hi = nullptr;
  int launches = 0;  // kernels launched by the last evaluation
  long long scale_modes = 0;  // k-space modes per component the last scaling step visited
  // D = 0: buffers whose zero padding is in place (pointer and component count at zeroing)
  void* zeroed_grid = nullptr;
  int zeroed_grid_C = 0;
  void* zeroed_tmp = nullptr;
  int zeroed_tmp_C = 0;
};

namespace se {

// record stage event i (per-stage timing, se_set_timing) on the plan's stream
inline void stage_event(se_plan_t* p, int i) {
  if (p->timers.on) cudaEventRecord(p->timers.ev[i], p->stream);
}

// buffer helper: returns device pointer with at least `bytes` bytes (grows, never shrinks)
se_status buf(se_plan_t* p, const char* name, size_t bytes, void** out);

template <typename T>
struct ScaleTables {
  const T* g0;
  const T* g1;
  const T* g2;
  const T* atab;  // precomputed scalar per half-spectrum mode (D = 0) or nullptr
};
template <typename T>
se_status launch_scale3p(se_plan_t* p, int kernel, int n_rhs, T* spec, const ScaleTables<T>& t);
// gridding on the CUDA cores (se_grid.cu): points sorted by 4^3 bins (bin_start)
template <typename T>
se_status grid_launch(se_plan_t* p, const int* bin_start, const int* base, const T* w, const T* sf, int C, T* grid,
                      long long cst, long long xst, int ncfg = 1);
// FP32 gridding on the tensor cores (se_spread_tc.cu)
se_status spread_tc_launch(se_plan_t* p, const int* tile_start, const int* base, const float* w, const float* sf,
                           int C, float* grid, long long cst, long long xst);
se_status free_plan_setup(se_plan_t* p);
// D = 0, SE_FLAG_FFT_TIMED: extents >= mmin whose transforms take the least time (se_free.cu)
se_status fft0_timed_extents(int prec, cudaStream_t st, const int mmin[3], int cin, int no, int out[3]);
template <typename T>
se_status fourier_free(se_plan_t* p, int kernel, int n_rhs, T* grid, int C, T* ugrid, int NC);
template <typename T>
se_status gauge_correction(se_plan_t* p, const T* f, int stride, int n, int n_rhs, int nt, T* u);
template <typename T>
se_status harmonic_constant(se_plan_t* p, const T* q, int n, int n_rhs, int nt, T* u);
// elements per component of the largest class buffer of the adaptive FFT (D = 2, 1; 0 else)
long long free_class_elems(const se_plan_t* p);
template <typename T>
se_status poly_correction(se_plan_t* p, int kernel, const double* x, const T* f, int n, int n_rhs, const double* t,
                          int nt, T* u);
double pot_mag(int kernel, double L, double Q, double xi);
double lambda_table(int kernel, int D);
void upsampling_rule(int D, const double* box, double h, const int* Mext, double lg, double* s_star,
                     int* kbar_star);

// ---- host-side helpers (se_host.cpp) ----
int round_extent(int x, int fM, bool smooth);
double bessel_i0(double x);
void window_setup(WindowDesc* w, int kind, int P, double h);
double window_hat(const WindowDesc& w, double k);
double window_value(const WindowDesc& w, double r);

}  // namespace se

#define SE_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return SE_ERR_CUDA;          \
  } while (0)
#define SE_CUFFT(call)                                  \
  do {                                                  \
    cufftResult r_ = (call);                            \
    if (r_ != CUFFT_SUCCESS) return SE_ERR_CUFFT;       \
  } while (0)
#define SE_TRY(call)                                    \
  do {                                                  \
    se_status s_ = (call);                              \
    if (s_ != SE_OK) return s_;                         \
  } while (0)
