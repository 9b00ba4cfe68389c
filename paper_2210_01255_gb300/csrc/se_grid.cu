// libse gridding step, Eq. (SE-gridding-disc): H(x_j) = sum_n f_n w(x_j - x_n) on the uniform
// grid, with the separable window w = w0 w0 w0 (Sec. 3.3) of support P grid points per direction.
//
// Output-driven, one warp per tile of 4 x 4 x TZ grid points (by default TZ = 4 for 9-12
// components, 8 for fewer; se_opts.tile forces either where the register block fits), no
// atomics for all but the densest tiles:
//   candidates  points are sorted by bins of 4^3 cells (z fastest), so the bins of one (x, y)
//               bin column that can reach the tile are one contiguous run of points; the runs are
//               set up one per lane and laid out as a flat list by a warp scan; each lane tests
//               one candidate (its taps against the tile) and the reaching points are compacted
//               into a pending list (ballot);
//   chunks      32 pending points at a time: lane p forms A[p][xy] = w0x w0y (16 values) and
//               B[p][z][c] = w0z f_c (TZ x C values) of its point in shared memory, then every lane
//               accumulates a 2 (xy) x RZ (z) x C register block of the tile as a sum of outer
//               products over the 32 points (one FMA per accumulator per point, operands read
//               from shared memory as broadcasts);
//   accuracy    each chunk's partial is folded into the accumulators with Kahan compensation
//               (FP32), so that grid values that sum 1e4 points keep FP32 accuracy;
//   balance     a tile with more than GK_ITEM candidates does the first GK_ITEM itself, stores
//               its partial and queues the rest as further items; a second launch works the queue
//               and adds its partials atomically.
// All products of the tile's 4 x 4 x TZ block are formed for every point that reaches it (the
// ones outside the point's support multiply zeros): with P = 8 about 40 % of the FMAs are inside
// the support, in exchange for a loop of plain FMAs on shared-memory broadcasts.
#include <cuda_runtime.h>

#include <algorithm>

#include "se_device.cuh"

namespace se {

namespace {

constexpr int GK_ITEM = 8192;  // candidates per work item
constexpr int GSEGCAP = 96;    // segments per round (32 columns x up to 3 z-runs)
constexpr int GZR = 4;         // z-runs per tile (periodic images)

template <int CG>
struct GPad {  // staging row width per z: a multiple of 4, chosen against bank conflicts
  static constexpr int v = CG <= 3 ? 4 : 12;
};

// warps per CTA (static shared memory <= 48 KB)
template <typename T, int TZ>
struct GWarps {
  static constexpr int v = sizeof(T) == 8 ? 1 : (TZ == 4 ? 4 : 2);
};

template <typename T, int TZ, int CG>
struct GSmem {
  T A[32][16];
  T B[32][TZ][GPad<CG>::v];
  int4 pend[64];
  int sbeg[GSEGCAP], sstart[GSEGCAP + 1], slen[GSEGCAP];
  int srel[GSEGCAP][3];
  int xb[SP_MAXB], xsh[SP_MAXB], yb[SP_MAXB], ysh[SP_MAXB];
  int zlo[GZR], zhi[GZR], zsh[GZR];
  int nx, ny, nz;
};

struct GridArgs {
  GridGeom g;
  int nb[3];                // bins per direction (4^3 cells each)
  int nt[3];                // tiles per direction
  const int* bin_start;     // [nbins + 1]
  const int* base;          // [N][3] first tap (cell - P/2 + 1), wrapped cell
  int Ctot, c0, C;          // components c0 .. c0 + C - 1 of Ctot
  long long cst, xst;       // grid: component c at c cst, point (x, y, z) at x xst + y n2 + z
  int2* queue;              // overflow items: (tile, slab)
  int* qcount;
  int qcap;
  int ncfg;                 // configurations of a group evaluation (1 otherwise): tile t of
                            // configuration c is item c ntiles + t, its bins are offset by
                            // c nbins and its components by c Ctot
};

// (bin, grid shift) pairs along direction d that can hold points reaching [o, o + E) (x, y), or
// z-runs of bins (lo, hi, shift) (z); a point in cell c reaches the tile iff
// c in [o - P/2, o + E - 2 + P/2]; periodic directions split that range per image.
__device__ inline void bin_lists(const GridGeom& g, const int* nb, int d, int o, int E, int* b, int* sh, int* n,
                                 int* zlo, int* zhi, bool runs) {
  const int P = g.P, m = g.m[d];
  int clo = o - P / 2, chi = o + E - 2 + P / 2;
  int k = 0;
  auto add = [&](int a, int e, int shift) {
    if (runs) {
      if (k < GZR) {
        zlo[k] = a / 4;
        zhi[k] = e / 4;
        sh[k] = shift;
        ++k;
      }
    } else {
      for (int q = a / 4; q <= e / 4 && k < SP_MAXB; ++q) {
        b[k] = q;
        sh[k] = shift;
        ++k;
      }
    }
  };
  if (!g.periodic[d]) {
    clo = max(clo, 0);
    chi = min(chi, m - 1);
    if (clo <= chi) add(clo, chi, 0);
  } else {
    int c = clo;
    while (c <= chi) {
      const int im = fdiv(c, m);
      const int hi = min(chi, (im + 1) * m - 1);
      add(c - im * m, hi - im * m, im * m);
      c = hi + 1;
    }
  }
  *n = k;
  (void)nb;
}

template <typename T, int TZ, int RZ, int CG, bool QUEUE>
__global__ void __launch_bounds__(32 * GWarps<T, TZ>::v) k_grid(GridArgs a, const T* __restrict__ wts,
                                                           const T* __restrict__ sf, T* __restrict__ grid) {
  constexpr int NW = GWarps<T, TZ>::v;
  __shared__ __align__(16) GSmem<T, TZ, CG> sm_all[NW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  GSmem<T, TZ, CG>& sm = sm_all[warp];
  const unsigned FULL = 0xffffffffu;
  const GridGeom& g = a.g;
  const int P = g.P;
  const int ntiles = a.nt[0] * a.nt[1] * a.nt[2];
  const int nbins = a.nb[0] * a.nb[1] * a.nb[2];
  // thread block of the tile: xy entries 2 ga, 2 ga + 1 (x = ga / 2, y = 2 (ga % 2) + {0, 1}),
  // z = gz RZ .. gz RZ + RZ - 1
  const int ga = lane & 7, gz = lane >> 3;
  const int tx = ga >> 1, ty0 = 2 * (ga & 1);
  int item = QUEUE ? blockIdx.x * NW + warp : 0;
  const int nq = QUEUE ? min(*a.qcount, a.qcap) : 0;
  for (;;) {
    int tile, slab;
    if (QUEUE) {
      if (item >= nq) return;
      const int2 e = a.queue[item];
      tile = e.x;
      slab = e.y;
      item += gridDim.x * NW;
    } else {
      tile = blockIdx.x * NW + warp;
      slab = 0;
      if (tile >= ntiles * a.ncfg) return;
    }
    const int cfg = tile / ntiles, lt = tile - cfg * ntiles;
    const int* bin_start = a.bin_start + (size_t)cfg * nbins;
    const int t2 = lt % a.nt[2], t1 = (lt / a.nt[2]) % a.nt[1], t0 = lt / (a.nt[2] * a.nt[1]);
    const int o0 = 4 * t0, o1 = 4 * t1, o2 = TZ * t2;
    __syncwarp();
    if (lane == 0) bin_lists(g, a.nb, 0, o0, 4, sm.xb, sm.xsh, &sm.nx, nullptr, nullptr, false);
    if (lane == 1) bin_lists(g, a.nb, 1, o1, 4, sm.yb, sm.ysh, &sm.ny, nullptr, nullptr, false);
    if (lane == 2) bin_lists(g, a.nb, 2, o2, TZ, nullptr, sm.zsh, &sm.nz, sm.zlo, sm.zhi, true);
    __syncwarp();
    const int nx = sm.nx, ny = sm.ny, nz = sm.nz;
    const int ncol = nx * ny;
    const int cpr = min(32, GSEGCAP / max(nz, 1));
    // ---- pass 1: the tile's number of candidates (and the work items it splits into)
    int total_all = 0;
    for (int r0 = 0; r0 < ncol; r0 += cpr) {
      int cnt = 0;
      const int k = r0 + lane;
      if (lane < cpr && k < ncol) {
        const int ix = k / ny, iy = k - (k / ny) * ny;
        const int colb = (sm.xb[ix] * a.nb[1] + sm.yb[iy]) * a.nb[2];
        for (int z = 0; z < nz; ++z) cnt += bin_start[colb + sm.zhi[z] + 1] - bin_start[colb + sm.zlo[z]];
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(FULL, cnt, off);
      total_all += cnt;
    }
    int nitems = (total_all + GK_ITEM - 1) / GK_ITEM;
    bool split = false;
    if (!QUEUE && nitems > 1) {
      // queue slabs 1 .. nitems - 1 (if the queue is full, the warp does the whole tile)
      int q0 = 0;
      if (lane == 0) {
        q0 = atomicAdd(a.qcount, nitems - 1);
        if (q0 + nitems - 1 > a.qcap) q0 = -1;
      }
      q0 = __shfl_sync(FULL, q0, 0);
      if (q0 >= 0) {
        for (int s = 1 + lane; s < nitems; s += 32) a.queue[q0 + s - 1] = make_int2(tile, s);
        split = true;
      }
    }
    const int lo = slab * GK_ITEM;
    const int hi = (QUEUE || split) ? min(total_all, lo + GK_ITEM) : total_all;
    // ---- pass 2: candidates lo .. hi of the flat list, chunks of 32 reaching points
    T acc[2][RZ][CG], cmp[2][RZ][CG];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int z = 0; z < RZ; ++z)
#pragma unroll
        for (int c = 0; c < CG; ++c) acc[i][z][c] = cmp[i][z][c] = T(0);
    int npend = 0;
    auto chunk = [&](int n) {  // uniform
      if (lane < n) {
        const int4 pe = sm.pend[lane];
        const int j = pe.x;
        const T* wj = wts + (size_t)j * 3 * P;
        T wx[4], wy[4], wz[TZ];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int qx = t - pe.y, qy = t - pe.z;
          wx[t] = (qx >= 0 && qx < P) ? wj[qx] : T(0);
          wy[t] = (qy >= 0 && qy < P) ? wj[P + qy] : T(0);
        }
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
          const int qz = t - pe.w;
          wz[t] = (qz >= 0 && qz < P) ? wj[2 * P + qz] : T(0);
        }
        T fv[CG];
        const T* fj = sf + (size_t)j * a.Ctot + a.c0;
#pragma unroll
        for (int c = 0; c < CG; ++c) fv[c] = c < a.C ? fj[c] : T(0);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) sm.A[lane][4 * x + y] = wx[x] * wy[y];
#pragma unroll
        for (int z = 0; z < TZ; ++z)
#pragma unroll
          for (int c = 0; c < CG; ++c) sm.B[lane][z][c] = wz[z] * fv[c];
      }
      __syncwarp();
      T part[2][RZ][CG];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int z = 0; z < RZ; ++z)
#pragma unroll
          for (int c = 0; c < CG; ++c) part[i][z][c] = T(0);
      for (int p = 0; p < n; ++p) {
        const T a0 = sm.A[p][4 * tx + ty0], a1 = sm.A[p][4 * tx + ty0 + 1];
#pragma unroll
        for (int z = 0; z < RZ; ++z) {
          T bv[CG];
#pragma unroll
          for (int c = 0; c < CG; ++c) bv[c] = sm.B[p][gz * RZ + z][c];
#pragma unroll
          for (int c = 0; c < CG; ++c) {
            part[0][z][c] = fma(a0, bv[c], part[0][z][c]);
            part[1][z][c] = fma(a1, bv[c], part[1][z][c]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int z = 0; z < RZ; ++z)
#pragma unroll
          for (int c = 0; c < CG; ++c) {
            if (sizeof(T) == 4) {
              const T y = part[i][z][c] - cmp[i][z][c];
              const T t = acc[i][z][c] + y;
              cmp[i][z][c] = (t - acc[i][z][c]) - y;
              acc[i][z][c] = t;
            } else {
              acc[i][z][c] += part[i][z][c];
            }
          }
      __syncwarp();
    };
    int fbase = 0;  // flat index of the first candidate of this round
    for (int r0 = 0; r0 < ncol && fbase < hi; r0 += cpr) {
      // segments of the columns r0 .. r0 + cpr - 1
      int nseg = 0, tot = 0;
      const int k = r0 + lane;
      const int slot0 = lane * nz;
      if (lane < cpr && k < ncol) {
        const int ix = k / ny, iy = k - (k / ny) * ny;
        const int colb = (sm.xb[ix] * a.nb[1] + sm.yb[iy]) * a.nb[2];
        for (int z = 0; z < nz; ++z) {
          const int b = bin_start[colb + sm.zlo[z]], e = bin_start[colb + sm.zhi[z] + 1];
          const int sl = slot0 + z;
          sm.sbeg[sl] = b;
          sm.slen[sl] = e - b;
          sm.srel[sl][0] = sm.xsh[ix] - o0;
          sm.srel[sl][1] = sm.ysh[iy] - o1;
          sm.srel[sl][2] = sm.zsh[z] - o2;
          tot += e - b;
          ++nseg;
        }
      } else if (lane < cpr) {
        for (int z = 0; z < nz; ++z) sm.slen[slot0 + z] = 0;
      }
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
        for (int z = 0; z < nz; ++z) {
          sm.sstart[slot0 + z] = run;
          run += sm.slen[slot0 + z];
        }
      }
      if (lane == 0) sm.sstart[cpr * nz] = total;
      __syncwarp();
      // this round's share of the item's range [lo, hi)
      const int f0 = max(lo - fbase, 0), f1 = min(hi - fbase, total);
      int sp = 0;
      for (int fb = f0; fb < f1; fb += 32) {
        const int f = fb + lane;
        bool reach = false;
        int j = 0, s0 = 0, s1 = 0, s2 = 0;
        if (f < f1) {
          while (sm.sstart[sp + 1] <= f) ++sp;
          j = sm.sbeg[sp] + (f - sm.sstart[sp]);
          s0 = a.base[3 * (size_t)j] + sm.srel[sp][0];
          s1 = a.base[3 * (size_t)j + 1] + sm.srel[sp][1];
          s2 = a.base[3 * (size_t)j + 2] + sm.srel[sp][2];
          reach = s0 < 4 && s0 + P > 0 && s1 < 4 && s1 + P > 0 && s2 < TZ && s2 + P > 0;
        }
        const unsigned bal = __ballot_sync(FULL, reach);
        if (reach) sm.pend[npend + __popc(bal & ((1u << lane) - 1u))] = make_int4(j, s0, s1, s2);
        npend += __popc(bal);
        __syncwarp();
        if (npend >= 32) {
          chunk(32);
          npend -= 32;
          int4 v = make_int4(0, 0, 0, 0);
          if (lane < npend) v = sm.pend[32 + lane];
          __syncwarp();
          if (lane < npend) sm.pend[lane] = v;
          __syncwarp();
        }
      }
      fbase += total;
    }
    if (npend > 0) chunk(npend);
    // ---- epilogue: store (the tile's only or first item) or add (queued items)
    const int x = o0 + tx;
    const bool atomic = QUEUE;
    if (x < g.m[0]) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int y = o1 + ty0 + i;
        if (y >= g.m[1]) continue;
#pragma unroll
        for (int z = 0; z < RZ; ++z) {
          const int zz = o2 + gz * RZ + z;
          if (zz >= g.m[2]) continue;
          const size_t off = (size_t)x * a.xst + (size_t)y * g.n[2] + zz;
#pragma unroll
          for (int c = 0; c < CG; ++c) {
            if (c < a.C) {
              T* dst = grid + (size_t)((size_t)cfg * a.Ctot + a.c0 + c) * a.cst + off;
              if (atomic) atomicAdd(dst, acc[i][z][c]);
              else *dst = acc[i][z][c];
            }
          }
        }
      }
    }
    if (!QUEUE) return;
  }
}

template <typename T, int TZ, int RZ, int CG>
void launch_grid(cudaStream_t st, GridArgs a, const T* w, const T* sf, T* grid, int* launches) {
  constexpr int NW = GWarps<T, TZ>::v;
  a.nt[0] = cdiv(a.g.m[0], 4);
  a.nt[1] = cdiv(a.g.m[1], 4);
  a.nt[2] = cdiv(a.g.m[2], TZ);
  const long long ntiles = (long long)a.nt[0] * a.nt[1] * a.nt[2] * a.ncfg;
  k_grid<T, TZ, RZ, CG, false><<<(unsigned)((ntiles + NW - 1) / NW), 32 * NW, 0, st>>>(a, w, sf, grid);
  k_grid<T, TZ, RZ, CG, true><<<152 * 4, 32 * NW, 0, st>>>(a, w, sf, grid);
  *launches += 2;
}

}  // namespace

// Gridding of the C spread components of the points sorted by 4^3 bins (bin_start), in groups
// of up to 12 (FP32) components per launch pair.
template <typename T>
se_status grid_launch(se_plan_t* p, const int* bin_start, const int* base, const T* w, const T* sf, int C, T* grid,
                      long long cst, long long xst, int ncfg) {
  const GridGeom& g = p->geom;
  GridArgs a;
  a.g = g;
  a.ncfg = ncfg;
  for (int d = 0; d < 3; ++d) a.nb[d] = cdiv(g.m[d], 4);
  a.bin_start = bin_start;
  a.base = base;
  a.Ctot = C;
  a.cst = cst;
  a.xst = xst;
  // overflow queue: at most one item per GK_ITEM candidates beyond each tile's first
  void* q;
  const size_t qcap = 1 << 20;
  SE_TRY(buf(p, "grid.queue", sizeof(int2) * (qcap + 1), &q));
  a.queue = (int2*)q + 1;
  a.qcount = (int*)q;
  a.qcap = (int)qcap;
  cudaStream_t st = p->stream;
  for (int c0 = 0; c0 < C; c0 += 12) {
    const int Cg = std::min(12, C - c0);
    a.c0 = c0;
    a.C = Cg;
    SE_CUDA(cudaMemsetAsync(a.qcount, 0, sizeof(int), st));
    // tile depth: the plan's choice, else 4 for 7-12 components and 8 for fewer; 10-12
    // components always take 4 (a 2 x 2 x 12 register block with its compensation and chunk
    // partials would not fit the register file)
    const int tz = Cg > 9 ? 4 : (p->opts.tile ? p->opts.tile : (Cg > 6 ? 4 : 8));
    if (Cg > 9) launch_grid<T, 4, 1, 12>(st, a, w, sf, grid, &p->launches);
    else if (Cg > 6) {
      if (tz == 4) launch_grid<T, 4, 1, 9>(st, a, w, sf, grid, &p->launches);
      else launch_grid<T, 8, 2, 9>(st, a, w, sf, grid, &p->launches);
    } else if (Cg > 3) {
      if (tz == 4) launch_grid<T, 4, 1, 6>(st, a, w, sf, grid, &p->launches);
      else launch_grid<T, 8, 2, 6>(st, a, w, sf, grid, &p->launches);
    } else if (Cg > 1) {
      if (tz == 4) launch_grid<T, 4, 1, 3>(st, a, w, sf, grid, &p->launches);
      else launch_grid<T, 8, 2, 3>(st, a, w, sf, grid, &p->launches);
    } else {
      if (tz == 4) launch_grid<T, 4, 1, 1>(st, a, w, sf, grid, &p->launches);
      else launch_grid<T, 8, 2, 1>(st, a, w, sf, grid, &p->launches);
    }
    SE_CUDA(cudaGetLastError());
  }
  return SE_OK;
}

template se_status grid_launch<float>(se_plan_t*, const int*, const int*, const float*, const float*, int, float*,
                                      long long, long long, int);
template se_status grid_launch<double>(se_plan_t*, const int*, const int*, const double*, const double*, int,
                                       double*, long long, long long, int);

}  // namespace se
