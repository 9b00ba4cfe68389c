// Gridding, Eq. (SE-gridding-disc), FP32, on the 5th-generation tensor cores (tcgen05);
// selected per plan with SE_FLAG_TC_GRIDDING (window supports P <= 16).
//
// For one output tile of TC_X x TC_Y x Z grid points and the points whose windows reach it,
// the gridding sum is a dense contraction over the points p:
//
//   H[(x, y), (z, c)] = sum_p  A[(x, y), p] * B[(z, c), p],
//   A[(x, y), p] = w0_p(x) w1_p(y),   B[(z, c), p] = w2_p(z) f_p(c),
//
// with the window values w_d aligned to the tile (zero outside the P-point support). That is
// a GEMM with M = TC_X TC_Y = 128 rows, N = Z CG = 48 columns and K = the points. The CTA
// builds A and B for 32 points at a time in shared memory (K-major, no swizzle), one elected
// thread issues tcgen05.mma kind::tf32 into a 128 x 48 FP32 accumulator in tensor memory
// (a fresh one per chunk, two alternating), and the threads read each chunk's sums back with
// tcgen05.ld and add them up in registers. FP32 accuracy comes from the split
// a = a_hi + a_lo into two TF32 numbers: A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (the
// dropped A_lo B_lo and the TF32 truncation of the low parts are below 2^-21 relative).
// Operand stages and accumulators are double-buffered; an mbarrier signalled by
// tcgen05.commit says when the MMAs of a chunk are done. Every wait is bounded: on timeout the CTA sets bit 2 of the
// plan's status word (SE_ERR_TIMEOUT at se_sync), stops issuing work, waits (bounded again) for the MMAs it
// has already committed before it releases its tensor memory, and writes nothing. A timeout therefore leaves the
// whole spread grid of that evaluation invalid (other CTAs' tiles complete, this CTA's tile missing); the caller
// must discard the evaluation's result when se_sync reports SE_ERR_TIMEOUT.

#include <cstdint>

#include "se_device.cuh"

namespace se {

namespace {

constexpr int TC_X = 16, TC_Y = 8;    // output tile extent along directions 0 and 1
constexpr int TC_M = TC_X * TC_Y;     // 128 accumulator rows
constexpr int TC_N = 48;              // accumulator columns: Z * CG
constexpr int TC_K = 32;              // points per operand stage (4 MMAs of K = 8)
constexpr int TC_THREADS = 256;
constexpr int TC_PMAX = 16;           // window supports handled here (larger P: CUDA cores)
constexpr uint32_t TC_TMEM_COLS = 128; // two accumulators of TC_N columns, at 0 and 64
constexpr long long TC_WAIT_LIMIT = 1LL << 22;

// core matrices: 8 rows x 16 bytes (4 TF32 along K); within a stage, core (row group r,
// K group kc) starts at r * SBO + kc * LBO bytes
constexpr uint32_t TC_LBO = 128;                 // next core matrix along K
constexpr uint32_t TC_SBO = 128 * (TC_K / 4);    // next 8-row group

constexpr int TC_WS = TC_K + 4;          // row stride (words) of the transposed window tables
constexpr int TC_RWS = 3 * TC_PMAX + 1;   // per-point stride (words) of the raw window values
constexpr int TC_PEND = 2 * TC_K + TC_THREADS;  // pending reaching points (< 64 + one pass)

template <int Z, int CG>
struct TcSmem {
  uint32_t a_hi[2][TC_M * TC_K];  // operand stages: core matrices (8 rows x 16 B), K-major
  uint32_t a_lo[2][TC_M * TC_K];
  uint32_t b_hi[2][TC_N * TC_K];
  uint32_t b_lo[2][TC_N * TC_K];
  // window values aligned to the tile, transposed: [grid point][point of the chunk]
  // (0 outside the support); rows padded to TC_WS words against bank conflicts
  float w0[TC_X][TC_WS];
  float w1[TC_Y][TC_WS];
  float w2[Z][TC_WS];
  float f[CG][TC_WS];
  float r_w[TC_K * TC_RWS];  // raw window values of the chunk's points (as in wts), odd stride
  int4 pend[TC_PEND];        // reaching points: (index, first tap - tile origin, per direction)
  int wcnt[TC_THREADS / 32];
  uint64_t mbar[2];
  uint32_t tmem_base;
  int bins[3][SP_MAXB], sh[3][SP_MAXB], nb[3];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t f2tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// shared-memory matrix descriptor: start, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N >> 3, M >> 4
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = TC_WAIT_LIMIT) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int Z, int CG>
__global__ void __launch_bounds__(TC_THREADS, 2) k_spread_tc(GridGeom g, const int* __restrict__ tile_start,
                                                             const int* __restrict__ base,
                                                             const float* __restrict__ wts,
                                                             const float* __restrict__ sf, int Ctot, int c0, int C,
                                                             int nslab, float* __restrict__ grid,
                                                             long long cst, long long xst,
                                                             int* __restrict__ status, long long drain_limit) {
  static_assert(Z * CG == TC_N, "accumulator width");
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  TcSmem<Z, CG>& sm = *reinterpret_cast<TcSmem<Z, CG>*>(tc_smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned FULL = 0xffffffffu;
  const int P = g.P;
  const int slab = blockIdx.x % nslab;
  const int o0 = (int)(blockIdx.x / nslab) * TC_X, o1 = (int)blockIdx.y * TC_Y, o2 = (int)blockIdx.z * Z;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 3)
    sm.nb[tid] = tile_list(g, tid, tid == 0 ? o0 : (tid == 1 ? o1 : o2), tid == 0 ? TC_X : (tid == 1 ? TC_Y : Z),
                           sm.bins[tid], sm.sh[tid]);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;
  const int nbx = sm.nb[0], nby = sm.nb[1], nbz = sm.nb[2];
  const int nbins = nbx * nby * nbz;
  constexpr uint32_t IDESC = idesc_tf32(TC_M, TC_N);

  // this thread's share of the accumulator: rows m = 32 (warp % 4) + lane, columns
  // 24 (warp / 4) .. + 23; each 32-point chunk is summed by the tensor cores into a fresh
  // TMEM accumulator (two, alternating) and added here in FP32 with round-to-nearest, so the
  // long sums over the points of a tile carry no accumulator rounding bias
  const int q = warp & 3, half = warp >> 2;
  const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(24 * half);
  float acc[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = 0.f;
  auto drain = [&](int c) {  // wait for chunk c's MMAs and add its accumulator; uniform
    const bool done = mbar_wait(&sm.mbar[c & 1], (uint32_t)((c >> 1) & 1), drain_limit);
    if (!__syncthreads_and(done)) return false;
    tc_fence_after();
    const uint32_t ta = trow + 64u * (uint32_t)(c & 1);
#pragma unroll
    for (int blk = 0; blk < 3; ++blk) {
      uint32_t r[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                     "=r"(r[7])
                   : "r"(ta + 8 * blk));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[8 * blk + i] += __uint_as_float(r[i]);
    }
    tc_fence_before();
    return true;
  };

  int chunk = 0;
  bool ok = true;
  int last = -1;  // last chunk whose MMAs were committed (uniform)
  int npend = 0;
  const unsigned lt_mask = (1u << lane) - 1u;

  // raw data of a chunk (pending points 0 .. cnt - 1), warp w holding points w, w + 8, ...:
  // loaded to registers, stored to shared memory later (all loads of a chunk in flight at once)
  float pw[TC_K / 8][2], pfv[TC_K / 8];
  auto fetch = [&](int first, int cnt) {
#pragma unroll
    for (int j = 0; j < TC_K / 8; ++j) {
      const int k = warp + 8 * j;
      const bool valid = k < cnt;
      const int gp = valid ? sm.pend[first + k].x : 0;
      const float* src = wts + (size_t)gp * 3 * P;
      pw[j][0] = (valid && lane < 3 * P) ? src[lane] : 0.f;
      pw[j][1] = (valid && lane + 32 < 3 * P) ? src[lane + 32] : 0.f;
      pfv[j] = (valid && lane < C) ? sf[(size_t)gp * Ctot + c0 + lane] : 0.f;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int j = 0; j < TC_K / 8; ++j) {
      const int k = warp + 8 * j;
      sm.r_w[k * TC_RWS + lane] = pw[j][0];
      if (lane + 32 < TC_RWS) sm.r_w[k * TC_RWS + lane + 32] = pw[j][1];
      if (lane < CG) sm.f[lane][k] = pfv[j];
    }
  };

  // ---- the source bins streamed through candidate passes: keep the points whose support
  // meets the tile (exact test on the first taps), appended to the pending list
  int it_ib = slab, it_p0 = 0, it_end = 0, it_rel0 = 0, it_rel1 = 0, it_rel2 = 0;
  bool more = it_ib < nbins;
  auto load_bin = [&]() {  // uniform
    while (it_ib < nbins) {
      const int ix = it_ib / (nby * nbz), iy = (it_ib / nbz) % nby, iz = it_ib % nbz;
      const int bin = (sm.bins[0][ix] * g.ntile[1] + sm.bins[1][iy]) * g.ntile[2] + sm.bins[2][iz];
      it_p0 = tile_start[bin];
      it_end = tile_start[bin + 1];
      it_rel0 = sm.sh[0][ix] - o0;
      it_rel1 = sm.sh[1][iy] - o1;
      it_rel2 = sm.sh[2][iz] - o2;
      if (it_p0 < it_end) return true;
      it_ib += nslab;
    }
    return false;
  };
  more = load_bin();
  auto refill = [&]() {  // until two chunks are pending or the bins are exhausted; uniform
    while (more && npend < 2 * TC_K) {
      const int gp = it_p0 + tid;
      bool reach = false;
      int s0 = 0, s1 = 0, s2 = 0;
      if (gp < it_end) {
        s0 = base[3 * (size_t)gp] + it_rel0;
        s1 = base[3 * (size_t)gp + 1] + it_rel1;
        s2 = base[3 * (size_t)gp + 2] + it_rel2;
        reach = s0 < TC_X && s0 + P > 0 && s1 < TC_Y && s1 + P > 0 && s2 < Z && s2 + P > 0;
      }
      const unsigned bal = __ballot_sync(FULL, reach);
      if (lane == 0) sm.wcnt[warp] = __popc(bal);
      __syncthreads();
      int off = npend, tot = 0;
#pragma unroll
      for (int w = 0; w < TC_THREADS / 32; ++w) {
        const int c = sm.wcnt[w];
        off += w < warp ? c : 0;
        tot += c;
      }
      if (reach) sm.pend[off + __popc(bal & lt_mask)] = make_int4(gp, s0, s1, s2);
      npend += tot;
      it_p0 += TC_THREADS;
      if (it_p0 >= it_end) {
        it_ib += nslab;
        more = load_bin();
      }
      __syncthreads();
    }
  };

  refill();
  if (npend > 0) {
    fetch(0, min(TC_K, npend));
    store();
  }
  __syncthreads();
  while (npend > 0 && ok) {
    const int st = chunk & 1;
    const int cnt = min(TC_K, npend), ncnt = min(TC_K, npend - cnt);
    if (ncnt > 0) fetch(cnt, ncnt);  // the next chunk's raw data, in flight during this one
    // ---- window values aligned to the tile, transposed; lane = point of the chunk
    {
      const int k = lane;
      const int4 pe = sm.pend[k];
      const bool valid = k < cnt;
      const float* rw = sm.r_w + k * TC_RWS;
      if (warp == 0 || warp == 4) {
        const int s0 = pe.y;
        for (int l = (warp == 0 ? 0 : TC_X / 2); l < (warp == 0 ? TC_X / 2 : TC_X); ++l) {
          const int qq = l - s0;
          sm.w0[l][k] = (valid && qq >= 0 && qq < P) ? rw[qq] : 0.f;
        }
      } else if (warp == 1) {
        const int s1 = pe.z;
        for (int l = 0; l < TC_Y; ++l) {
          const int qq = l - s1;
          sm.w1[l][k] = (valid && qq >= 0 && qq < P) ? rw[P + qq] : 0.f;
        }
      } else if (warp == 2 || warp == 6) {
        const int s2 = pe.w;
        const int lb = warp == 2 ? 0 : Z / 2, le = warp == 2 ? Z / 2 : Z;
        for (int l = lb; l < le; ++l) {
          const int qq = l - s2;
          sm.w2[l][k] = (valid && qq >= 0 && qq < P) ? rw[2 * P + qq] : 0.f;
        }
      }
    }
    __syncthreads();
    // ---- operands: one task = 4 consecutive K (points) of one row of a core matrix, built
    // from two 128-bit loads and written as two 128-bit stores (hi, lo); 8 lanes of a row
    // group write 128 contiguous bytes
    {
      const int r = tid & 7, kc = (tid >> 3) & 7, rg0 = tid >> 6;  // A: rows m = 8 x + y, x = rg
      const float4 v = *reinterpret_cast<const float4*>(&sm.w1[r][4 * kc]);
#pragma unroll
      for (int j = 0; j < TC_M / 8 / 4; ++j) {
        const int rg = rg0 + 4 * j;
        const float4 u = *reinterpret_cast<const float4*>(&sm.w0[rg][4 * kc]);
        const float a0 = u.x * v.x, a1 = u.y * v.y, a2 = u.z * v.z, a3 = u.w * v.w;
        uint4 hi, lo;
        hi.x = f2tf32(a0);
        hi.y = f2tf32(a1);
        hi.z = f2tf32(a2);
        hi.w = f2tf32(a3);
        // low parts: exact remainders; the tensor core reads their leading TF32 bits
        lo.x = __float_as_uint(a0 - __uint_as_float(hi.x));
        lo.y = __float_as_uint(a1 - __uint_as_float(hi.y));
        lo.z = __float_as_uint(a2 - __uint_as_float(hi.z));
        lo.w = __float_as_uint(a3 - __uint_as_float(hi.w));
        const int widx = (rg * (TC_K / 4) + kc) * 32 + r * 4;  // (rg SBO + kc LBO + r 16 B) / 4
        *reinterpret_cast<uint4*>(&sm.a_hi[st][widx]) = hi;
        *reinterpret_cast<uint4*>(&sm.a_lo[st][widx]) = lo;
      }
      for (int t = tid; t < TC_N * (TC_K / 4); t += TC_THREADS) {  // B: rows n = z CG + c
        const int rb = t & 7, kcb = (t >> 3) & 7, ng = t >> 6;
        const int n = ng * 8 + rb, z = n / CG, c = n - z * CG;
        const float4 u = *reinterpret_cast<const float4*>(&sm.w2[z][4 * kcb]);
        const float4 fv = *reinterpret_cast<const float4*>(&sm.f[c][4 * kcb]);
        const float b0 = u.x * fv.x, b1 = u.y * fv.y, b2 = u.z * fv.z, b3 = u.w * fv.w;
        uint4 hi, lo;
        hi.x = f2tf32(b0);
        hi.y = f2tf32(b1);
        hi.z = f2tf32(b2);
        hi.w = f2tf32(b3);
        lo.x = __float_as_uint(b0 - __uint_as_float(hi.x));
        lo.y = __float_as_uint(b1 - __uint_as_float(hi.y));
        lo.z = __float_as_uint(b2 - __uint_as_float(hi.z));
        lo.w = __float_as_uint(b3 - __uint_as_float(hi.w));
        const int widx = (ng * (TC_K / 4) + kcb) * 32 + rb * 4;
        *reinterpret_cast<uint4*>(&sm.b_hi[st][widx]) = hi;
        *reinterpret_cast<uint4*>(&sm.b_lo[st][widx]) = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t d = tmem + 64u * (uint32_t)st;
      const uint32_t ah = smem_u32(sm.a_hi[st]), al = smem_u32(sm.a_lo[st]);
      const uint32_t bh = smem_u32(sm.b_hi[st]), bl = smem_u32(sm.b_lo[st]);
#pragma unroll
      for (int ks = 0; ks < TC_K / 8; ++ks) {
        const uint32_t off = ks * 2 * TC_LBO;
        const uint64_t dah = smem_desc(ah + off, TC_LBO, TC_SBO), dal = smem_desc(al + off, TC_LBO, TC_SBO);
        const uint64_t dbh = smem_desc(bh + off, TC_LBO, TC_SBO), dbl = smem_desc(bl + off, TC_LBO, TC_SBO);
        mma_tf32(d, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
        mma_tf32(d, dah, dbl, IDESC, 1u);
        mma_tf32(d, dal, dbh, IDESC, 1u);
      }
      mma_commit(&sm.mbar[st]);
    }
    last = chunk;
    if (ncnt > 0) store();  // staging and formation of this chunk are done (barrier above)
    // ---- add the previous chunk (its MMAs ran while this chunk's operands were built); the
    // stage and accumulator of chunk - 1 are then free for chunk + 1
    if (chunk >= 1 && !drain(chunk - 1)) {
      ok = false;
      break;
    }
    ++chunk;
    // ---- drop this chunk from the pending list, then top it up
    {
      const int rest = npend - cnt;
      int4 v0 = make_int4(0, 0, 0, 0), v1 = v0;
      if (tid < rest) v0 = sm.pend[cnt + tid];
      if (tid + TC_THREADS < rest) v1 = sm.pend[cnt + tid + TC_THREADS];
      __syncthreads();
      if (tid < rest) sm.pend[tid] = v0;
      if (tid + TC_THREADS < rest) sm.pend[tid + TC_THREADS] = v1;
      npend = rest;
      __syncthreads();
    }
    refill();
  }
  if (!ok && tid == 0) atomicOr(status, 2);
  if (ok && chunk >= 1 && !drain(chunk - 1)) {
    if (tid == 0) atomicOr(status, 2);
    ok = false;
  }
  // ---- epilogue
  if (ok && (chunk > 0 || nslab == 1)) {
    const int m = 32 * q + lane;
    const int x = o0 + (m >> 3), y = o1 + (m & 7);
    if (x < g.m[0] && y < g.m[1]) {
      const size_t row = (size_t)x * xst + (size_t)y * g.n[2];
#pragma unroll
      for (int i = 0; i < 24; ++i) {
        const int n = 24 * half + i, z = o2 + n / CG, c = n % CG;
        if (z < g.m[2] && c < C) {
          float* dst = grid + (size_t)(c0 + c) * cst + row + z;
          if (nslab == 1) *dst = acc[i];
          else atomicAdd(dst, acc[i]);
        }
      }
    }
  }
  if (!ok && last >= 0) {
    // a wait gave up: the commit of the last chunk arrives once every MMA this CTA issued has
    // completed; wait for it (bounded) before the accumulators' tensor memory is released
    mbar_wait(&sm.mbar[last & 1], (uint32_t)((last >> 1) & 1));
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

template <int Z, int CG>
se_status launch_group(se_plan_t* p, const int* tile_start, const int* base, const float* w, const float* sf,
                       int Ctot, int c0, int C, float* grid, long long cst, long long xst) {
  const GridGeom& g = p->geom;
  const size_t smem = sizeof(TcSmem<Z, CG>);
  // per function and device; set at every launch (a host-side call, cheap, thread-safe)
  SE_CUDA(cudaFuncSetAttribute(k_spread_tc<Z, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int t0 = cdiv(g.m[0], TC_X), t1 = cdiv(g.m[1], TC_Y), t2 = cdiv(g.m[2], Z);
  const long long tiles = (long long)t0 * t1 * t2;
  // two CTAs fit an SM; split the source bins of a tile over nslab CTAs when the tiles
  // alone would leave SMs idle (partial tiles are then added atomically into a zeroed grid)
  const int nslab = (int)std::min<long long>(8, std::max<long long>(1, (2LL * 152 + tiles - 1) / tiles));
  dim3 grd((unsigned)(t0 * nslab), (unsigned)t1, (unsigned)t2);
  ++p->launches;
  // SE_FLAG_TEST_TIMEOUT (a testing aid): the waits for finished chunks give up at once,
  // which exercises the timeout path (status, drain of the MMAs in flight, release)
  const long long drain_limit = (p->flags & SE_FLAG_TEST_TIMEOUT) ? 0 : TC_WAIT_LIMIT;
  k_spread_tc<Z, CG><<<grd, TC_THREADS, smem, p->stream>>>(g, tile_start, base, w, sf, Ctot, c0, C, nslab, grid,
                                                           cst, xst, p->d_status, drain_limit);
  SE_CUDA(cudaGetLastError());
  return SE_OK;
}

}  // namespace

// FP32 gridding of C components on the tensor cores: components in groups of 6 (8 grid
// points along direction 2 per tile) or a last group of up to 3 (16 points per tile).
se_status spread_tc_launch(se_plan_t* p, const int* tile_start, const int* base, const float* w, const float* sf,
                           int C, float* grid, long long cst, long long xst) {
  // tiles split over several CTAs add their partial tiles atomically: zero the whole grid first
  SE_CUDA(cudaMemsetAsync(grid, 0, sizeof(float) * (size_t)C * p->geom.cs, p->stream));
  for (int c0 = 0; c0 < C; c0 += 6) {
    const int Cc = std::min(6, C - c0);
    if (Cc <= 3) SE_TRY((launch_group<16, 3>(p, tile_start, base, w, sf, C, c0, Cc, grid, cst, xst)));
    else SE_TRY((launch_group<8, 6>(p, tile_start, base, w, sf, C, c0, Cc, grid, cst, xst)));
  }
  return SE_OK;
}

}  // namespace se
