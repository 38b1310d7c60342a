// Split-precision batch products on the tcgen05 tensor cores.
//
// Every batch product C = (D Q_a)^T Q_b (Eqs. 29-32 with F = v; D = diag(w v),
// Q in {Phi, X, Y, Z}) is computed exactly enough for ~1e-9 relative error
// from BF16 slices (an Ozaki-type error-free splitting; Ozaki, Ogita, Oishi
// and Rump 2012):
//   x = sum_s d_s 2^(e - 6 - 8s),  s = 0..5,  |d_0| <= 64, |d_1|, |d_2| <= 128,
//   |d_3| <= 160, |d_4|, |d_5| <= 128,
// with e a per-column binary exponent (|x| <= 2^e over the batch); the digits
// come from FP32 round-to-multiple steps (tc::slice6).  Each digit has <= 8
// significant bits, so it is exact in BF16 and every slice product is exact
// in FP32.  Per output element six FP32 accumulators (one per level s + t)
// are kept in tensor memory:
//   L0 = sum d0 e0, L1 = sum d0 e1 + d1 e0, L2 = sum_{s+t=2} d_s e_t
//       (integer sums of at most 2^15 units per term: exact for K <= 512
//       terms, i.e. n_p <= 512 for V and the A products and n_p <= 170 for
//       the 3 n_p terms of W0; beyond that a rounding of L2 sits ~2^-40
//       below the column scale)
//   L3, L4, L5 (rounded; 2^-24 and further below L0, so the truncating FP32
//       accumulation of the tensor cores cannot reach the result's bits)
// and combined as a double-float, then added into the FP64 block pattern.
//
// The precision is relative to the column maxima of each batch, which near
// heavy nuclei sit far above the typical values, hence six slices (47 bits).
//
// Layout trick: the six slices of the A operand live in shared memory as
// seven consecutive 64-row tiles [Z, A0, A1, A2, A3, A4, A5] (Z = zeros), so an
// M = 128 MMA starting at tile k reads rows [A_(k-1); A_k] and adds A_s B_t to
// the top half (level s + t) and A_(s+1) B_t to the bottom half (level
// s + t + 1) of a TMEM block; the B slices are stored [B0, B2, B4, B1, B3, B5],
// so one MMA with N = 64, 128 or 192 covers B_t, B_(t+2), ... and lands in
// consecutive blocks [L0;L1], [L2;L3], [L4;L5].  Six MMAs per K-step cover the
// twenty-one slice pairs with s + t <= 5 (tc::mma_levels lists them).
//
// Outputs per (batch, 64x64 tile): V = (D Phi)^T Phi, W0 = sum_q (D Q)^T Q
// (three products into one accumulator, sliced against a common exponent per
// function so that the exact levels keep one unit), and A_yz = (D Y)^T Z,
// A_zx = (D Z)^T X, A_xy = (D X)^T Y with SO_x = A_yz - A_yz^T etc. applied
// while scattering.  One warp-specialised CTA per SM (slicers, one MMA
// thread, epilogue warps; 512 TMEM columns) loops over the work items; every
// mbarrier wait is bounded and sets a status bit instead of hanging.
#include "internal.h"
#include "tc.cuh"

namespace q4c {
namespace split {
using namespace tc;

constexpr int kTile = 64;                    // functions per tile (rows of one half of M)
constexpr int kKc = 16;                      // points per step (one K = 16 MMA step)
constexpr int kTileBytes = kTile * kKc * 2;  // 2 KB
constexpr int kSBO = (kKc / 8) * 128;        // 256 B between 8-row groups
constexpr int kSlicers = 256;                // warps 0-7 slice the operands
constexpr int kEpiWarp0 = 8;                 // warps 8-15 drain tensor memory (two groups of four)
constexpr int kEpiThreads = 256;
constexpr int kMmaWarp = 16;                 // warp 16 owns tensor memory and issues the MMAs
constexpr int kThreads = 17 * 32;
constexpr int kEpiPitch = 17;                // floats per staged TMEM lane (16 columns + pad)
constexpr int kEpiStage = 3 * 128 * kEpiPitch * 4;  // one group's staging, 26 KB
constexpr int kUnits = 16 / (kSlicers / 32);  // slicing units per side per thread
constexpr int kMaxProducts = 3;
constexpr int kStageA = (kSlices + 1) * kTileBytes;  // [Z, A0..A5]
constexpr int kStageB = kSlices * kTileBytes;        // [B0..B5]
constexpr int kStage = kStageA + kStageB;            // 26 KB
constexpr int kStages = 4;                           // ring depth of sliced operands
constexpr int kRaw = 4;                              // ring depth of raw operand values
constexpr int kRawStage = kSlicers * 2 * kUnits * 16;  // one step's float2 pairs, 16 KB
constexpr int kSmemStages = 0;
constexpr int kSmemEpi = kSmemStages + kStages * kStage;  // epilogue staging, 2 x 26 KB
constexpr int kSmemRaw = kSmemEpi + 2 * kEpiStage;
constexpr int kSmemD = kSmemRaw + kRaw * kRawStage;
constexpr int kMaxNp = 344;  // D values of one batch (double-float)
constexpr int kSmemExp = kSmemD + kMaxNp * 8;
constexpr int kSmemBar = kSmemExp + 2 * kTile * 4;
constexpr int kNumBars = 2 * kStages + 5;  // full[S], empty[S], accfull[2], accempty[2], drain
constexpr int kSmemTotal = kSmemBar + kNumBars * 8 + 16;
constexpr uint32_t kTmemCols = 512;  // two accumulator sets of three 64-column blocks
constexpr uint32_t kSetCols = 256;

// ------------------------------------------------------------ kernel
// The products of one output, in registers: n of them, the A-side (D-scaled)
// and B-side quantities of product pr in bits 2pr..2pr+1 of qa and qb
// (0 Phi, 1 X, 2 Y, 3 Z).
struct Products {
  int n;
  unsigned qa, qb;
  __device__ __forceinline__ int a(int pr) const { return static_cast<int>((qa >> (2 * pr)) & 3u); }
  __device__ __forceinline__ int b(int pr) const { return static_cast<int>((qb >> (2 * pr)) & 3u); }
};

__device__ __forceinline__ Products products_of(int o) {
  switch (o) {
    case 0: return {1, 0u, 0u};                // V
    case 1: return {3, 0x39u, 0x39u};          // W0: (X, X), (Y, Y), (Z, Z)
    case 2: return {1, 2u, 3u};                // A_yz -> SO_x
    case 3: return {1, 3u, 1u};                // A_zx -> SO_y
    default: return {1, 1u, 2u};               // A_xy -> SO_z
  }
}

__device__ __forceinline__ int item_steps(const DevGrid& G, int4 item) {
  const int np = static_cast<int>(G.pt_ptr[item.x + 1] - G.pt_ptr[item.x]);
  return ((np + kKc - 1) / kKc) * (item.y == 1 ? 3 : 1);
}

// Issue the asynchronous copies of one K-step's operand values for this
// thread: per side, kUnits units of two consecutive points (16 bytes each)
// into its slots of a raw stage (slot (side * kUnits + k) * kSlicers + tid).
// Values past the batch's points or functions arrive as zeros.
__device__ __forceinline__ void issue_step(const float2* base, int64_t plane, int ldp, int np, int nb, int i0,
                                           int j0, const Products& P, int s, int warp, int lane, int tid,
                                           uint32_t raw) {
  const int c = P.n == 1 ? s : s / 3, pr = s - c * P.n;
  const int kc0 = c * kKc;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int q = side == 0 ? P.a(pr) : P.b(pr);
    const int row0 = side == 0 ? i0 : j0;
#pragma unroll
    for (int k = 0; k < kUnits; ++k) {
      const int u = warp + (kSlicers / 32) * k;
      const int r = (u >> 1) * 8 + (lane >> 2), p = kc0 + 2 * ((u & 1) * 4 + (lane & 3));
      const int f = row0 + r;
      const bool live = f < nb && p < np;
      const int bytes = !live ? 0 : (p + 1 < np ? 16 : 8);  // row padding is not written
      const float2* src = live ? base + q * plane + static_cast<int64_t>(f) * ldp + p : base;
      cp_async16(raw + ((side * kUnits + k) * kSlicers + tid) * 16, src, bytes);
    }
  }
}

// One work item = (batch, output, 64x64 tile).  Its K dimension is a stream
// of steps of 16 points; W0 streams its three gradient products one after
// the other (a K-concatenation into one accumulator, common exponents).
//
// Warp roles (one CTA per SM, items strided over the CTAs):
//   warps 0-7   slice step g into ring stage g mod 4 once the MMAs that last
//               read it have completed (empty[stage], a tcgen05.commit), then
//               arrive on full[stage]; each thread's raw values arrive by
//               cp.async three steps ahead, in a ring of its own;
//   warp 16     (one thread) waits full[stage], issues the six MMAs into the
//               item's accumulator set (items alternate between two sets of
//               192 TMEM columns), commits empty[stage], and after an item's
//               last step commits accfull[set];
//   warps 8-15  wait accfull[set], read the six levels, combine and scatter
//               (two groups of four warps take alternate 16-column chunks;
//               the scatter offsets come from the batch's dense offset
//               table), then arrive on accempty[set] so the set can take
//               item k + 2.
// Every wait is bounded; a role that times out sets the status bit and an
// abort flag that ends the other roles' waits, and the MMA thread drains its
// outstanding MMAs (bounded) before tensor memory is freed.
__global__ void __launch_bounds__(kThreads, 1)
    k_split_products(DevBasis B, DevGrid G, const int4* __restrict__ items, int n_items,
                     const int64_t* __restrict__ scr_off, const double* __restrict__ scratch,
                     const int* __restrict__ colexp, const double* __restrict__ v, double* V, double* W0,
                     double* SOx, double* SOy, double* SOz, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* stage = reinterpret_cast<float*>(smem + kSmemEpi);
  df* sD = reinterpret_cast<df*>(smem + kSmemD);
  float* sMagA = reinterpret_cast<float*>(smem + kSmemExp);  // rounding constants of the rows
  float* sMagB = sMagA + kTile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSmemBar + kNumBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kSmemBar + kNumBars * 8 + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int st) { return bar0 + 8u * st; };
  auto empty_bar = [&](int st) { return bar0 + 8u * (kStages + st); };
  auto accfull_bar = [&](int set) { return bar0 + 8u * (2 * kStages + set); };
  auto accempty_bar = [&](int set) { return bar0 + 8u * (2 * kStages + 2 + set); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 4);

  // zero tile Z at the head of each stage (never overwritten)
  for (int i = tid; i < kStages * kTileBytes / 16; i += kThreads) {
    const int st = i / (kTileBytes / 16), off = i - st * (kTileBytes / 16);
    reinterpret_cast<uint4*>(smem + kSmemStages + st * kStage)[off] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(full_bar(st), kSlicers);
      mbar_init(empty_bar(st), 1);
    }
    for (int set = 0; set < 2; ++set) {
      mbar_init(accfull_bar(set), 1);
      mbar_init(accempty_bar(set), kEpiThreads);
    }
    mbar_init(drain_bar, 1);
    *s_abort = 0;
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < kSlicers / 32) {
    // ---------------------------------------------------------- slicers
    bool ok = true;
    int g = 0;  // steps sliced by this CTA
    for (int n = blockIdx.x;; n += gridDim.x) {
      // the previous item's constants are no longer read; agree on stopping
      if (bar_red_or(1, kSlicers, !ok || *s_abort) || n >= n_items) break;
      const int4 item = items[n];
      const int64_t b = item.x;
      const int o = item.y, ti = item.z, tj = item.w;
      const int64_t p0 = G.pt_ptr[b];
      const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
      const int ldp = (np + 7) & ~7;
      const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
      const int64_t plane = static_cast<int64_t>(nb) * ldp;
      const float2* base = reinterpret_cast<const float2*>(scratch) + scr_off[b];
      const int* cexp = colexp + 8 * G.bat_fn_ptr[b];
      const Products P = products_of(o);
      const int i0 = ti * kTile, j0 = tj * kTile;
      // Column exponents (W0: one exponent per function over its three gradient
      // components, so that its K-concatenated products share units) and D.
      if (tid < kTile) {
        const int r = tid;
        int ea = -30000, eb = -30000;
        if (o == 1) {
          if (i0 + r < nb) ea = max(cexp[1 * nb + i0 + r], max(cexp[2 * nb + i0 + r], cexp[3 * nb + i0 + r]));
          if (j0 + r < nb) eb = max(cexp[5 * nb + j0 + r], max(cexp[6 * nb + j0 + r], cexp[7 * nb + j0 + r]));
        } else {
          if (i0 + r < nb) ea = cexp[P.a(0) * nb + i0 + r];
          if (j0 + r < nb) eb = cexp[(4 + P.b(0)) * nb + j0 + r];
        }
        sMagA[r] = magic0(ea);
        sMagB[r] = magic0(eb);
      }
      for (int p = tid; p < np; p += kSlicers) {
        const double Dp = G.w[p0 + p] * v[p0 + p];
        const float h = static_cast<float>(Dp);
        sD[p] = df{h, static_cast<float>(Dp - static_cast<double>(h))};
      }
      bar_sync(1, kSlicers);
      const int n_steps = item_steps(G, item);
      const uint32_t raw0 = smem_u32(smem + kSmemRaw);
      // copies run kRaw - 1 steps ahead of the slicing (one commit group per step)
#pragma unroll
      for (int q = 0; q < kRaw - 1; ++q) {
        if (q < n_steps) issue_step(base, plane, ldp, np, nb, i0, j0, P, q, warp, lane, tid, raw0 + q * kRawStage);
        cp_async_commit();
      }
      for (int s = 0; s < n_steps; ++s, ++g) {
        const int sa = s + kRaw - 1;
        if (sa < n_steps)
          issue_step(base, plane, ldp, np, nb, i0, j0, P, sa, warp, lane, tid, raw0 + (sa % kRaw) * kRawStage);
        cp_async_commit();
        cp_async_wait<kRaw - 1>();  // this thread's copies of step s have landed
        const float4* rawp = reinterpret_cast<const float4*>(smem + kSmemRaw + (s % kRaw) * kRawStage);
        float4 cur[2][kUnits];
#pragma unroll
        for (int side = 0; side < 2; ++side)
#pragma unroll
          for (int k = 0; k < kUnits; ++k) cur[side][k] = rawp[(side * kUnits + k) * kSlicers + tid];
        const int st = g % kStages;
        if (!mbar_wait_abort(empty_bar(st), ((g / kStages) & 1) ^ 1, s_abort, status)) {
          ok = false;
          break;
        }
        const int c = P.n == 1 ? s : s / 3;
        const int kc0 = c * kKc;
        unsigned char* sA = smem + kSmemStages + st * kStage;
        unsigned char* sB = sA + kStageA;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const float* mg = side == 0 ? sMagA : sMagB;
          unsigned char* dst = side == 0 ? sA + kTileBytes : sB;
#pragma unroll
          for (int k = 0; k < kUnits; ++k) {
            const int u = warp + (kSlicers / 32) * k;
            const int rg = u >> 1, kq = u & 1;
            const int r = rg * 8 + (lane >> 2), p = kc0 + 2 * (kq * 4 + (lane & 3));
            const float m0 = mg[r];
            const float4 x = cur[side][k];
            float d0[kSlices], d1[kSlices];
            if (side == 0) {  // A side: D-scaled values, the product in double-float
              const df a0v = p < np ? df_mul(df{x.x, x.y}, sD[p]) : df{0.f, 0.f};
              const df a1v = p + 1 < np ? df_mul(df{x.z, x.w}, sD[p + 1]) : df{0.f, 0.f};
              slice6(a0v.hi, a0v.lo, m0, d0);
              slice6(a1v.hi, a1v.lo, m0, d1);
            } else {
              slice6(x.x, x.y, m0, d0);
              slice6(x.z, x.w, m0, d1);
            }
            const int off = rg * kSBO + kq * kLBO + (lane >> 2) * 16 + (lane & 3) * 4;
#pragma unroll
            for (int t = 0; t < kSlices; ++t)  // A: [Z, A0..A5]; B: [B0, B2, B4, B1, B3, B5]
              *reinterpret_cast<__nv_bfloat162*>(dst + (side == 0 ? t : b_tile(t)) * kTileBytes + off) =
                  __floats2bfloat162_rn(d0[t], d1[t]);
          }
        }
        fence_async_smem();
        mbar_arrive(full_bar(st));
      }
      cp_async_wait<0>();  // no copy of this item outlives it
    }
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      int g = 0, k = 0;
      for (int n = blockIdx.x; n < n_items; n += gridDim.x, ++k) {
        const int4 item = items[n];
        const int n_steps = item_steps(G, item);
        const int set = k & 1;
        if (!mbar_wait_abort(accempty_bar(set), ((k >> 1) & 1) ^ 1, s_abort, status, 64)) break;
        tc_fence_after();
        const uint32_t t0 = tmem + set * kSetCols;
        bool ok = true;
        for (int s = 0; s < n_steps; ++s, ++g) {
          const int st = g % kStages;
          if (!mbar_wait_abort(full_bar(st), (g / kStages) & 1, s_abort, status, 32)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + kSmemStages + st * kStage), bb = a + kStageA;
          mma_levels(t0, a, bb, s == 0 ? 0u : 1u);
          mma_commit(empty_bar(st));
        }
        if (!ok) break;
        mma_commit(accfull_bar(set));
      }
      // every MMA issued by this thread has completed before tensor memory is freed
      mma_commit(drain_bar);
      (void)mbar_wait(drain_bar, 0, status);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    const int eg = (warp - kEpiWarp0) >> 2;        // column group
    const int et = (warp & 3) * 32 + lane;         // TMEM lane 0..127
    const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
    float* stg = stage + eg * (kEpiStage / 4);
    int k = 0;
    for (int n = blockIdx.x; n < n_items; n += gridDim.x, ++k) {
      const int set = k & 1;
      bool ok = mbar_wait_abort(accfull_bar(set), (k >> 1) & 1, s_abort, status, 256);
      if (bar_red_or(2, kEpiThreads, !ok)) break;
      tc_fence_after();
      const int4 item = items[n];
      const int64_t b = item.x;
      const int o = item.y, i0 = item.z * kTile, j0 = item.w * kTile;
      const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
      const int N = (min(kTile, nb - j0) + 15) & ~15;
      const int* idx = G.bat_idx + G.bat_idx_ptr[b];
      double* out = o == 0 ? V : o == 1 ? W0 : o == 2 ? SOx : o == 3 ? SOy : SOz;
      for (int c0 = eg * 16; c0 < N; c0 += 32) {
#pragma unroll
        for (int blk = 0; blk < 3; ++blk) {
          float vv[16];
          tmem_ld16(tmem + lane_base + set * kSetCols + blk * kTile + c0, vv);
#pragma unroll
          for (int i = 0; i < 16; ++i) stg[(blk * 128 + et) * kEpiPitch + i] = vv[i];
        }
        bar_sync(3 + eg, 128);
        // thread -> (column, rows): a warp covers 16 consecutive columns of two rows
        const int col = et & 15, j = j0 + c0 + col;
#pragma unroll 2
        for (int q = 0; q < 8; ++q) {
          const int r = (et >> 4) + 8 * q, i = i0 + r;
          if (i >= nb || j >= nb) continue;
          const float L0 = stg[r * kEpiPitch + col], L1 = stg[(r + 64) * kEpiPitch + col];
          const float L2 = stg[(128 + r) * kEpiPitch + col], L3 = stg[(192 + r) * kEpiPitch + col];
          const float L4 = stg[(256 + r) * kEpiPitch + col], L5 = stg[(320 + r) * kEpiPitch + col];
          // exact levels by two-sums, rounded tail on top
          float sm = L0 + L1;
          float bp = sm - L0;
          const float e1 = (L0 - (sm - bp)) + (L1 - bp);
          const float s1 = sm;
          sm = s1 + L2;
          bp = sm - s1;
          const float e2 = (s1 - (sm - bp)) + (L2 - bp);
          const float lo = (e1 + e2) + (L3 + (L4 + L5));
          const double val = static_cast<double>(sm) + static_cast<double>(lo);
          int ri = i, rj = j;
          double sgn = 1.0;
          if (o <= 1) {
            if (i > j) continue;
          } else {
            if (i == j) continue;
            if (i > j) { ri = j; rj = i; sgn = -1.0; }
          }
          const int off = __ldg(idx + ri * nb + rj);
          if (off >= 0) atomicAdd(out + off, sgn * val);
        }
        bar_sync(3 + eg, 128);
      }
      tc_fence_before();
      mbar_arrive(accempty_bar(set));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace split

q4c_status integrate_split(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* out,
                           cudaStream_t s) {
  if (g->max_np > 341) {  // exactness bound of the level sums (and the D buffer)
    set_error("q4c_integrate: the split path needs batches of at most 341 points");
    return Q4C_EUNSUPPORTED;
  }
  double* outs[5] = {out->V, out->W0, out->SOx, out->SOy, out->SOz};
  for (double* o : outs) Q4C_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * g->nnz, s));
  const int n_waves = static_cast<int>(g->wave_b0.size()) - 1;
  Q4C_CUDA(cudaFuncSetAttribute(split::k_split_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                split::kSmemTotal));
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_fill_idx(t, g, b0, b1, s)) return st;
    if (q4c_status st = launch_basis_df(t, g, b0, b1, v, g->d_colexp, nullptr, 4, s)) return st;
    const int64_t i0 = g->split_w0[wv], i1 = g->split_w0[wv + 1];
    const int n_items = static_cast<int>(i1 - i0);
    if (n_items == 0) continue;
    const int grid = std::min(n_items, n_sm);
    {
      KernelScope ks("split_products", s);
      split::k_split_products<<<grid, split::kThreads, split::kSmemTotal, s>>>(
          t->view(), g->view(), g->d_split_items + i0, n_items, g->d_scr_off, g->d_scratch,
          g->d_colexp, v, out->V, out->W0, out->SOx, out->SOy, out->SOz, g->d_status);
    }
    Q4C_CUDA(cudaGetLastError());
  }
  return mirror_and_spinor(g, out, s);
}

}  // namespace q4c
