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
// Layout trick: the six slices of one operand set live in shared memory as
// seven consecutive 64-row tiles [Z, A0, A1, A2, A3, A4, A5] (Z = zeros).  An
// M = 128 MMA starting at tile k reads rows [tile_k; tile_k+1] and so adds
// A_s B_t to the top half (level s + t) and A_(s+1) B_t to the bottom half
// (level s + t + 1) of a TMEM block: twelve MMAs per K-step cover the
// twenty-one slice pairs with s + t <= 5,
//   block 0 = [L0; L1]: [A0;A1] x B0, [Z;A0] x B1
//   block 1 = [L2; L3]: [A2;A3] x B0, [A1;A2] x B1, [A0;A1] x B2, [Z;A0] x B3
//   block 2 = [L4; L5]: [A4;A5] x B0, [A3;A4] x B1, [A2;A3] x B2,
//                       [A1;A2] x B3, [A0;A1] x B4, [Z;A0] x B5.
//
// Outputs per (batch, 64x64 tile): V = (D Phi)^T Phi, W0 = sum_q (D Q)^T Q
// (three products into one accumulator, sliced against a common exponent per
// function so that the exact levels keep one unit), and A_yz = (D Y)^T Z,
// A_zx = (D Z)^T X, A_xy = (D X)^T Y with SO_x = A_yz - A_yz^T etc. applied
// while scattering.  Persistent CTAs (128 threads, 256 TMEM columns, two
// per SM) loop over work items; every mbarrier wait is bounded and sets a
// status bit instead of hanging.
#include "internal.h"
#include "tc.cuh"

namespace q4c {
namespace split {
using namespace tc;

constexpr int kTile = 64;                    // functions per tile (rows of one half of M)
constexpr int kKc = 16;                      // points per step (one K = 16 MMA step)
constexpr int kTileBytes = kTile * kKc * 2;  // 2 KB
constexpr int kSBO = (kKc / 8) * 128;        // 256 B between 8-row groups
constexpr int kThreads = 256;
constexpr int kUnits = 16 / (kThreads / 32);  // slicing units per side per thread
constexpr int kMaxProducts = 3;
constexpr int kStageA = (kSlices + 1) * kTileBytes;  // [Z, A0..A5]
constexpr int kStageB = kSlices * kTileBytes;        // [B0..B5]
constexpr int kStage = kStageA + kStageB;            // 26 KB
constexpr int kSmemStages = 0;                       // two stages (double buffer)
constexpr int kSmemEpi = kSmemStages + 2 * kStage;   // epilogue staging, 24 KB
constexpr int kSmemD = kSmemEpi + 128 * 16 * 3 * 4;
constexpr int kMaxNp = 344;                          // D values of one batch (double-float)
constexpr int kSmemExp = kSmemD + kMaxNp * 8;
constexpr int kSmemBar = kSmemExp + 2 * kTile * 4;
constexpr int kSmemTotal = kSmemBar + 64;
constexpr uint32_t kTmemCols = 256;  // three 64-column blocks

// ------------------------------------------------------------ kernel
struct Products {
  int n;
  int qa[kMaxProducts];  // A-side (D-scaled) quantity: 0 Phi, 1 X, 2 Y, 3 Z
  int qb[kMaxProducts];  // B-side quantity
};

__device__ __forceinline__ Products products_of(int o) {
  Products P;
  switch (o) {
    case 0: P.n = 1; P.qa[0] = 0; P.qb[0] = 0; break;              // V
    case 1: P.n = 3; P.qa[0] = 1; P.qb[0] = 1; P.qa[1] = 2; P.qb[1] = 2; P.qa[2] = 3; P.qb[2] = 3; break;  // W0
    case 2: P.n = 1; P.qa[0] = 2; P.qb[0] = 3; break;              // A_yz -> SO_x
    case 3: P.n = 1; P.qa[0] = 3; P.qb[0] = 1; break;              // A_zx -> SO_y
    default: P.n = 1; P.qa[0] = 1; P.qb[0] = 2; break;             // A_xy -> SO_z
  }
  return P;
}

__device__ __forceinline__ int local_nf(const DevBasis& B, const DevGrid& G, int a0, int a) {
  return __ldg(B.sp_nfn + G.atom_sp[G.bat_atoms[a0 + a]]);
}

// One work item = (batch, output, 64x64 tile).  Its K dimension is a stream
// of steps of 16 points; W0 streams its three gradient products one after
// the other (a K-concatenation into one accumulator, common exponents).
// Steps alternate between two shared-memory stages: the 128 threads slice
// step s + 1 while the tensor core runs the twelve MMAs of step s.
__global__ void __launch_bounds__(kThreads, 2)
    k_split_products(DevBasis B, DevGrid G, const int4* __restrict__ items, int n_items, int* counter,
                     const int64_t* __restrict__ scr_off, const double* __restrict__ scratch,
                     const int* __restrict__ colexp, const double* __restrict__ v, double* V, double* W0,
                     double* SOx, double* SOy, double* SOz, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* stage = reinterpret_cast<float*>(smem + kSmemEpi);
  df* sD = reinterpret_cast<df*>(smem + kSmemD);
  float* sMagA = reinterpret_cast<float*>(smem + kSmemExp);  // rounding constants of the rows
  float* sMagB = sMagA + kTile;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSmemBar);  // two barriers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSmemBar + 16);
  int* s_item = reinterpret_cast<int*>(smem + kSmemBar + 32);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_addr[2] = {smem_u32(bar), smem_u32(bar + 1)};

  // zero tile Z at the head of each stage (never overwritten)
  for (int i = tid; i < 2 * kTileBytes / 16; i += kThreads) {
    const int st = i / (kTileBytes / 16), off = i - st * (kTileBytes / 16);
    reinterpret_cast<uint4*>(smem + kSmemStages + st * kStage)[off] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    mbar_init(bar_addr[0], 1);
    mbar_init(bar_addr[1], 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t ph[2] = {0, 0};
  bool pending[2] = {false, false};  // a commit on this stage not yet waited for
  bool ok = true;

  while (ok) {
    if (tid == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= n_items) break;
    const int4 item = items[it];
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
    const int ncols = min(kTile, nb - j0);
    const int N = (ncols + 15) & ~15;
    const uint32_t idesc = make_idesc(128, N);

    // Column exponents (W0: one exponent per function over its three gradient
    // components, so that its K-concatenated products share units) and D.
    if (tid < kTile) {
      const int r = tid;
      int ea = -30000, eb = -30000;
      if (o == 1) {
        if (i0 + r < nb) ea = max(cexp[1 * nb + i0 + r], max(cexp[2 * nb + i0 + r], cexp[3 * nb + i0 + r]));
        if (j0 + r < nb) eb = max(cexp[5 * nb + j0 + r], max(cexp[6 * nb + j0 + r], cexp[7 * nb + j0 + r]));
      } else {
        if (i0 + r < nb) ea = cexp[P.qa[0] * nb + i0 + r];
        if (j0 + r < nb) eb = cexp[(4 + P.qb[0]) * nb + j0 + r];
      }
      sMagA[r] = magic0(ea);
      sMagB[r] = magic0(eb);
    }
    for (int p = tid; p < np; p += kThreads) {
      const double Dp = G.w[p0 + p] * v[p0 + p];
      const float h = static_cast<float>(Dp);
      sD[p] = df{h, static_cast<float>(Dp - static_cast<double>(h))};
    }
    __syncthreads();

    const int n_chunks = (np + kKc - 1) / kKc;
    const int n_steps = n_chunks * P.n;
    for (int s = 0; s < n_steps && ok; ++s) {
      const int buf = s & 1;
      if (pending[buf]) {  // the stage is free once the MMAs that read it finished
        ok = __syncthreads_and(mbar_wait(bar_addr[buf], ph[buf], status));
        ph[buf] ^= 1;
        pending[buf] = false;
        if (!ok) break;
      }
      const int c = s / P.n, pr = s - c * P.n;
      const int kc0 = c * kKc;
      unsigned char* sA = smem + kSmemStages + buf * kStage;
      unsigned char* sB = sA + kStageA;
      // all global loads of the step first (eight units per thread: four per
      // side), then the splitting and the shared-memory stores
      float2 xs[2][kUnits][2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int q = side == 0 ? P.qa[pr] : P.qb[pr];
        const int row0 = side == 0 ? i0 : j0;
#pragma unroll
        for (int k = 0; k < kUnits; ++k) {
          const int u = warp + (kThreads / 32) * k;
          const int r = (u >> 1) * 8 + (lane >> 2), p = kc0 + 2 * ((u & 1) * 4 + (lane & 3));
          const int f = row0 + r;
          const float2* src = base + q * plane + static_cast<int64_t>(f) * ldp + p;
          xs[side][k][0] = (f < nb && p < np) ? src[0] : make_float2(0.f, 0.f);
          xs[side][k][1] = (f < nb && p + 1 < np) ? src[1] : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const float* mg = side == 0 ? sMagA : sMagB;
        unsigned char* dst = side == 0 ? sA + kTileBytes : sB;
#pragma unroll
        for (int k = 0; k < kUnits; ++k) {
          const int u = warp + (kThreads / 32) * k;
          const int rg = u >> 1, kq = u & 1;
          const int r = rg * 8 + (lane >> 2), p = kc0 + 2 * (kq * 4 + (lane & 3));
          const float m0 = mg[r];
          float d0[kSlices], d1[kSlices];
          if (side == 0) {  // A side: D-scaled values, the product in double-float
            const df a0v = p < np ? df_mul(df{xs[0][k][0].x, xs[0][k][0].y}, sD[p]) : df{0.f, 0.f};
            const df a1v = p + 1 < np ? df_mul(df{xs[0][k][1].x, xs[0][k][1].y}, sD[p + 1]) : df{0.f, 0.f};
            slice6(a0v.hi, a0v.lo, m0, d0);
            slice6(a1v.hi, a1v.lo, m0, d1);
          } else {
            slice6(xs[1][k][0].x, xs[1][k][0].y, m0, d0);
            slice6(xs[1][k][1].x, xs[1][k][1].y, m0, d1);
          }
          const int off = rg * kSBO + kq * kLBO + (lane >> 2) * 16 + (lane & 3) * 4;
#pragma unroll
          for (int t = 0; t < kSlices; ++t)
            *reinterpret_cast<__nv_bfloat162*>(dst + t * kTileBytes + off) = __floats2bfloat162_rn(d0[t], d1[t]);
        }
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a = smem_u32(sA), bb = smem_u32(sB);
        const uint32_t t0 = tmem, t1 = tmem + kTile, t2 = tmem + 2 * kTile;
        const uint32_t acc = s == 0 ? 0u : 1u;
        auto A = [&](int k) { return make_desc(a + k * kTileBytes, kSBO); };
        auto Bt = [&](int t) { return make_desc(bb + t * kTileBytes, kSBO); };
        mma_bf16(t0, A(1), Bt(0), idesc, acc);  // [A0;A1] x B0 -> L0, L1
        mma_bf16(t0, A(0), Bt(1), idesc, 1u);   // [Z;A0]  x B1 -> L1
        mma_bf16(t1, A(3), Bt(0), idesc, acc);  // [A2;A3] x B0 -> L2, L3
        mma_bf16(t1, A(2), Bt(1), idesc, 1u);   // [A1;A2] x B1
        mma_bf16(t1, A(1), Bt(2), idesc, 1u);   // [A0;A1] x B2
        mma_bf16(t1, A(0), Bt(3), idesc, 1u);   // [Z;A0]  x B3 -> L3
        mma_bf16(t2, A(5), Bt(0), idesc, acc);  // [A4;A5] x B0 -> L4, L5
        mma_bf16(t2, A(4), Bt(1), idesc, 1u);   // [A3;A4] x B1
        mma_bf16(t2, A(3), Bt(2), idesc, 1u);   // [A2;A3] x B2
        mma_bf16(t2, A(2), Bt(3), idesc, 1u);   // [A1;A2] x B3
        mma_bf16(t2, A(1), Bt(4), idesc, 1u);   // [A0;A1] x B4
        mma_bf16(t2, A(0), Bt(5), idesc, 1u);   // [Z;A0]  x B5 -> L5
        mma_commit(bar_addr[buf]);
      }
      pending[buf] = true;
    }
    if (!ok) break;
    // drain the outstanding commits (oldest first) before reading TMEM
    for (int d = 0; d < 2 && ok; ++d) {
      const int buf = (n_steps + d) & 1;
      if (!pending[buf]) continue;
      ok = __syncthreads_and(mbar_wait(bar_addr[buf], ph[buf], status));
      ph[buf] ^= 1;
      pending[buf] = false;
    }
    tc_fence_after();
    if (!ok) break;

    // epilogue: combine the six levels per element, scatter into FP64
    const int64_t f0 = G.bat_fn_ptr[b];
    const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
    const int64_t pp = G.bat_pair_ptr[b];
    double* out = o == 0 ? V : o == 1 ? W0 : o == 2 ? SOx : o == 3 ? SOy : SOz;
    for (int c0 = 0; c0 < N; c0 += 16) {
      if (warp < 4) {  // warp w reads TMEM lanes 32w..32w+31
        const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
#pragma unroll
        for (int blk = 0; blk < 3; ++blk) {
          float vv[16];
          tmem_ld16(tmem + lane_base + blk * kTile + c0, vv);
#pragma unroll
          for (int i = 0; i < 16; ++i) stage[(tid * 16 + i) * 3 + blk] = vv[i];
        }
      }
      __syncthreads();
      const int r = tid & 63, part = tid >> 6;
      const int i = i0 + r;
      for (int cc = 0; cc < 16 / (kThreads / 64); ++cc) {
        const int col = part * (16 / (kThreads / 64)) + cc;
        const int j = j0 + c0 + col;
        if (i >= nb || j >= nb) continue;
        const float* top = stage + (r * 16 + col) * 3;
        const float* bot = stage + ((r + 64) * 16 + col) * 3;
        const float L0 = top[0], L1 = bot[0], L2 = top[1], L3 = bot[1], L4 = top[2], L5 = bot[2];
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
        const int ii = G.fn_info[f0 + ri], jj = G.fn_info[f0 + rj];
        const int ai = ii >> 16, ki = ii & 0xffff, aj = jj >> 16, kj = jj & 0xffff;
        const int64_t off = G.pair_off[pp + static_cast<int64_t>(ai) * na + aj];
        if (off < 0) continue;
        atomicAdd(out + off + static_cast<int64_t>(ki) * local_nf(B, G, a0, aj) + kj, sgn * val);
      }
      __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
  }
  // on an expired wait give in-flight MMAs one more bounded chance before freeing TMEM
  if (!ok) {
    for (int d = 0; d < 2; ++d)
      if (pending[d]) (void)__syncthreads_and(mbar_wait(bar_addr[d], ph[d], status));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
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
  Q4C_CUDA(cudaMemsetAsync(g->d_counter, 0, sizeof(int) * std::max(n_waves, 1), s));
  Q4C_CUDA(cudaFuncSetAttribute(split::k_split_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                split::kSmemTotal));
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_basis_df(t, g, b0, b1, v, g->d_colexp, nullptr, s)) return st;
    const int64_t i0 = g->split_w0[wv], i1 = g->split_w0[wv + 1];
    const int n_items = static_cast<int>(i1 - i0);
    if (n_items == 0) continue;
    const int grid = std::min(n_items, 2 * n_sm);
    {
      KernelScope ks("split_products", s);
      split::k_split_products<<<grid, split::kThreads, split::kSmemTotal, s>>>(
          t->view(), g->view(), g->d_split_items + i0, n_items, g->d_counter + wv, g->d_scr_off, g->d_scratch,
          g->d_colexp, v, out->V, out->W0, out->SOx, out->SOy, out->SOz, g->d_status);
    }
    Q4C_CUDA(cudaGetLastError());
  }
  return mirror_and_spinor(g, out, s);
}

}  // namespace q4c
