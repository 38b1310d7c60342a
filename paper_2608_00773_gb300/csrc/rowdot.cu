// Split-precision density (Eqs. 39-40) and adjoint of the integration on the
// tcgen05 tensor cores.
//
// Both are row-dot contractions over the batch's active functions:
//   density   n_p     = sum_j Phi_pj (Phi P)_pj
//   adjoint   dL/dv_p = w_p [ sum_j Phi_pj (Phi G^V)_pj + sum_{Q=X,Y,Z} sum_j Q_pj (Q G^W)_pj
//                             + 2 sum_j ( Z_pj (Y Gx)_pj + X_pj (Z Gy)_pj + Y_pj (X Gz)_pj ) ]
// with Gk the antisymmetric part of G^SOk (the cross product is antisymmetric
// in i, j, so only that part contributes), i.e. seven products U = F G'
// (M = points, K = functions i, N = functions j) whose rows are dotted with
// R in the epilogue, one point per tensor-memory lane.
//
// Each U is computed from six BF16 slices of F (per-point exponents) and of
// G' (per-column exponents) with the same tile sequence and exact-level
// accumulation as the integration (see split.cu): levels 0-2 are exact
// integer sums (K = n_b <= 512), levels 3-5 are rounded 2^-24 below.
#include "internal.h"
#include "tc.cuh"

namespace q4c {
namespace rowdot {
using namespace tc;

constexpr int kTile = 64;                    // points per tile (and functions per j-tile)
constexpr int kKc = 16;                      // functions i per chunk (one K = 16 MMA step)
constexpr int kTileBytes = kTile * kKc * 2;  // 2 KB
constexpr int kSBO = (kKc / 8) * 128;        // 256 B
constexpr int kThreads = 256;
constexpr int kUnits = 16 / (kThreads / 32);  // slicing units per side per thread
constexpr int kSmemA = 0;                                      // two stages of [Z, A0..A5][B0..B5]
constexpr int kSmemStage = kSmemA + 2 * (2 * kSlices + 1) * kTileBytes;  // epilogue staging (24 KB)
constexpr int kSmemExpF = kSmemStage + 128 * 16 * 3 * 4;
constexpr int kSmemExpG = kSmemExpF + kTile * 4;
constexpr int kSmemY = kSmemExpG + kTile * 4;
constexpr int kSmemBar = kSmemY + kThreads * 8;
constexpr int kSmemTotal = kSmemBar + 64;
constexpr uint32_t kTmemCols = 256;
constexpr int kMaxNb = 512;

struct Product {
  int qf, gm, anti, qr;
  double factor;
};

__device__ __forceinline__ int local_nf(const DevBasis& B, const DevGrid& G, int a0, int a) {
  return __ldg(B.sp_nfn + G.atom_sp[G.bat_atoms[a0 + a]]);
}

// G'_ij of the batch (i, j local) through the batch's dense offset table
__device__ __forceinline__ double gprime(const double* M, const int* __restrict__ idx, int nb, int anti, int i,
                                         int j) {
  const int o = __ldg(idx + i * nb + j);
  const double g = o < 0 ? 0.0 : M[o];
  if (!anti) return g;
  const int oT = __ldg(idx + j * nb + i);
  return 0.5 * (g - (oT < 0 ? 0.0 : M[oT]));
}

// the same from the matrix as FP32 pairs (the antisymmetric part in double-float)
__device__ __forceinline__ df gprime_df(const float2* M, const int* __restrict__ idx, int nb, int anti, int i,
                                        int j) {
  const int o = __ldg(idx + i * nb + j);
  const float2 g = o < 0 ? make_float2(0.f, 0.f) : __ldg(M + o);
  if (!anti) return df{g.x, g.y};
  const int oT = __ldg(idx + j * nb + i);
  const float2 gT = oT < 0 ? make_float2(0.f, 0.f) : __ldg(M + oT);
  const df d = df_sub(df{g.x, g.y}, df{gT.x, gT.y});
  return df{0.5f * d.hi, 0.5f * d.lo};  // exact
}

// FP32-pair copy of an FP64 matrix: x = hi + lo within 2^-48 relative
__global__ void k_to_df(const double* __restrict__ M, int64_t n, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double x = M[i];
    const float h = __double2float_rn(x);
    out[i] = make_float2(h, __double2float_rn(x - static_cast<double>(h)));
  }
}

__device__ __forceinline__ int binexp(double x) {
  return static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF) - 1022;
}

// per batch, matrix and local function j: exponent of max_i |G'_ij|
// (G' the matrix itself, or its antisymmetric part for the SO seeds)
__global__ void k_gexp(DevBasis B, DevGrid G, int64_t b0, int n_mats, int anti_from, const double* M0,
                       const double* M1, const double* M2, const double* M3, const double* M4,
                       int* __restrict__ gexp) {
  const int64_t b = b0 + blockIdx.x;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  const int64_t f0 = G.bat_fn_ptr[b];
  const int* idx = G.bat_idx + G.bat_idx_ptr[b];
  const double* mats[5] = {M0, M1, M2, M3, M4};
  for (int e = threadIdx.x; e < n_mats * nb; e += blockDim.x) {
    const int m = e / nb, j = e - m * nb;
    int mx = -30000;
    if (mats[m]) {
      for (int i = 0; i < nb; ++i) {
        const double g = gprime(mats[m], idx, nb, m >= anti_from, i, j);
        if (g != 0.0) mx = max(mx, binexp(g));
      }
    }
    gexp[5 * f0 + m * nb + j] = mx;
  }
}

constexpr int kStageA = (kSlices + 1) * kTileBytes;  // [Z, A0..A5]
constexpr int kStage = kStageA + kSlices * kTileBytes;

// One work item = (batch, 64-point tile).  For every j-tile and product the K
// dimension (functions i) is a stream of 16-wide steps that alternate between
// two shared-memory stages: the threads slice step s + 1 while the tensor core
// runs the twelve MMAs of step s.
template <int MODE>  // 0: density, 1: adjoint
__global__ void __launch_bounds__(kThreads, 2)
    k_split_rowdot(DevBasis B, DevGrid G, const int2* __restrict__ items, int n_items, int* counter,
                   const int64_t* __restrict__ scr_off, const double* __restrict__ scratch,
                   const int* __restrict__ rowexp, const int* __restrict__ gexp, const float2* M0,
                   const float2* M1, const float2* M2, const float2* M3, const float2* M4, double* __restrict__ out,
                   unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* stage = reinterpret_cast<float*>(smem + kSmemStage);
  float* sMagF = reinterpret_cast<float*>(smem + kSmemExpF);  // rounding constants per point
  float* sMagG = reinterpret_cast<float*>(smem + kSmemExpG);  // and per function j
  double* sY = reinterpret_cast<double*>(smem + kSmemY);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSmemBar + 16);
  int* s_item = reinterpret_cast<int*>(smem + kSmemBar + 32);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_addr[2] = {smem_u32(bar), smem_u32(bar + 1)};
  const float2* mats[5] = {M0, M1, M2, M3, M4};
  // (F quantity, G matrix, antisymmetric part?, R quantity, factor)
  const Product prods_adj[7] = {{0, 0, 0, 0, 1.0}, {1, 1, 0, 1, 1.0}, {2, 1, 0, 2, 1.0}, {3, 1, 0, 3, 1.0},
                                {2, 2, 1, 3, 2.0}, {3, 3, 1, 1, 2.0}, {1, 4, 1, 2, 2.0}};
  const Product prod_den = {0, 0, 0, 0, 1.0};
  const int n_prod = MODE == 0 ? 1 : 7;

  for (int i = tid; i < 2 * kTileBytes / 16; i += kThreads) {  // tile Z of both stages
    const int st = i / (kTileBytes / 16), off = i - st * (kTileBytes / 16);
    reinterpret_cast<uint4*>(smem + kSmemA + st * kStage)[off] = make_uint4(0, 0, 0, 0);
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
  int gstep = 0;                     // steps issued by this CTA (stage = gstep & 1)
  bool ok = true;

  while (ok) {
    if (tid == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= n_items) break;
    const int2 item = items[it];
    const int64_t b = item.x;
    const int pt = item.y;
    const int64_t bp0 = G.pt_ptr[b];
    const int np = static_cast<int>(G.pt_ptr[b + 1] - bp0);
    const int ldp = (np + 7) & ~7;
    const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
    const int64_t plane = static_cast<int64_t>(nb) * ldp;
    const float2* base = reinterpret_cast<const float2*>(scratch) + scr_off[b];
    const int64_t f0 = G.bat_fn_ptr[b];
    const int* idx = G.bat_idx + G.bat_idx_ptr[b];
    const int r0 = pt * kTile;  // first point of the tile within the batch
    df y = {0.f, 0.f};          // partial of point r0 + (tid & 63)
    const int n_ic = (nb + kKc - 1) / kKc;

    for (int j0 = 0; j0 < nb && ok; j0 += kTile) {
      const int N = (min(kTile, nb - j0) + 15) & ~15;
      const uint32_t idesc = make_idesc(128, N);
      for (int k = 0; k < n_prod && ok; ++k) {
        const Product P = MODE == 0 ? prod_den : prods_adj[k];
        const float2* Gm = mats[P.gm];
        if (Gm == nullptr) continue;
        if (tid < kTile) {
          const int p = r0 + tid, j = j0 + tid;
          sMagF[tid] = magic0(p < np ? rowexp[4 * (bp0 + p) + P.qf] : -30000);
          sMagG[tid] = magic0(j < nb ? gexp[5 * f0 + P.gm * nb + j] : -30000);
        }
        __syncthreads();
        for (int ic = 0; ic < n_ic && ok; ++ic, ++gstep) {
          const int buf = gstep & 1;
          if (pending[buf]) {  // the stage is free once the MMAs that read it finished
            ok = __syncthreads_and(mbar_wait(bar_addr[buf], ph[buf], status));
            ph[buf] ^= 1;
            pending[buf] = false;
            if (!ok) break;
          }
          const int i0 = ic * kKc;
          unsigned char* sA = smem + kSmemA + buf * kStage;
          unsigned char* sB = sA + kStageA;
          // all loads and gathers of the step first, then the splitting
          float2 xa[kUnits][2];
          df xs[kUnits][2];
#pragma unroll
          for (int k = 0; k < kUnits; ++k) {
            const int u = warp + (kThreads / 32) * k;
            const int r = (u >> 1) * 8 + (lane >> 2), i = i0 + 2 * ((u & 1) * 4 + (lane & 3));
            const int p = r0 + r, j = j0 + r;
            const float2* src = base + P.qf * plane + static_cast<int64_t>(i) * ldp + p;
            xa[k][0] = (p < np && i < nb) ? src[0] : make_float2(0.f, 0.f);
            xa[k][1] = (p < np && i + 1 < nb) ? src[ldp] : make_float2(0.f, 0.f);
            xs[k][0] = (j < nb && i < nb) ? gprime_df(Gm, idx, nb, P.anti, i, j) : df{0.f, 0.f};
            xs[k][1] = (j < nb && i + 1 < nb) ? gprime_df(Gm, idx, nb, P.anti, i + 1, j) : df{0.f, 0.f};
          }
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            unsigned char* dst = side == 0 ? sA + kTileBytes : sB;
            const float* mg = side == 0 ? sMagF : sMagG;
#pragma unroll
            for (int k = 0; k < kUnits; ++k) {
              const int u = warp + (kThreads / 32) * k;
              const int rg = u >> 1, kq = u & 1;
              const int r = rg * 8 + (lane >> 2);
              const float m0 = mg[r];
              float d0[kSlices], d1[kSlices];
              if (side == 0) {
                slice6(xa[k][0].x, xa[k][0].y, m0, d0);
                slice6(xa[k][1].x, xa[k][1].y, m0, d1);
              } else {
                slice6(xs[k][0].hi, xs[k][0].lo, m0, d0);
                slice6(xs[k][1].hi, xs[k][1].lo, m0, d1);
              }
              const int off = rg * kSBO + kq * kLBO + (lane >> 2) * 16 + (lane & 3) * 4;
#pragma unroll
              for (int s = 0; s < kSlices; ++s)
                *reinterpret_cast<__nv_bfloat162*>(dst + s * kTileBytes + off) = __floats2bfloat162_rn(d0[s], d1[s]);
            }
          }
          fence_async_smem();
          __syncthreads();
          if (tid == 0) {
            tc_fence_after();
            const uint32_t a = smem_u32(sA), bb = smem_u32(sB);
            const uint32_t t0 = tmem, t1 = tmem + kTile, t2 = tmem + 2 * kTile;
            const uint32_t acc = ic == 0 ? 0u : 1u;
            auto A = [&](int q) { return make_desc(a + q * kTileBytes, kSBO); };
            auto Bt = [&](int t) { return make_desc(bb + t * kTileBytes, kSBO); };
            mma_bf16(t0, A(1), Bt(0), idesc, acc);
            mma_bf16(t0, A(0), Bt(1), idesc, 1u);
            mma_bf16(t1, A(3), Bt(0), idesc, acc);
            mma_bf16(t1, A(2), Bt(1), idesc, 1u);
            mma_bf16(t1, A(1), Bt(2), idesc, 1u);
            mma_bf16(t1, A(0), Bt(3), idesc, 1u);
            mma_bf16(t2, A(5), Bt(0), idesc, acc);
            mma_bf16(t2, A(4), Bt(1), idesc, 1u);
            mma_bf16(t2, A(3), Bt(2), idesc, 1u);
            mma_bf16(t2, A(2), Bt(3), idesc, 1u);
            mma_bf16(t2, A(1), Bt(4), idesc, 1u);
            mma_bf16(t2, A(0), Bt(5), idesc, 1u);
            mma_commit(bar_addr[buf]);
          }
          pending[buf] = true;
        }
        if (!ok) break;
        // drain the outstanding commits (oldest first) before reading TMEM
        for (int d = 0; d < 2 && ok; ++d) {
          const int buf = (gstep + d) & 1;
          if (!pending[buf]) continue;
          ok = __syncthreads_and(mbar_wait(bar_addr[buf], ph[buf], status));
          ph[buf] ^= 1;
          pending[buf] = false;
        }
        tc_fence_after();
        if (!ok) break;
        // epilogue: U_rj from the six levels, dotted with R_rj
        const int r = tid & 63, part = tid >> 6;
        const int p = r0 + r;
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
          if (p < np) {
            for (int cc = 0; cc < 16 / (kThreads / 64); ++cc) {
              const int col = part * (16 / (kThreads / 64)) + cc, j = j0 + c0 + col;
              if (j >= nb) continue;
              const float* top = stage + (r * 16 + col) * 3;
              const float* bot = stage + ((r + 64) * 16 + col) * 3;
              const float L0 = top[0], L1 = bot[0], L2 = top[1], L3 = bot[1], L4 = top[2], L5 = bot[2];
              float sm = L0 + L1;
              float bp = sm - L0;
              const float e1 = (L0 - (sm - bp)) + (L1 - bp);
              const float s1 = sm;
              sm = s1 + L2;
              bp = sm - s1;
              const float e2 = (s1 - (sm - bp)) + (L2 - bp);
              const float lo = (e1 + e2) + (L3 + (L4 + L5));
              const float2 Rv = base[P.qr * plane + static_cast<int64_t>(j) * ldp + p];
              const df prod = df_mul(df{Rv.x, Rv.y}, fast_two_sum(sm, lo));
              y = df_add(y, df_mul_f(prod, static_cast<float>(P.factor)));
            }
          }
          __syncthreads();
        }
        tc_fence_before();
        __syncthreads();
      }
    }
    // combine the column parts of each point and write
    sY[tid] = static_cast<double>(y.hi) + static_cast<double>(y.lo);
    __syncthreads();
    if (tid < kTile && r0 + tid < np) {
      const int64_t gp = bp0 + r0 + tid;
      double val = 0.0;
      for (int q = 0; q < kThreads / 64; ++q) val += sY[tid + 64 * q];
      out[gp] = MODE == 0 ? val : G.w[gp] * val;
    }
    __syncthreads();
  }
  if (!ok) {
    for (int d = 0; d < 2; ++d)
      if (pending[d]) (void)__syncthreads_and(mbar_wait(bar_addr[d], ph[d], status));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int MODE>
q4c_status run(const q4c_tables* t, const q4c_grid* g, const double* const mats[5], double* out, cudaStream_t s) {
  if (g->max_nb > kMaxNb) {
    set_error("the split density/adjoint need at most 512 active functions per batch");
    return Q4C_EUNSUPPORTED;
  }
  const int n_waves = static_cast<int>(g->wave_b0.size()) - 1;
  Q4C_CUDA(cudaMemsetAsync(g->d_counter, 0, sizeof(int) * std::max(n_waves, 1), s));
  Q4C_CUDA(cudaFuncSetAttribute(k_split_rowdot<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal));
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // FP32-pair copies of the matrices for the B operands
  const float2* mdf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  {
    KernelScope ks(MODE == 0 ? "split_density" : "split_backward", s);
    for (int m = 0; m < 5; ++m) {
      if (!mats[m] || g->nnz == 0) continue;
      float2* dst = g->d_gdf + m * g->nnz;
      const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((g->nnz + 255) / 256, 8 * n_sm));
      k_to_df<<<blocks, 256, 0, s>>>(mats[m], g->nnz, dst);
      mdf[m] = dst;
    }
  }
  Q4C_CUDA(cudaGetLastError());
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_basis_df(t, g, b0, b1, nullptr, nullptr, g->d_rowexp, s)) return st;
    {
      KernelScope ks("split_gexp", s);
      k_gexp<<<static_cast<unsigned>(b1 - b0), 128, 0, s>>>(t->view(), g->view(), b0, MODE == 0 ? 1 : 5,
                                                            MODE == 0 ? 5 : 2, mats[0], mats[1], mats[2], mats[3],
                                                            mats[4], g->d_gexp);
    }
    Q4C_CUDA(cudaGetLastError());
    const int64_t i0 = g->rd_w0[wv], i1 = g->rd_w0[wv + 1];
    const int n_items = static_cast<int>(i1 - i0);
    if (n_items == 0) continue;
    const int grid = std::min(n_items, 2 * n_sm);
    {
      KernelScope ks(MODE == 0 ? "split_density" : "split_backward", s);
      k_split_rowdot<MODE><<<grid, kThreads, kSmemTotal, s>>>(
          t->view(), g->view(), g->d_rd_items + i0, n_items, g->d_counter + wv, g->d_scr_off, g->d_scratch,
          g->d_rowexp, g->d_gexp, mdf[0], mdf[1], mdf[2], mdf[3], mdf[4], out, g->d_status);
    }
    Q4C_CUDA(cudaGetLastError());
  }
  return Q4C_OK;
}

}  // namespace rowdot

q4c_status density_split(const q4c_tables* t, const q4c_grid* g, const double* P, double* n, cudaStream_t s) {
  const double* mats[5] = {P, nullptr, nullptr, nullptr, nullptr};
  return rowdot::run<0>(t, g, mats, n, s);
}

q4c_status backward_split(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* Gm, double* dLdv,
                          cudaStream_t s) {
  const double* mats[5] = {Gm->V, Gm->W0, Gm->SOx, Gm->SOy, Gm->SOz};
  // with every slot NULL the gradient is zero
  if (!Gm->V && !Gm->W0 && !Gm->SOx && !Gm->SOy && !Gm->SOz) {
    Q4C_CUDA(cudaMemsetAsync(dLdv, 0, sizeof(double) * g->n_pts, s));
    return Q4C_OK;
  }
  return rowdot::run<1>(t, g, mats, dLdv, s);
}

}  // namespace q4c
