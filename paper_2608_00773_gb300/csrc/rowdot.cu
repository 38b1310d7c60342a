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
// integer sums for K <= 512 terms, levels 3-5 are rounded 2^-24 below.  A
// batch of more than 512 functions splits K into segments of at most 512
// (32 chunks of 16), each a group of its own: its level sums are exact, and
// the epilogue adds its row-dot into the point's running sum like any other
// group's (the dot with R is linear in U).
//
// G' does not depend on the points, so a pre-pass slices every batch's G'
// once into BF16 digit tiles laid out exactly as the MMA reads them (per
// matrix, 64-function j-tile and 16-function i-chunk: six 2 KB tiles); the
// main kernel fetches one 12 KB block per K-step with a bulk copy.
#include <cuda.h>

#include "internal.h"
#include "tc.cuh"

namespace q4c {
namespace rowdot {
using namespace tc;

constexpr int kTile = 64;                      // points per tile (and functions per j-tile)
constexpr int kKc = 16;                        // functions i per chunk (one K = 16 MMA step)
constexpr int kTileBytes = kTile * kKc * 2;    // 2 KB
constexpr int kSBO = (kKc / 8) * 128;          // 256 B
constexpr int kBlockB = kSlices * kTileBytes;  // one step's G' digits, 12 KB
constexpr int kSlicers = 256;                  // warps 0-7 slice F
constexpr int kEpiWarp0 = 8;                   // warps 8-15 drain tensor memory (two groups of four)
constexpr int kEpiThreads = 256;
constexpr int kMmaWarp = 16;  // warp 16 owns tensor memory and issues the MMAs
constexpr int kProdWarp = 17;  // warp 17 issues the TMA loads of F
constexpr int kThreads = 18 * 32;
constexpr int kStageA = (kSlices + 1) * kTileBytes;  // [Z, A0..A5] of one K-step
constexpr int kHalf = kStageA + kBlockB;             // one K-step's operands, 26 KB
constexpr int kRawTile = kKc * kTile * 8;            // one box of F (16 functions x 64 points), 8 KB

// Shared-memory layout with KS K-steps of 16 functions per pipeline stage
// (the stage shape the tuner chooses): KS = 1 keeps four operand and four
// raw stages, KS = 2 three of each.
//   raw stage:     per K-step h the box of F (16 functions x 64 points of
//                  (hi, lo), 512-byte rows) at h * 8 KB and, on an item's
//                  first stage, the points' exponents;
//   operand stage: per K-step h the six F digit tiles after a zero tile and
//                  the j-tile's six G' digit tiles, at h * 26 KB.
template <int KS>
struct Layout {
  static constexpr int kStages = KS == 1 ? 4 : 3;
  static constexpr int kRaw = KS == 1 ? 4 : 3;
  static constexpr int kStage = KS * kHalf;
  static constexpr int kRawExp = KS * kRawTile;  // [64][4] per-point exponents
  static constexpr int kRawStage = kRawExp + 1024;
  static constexpr int kSmemRaw = 0;
  static constexpr int kSmemStages = kSmemRaw + kRaw * kRawStage;
  static constexpr int kSmemY = kSmemStages + kStages * kStage;  // [4][64] double partials per point
  static constexpr int kSmemBar = kSmemY + 4 * kTile * 8;
  // full, empty, accfull[2], accempty[2], drain, raw full/empty, G' copy full
  static constexpr int kNumBars = 3 * kStages + 5 + 2 * kRaw;
  static constexpr int kSmemTotal = kSmemBar + kNumBars * 8 + 16;
  static_assert(kSmemTotal <= 232448, "shared memory per CTA");
};
static_assert(Layout<1>::kRawStage == 9 * 1024 && Layout<1>::kStage == 26624, "the one-step layout");
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSetCols = 256;
constexpr int kMaxNb = 4096;
constexpr int kSegIc = 32;  // chunks of 16 functions per exact K segment (K <= 512)

struct Product {
  int qf, gm, qr;
  float factor;
};

// (F quantity, G matrix, R quantity, factor) of adjoint product k, packed one
// byte per product (qf | gm << 2 | qr << 5 | (factor == 2) << 7) so that the
// lookup stays in registers; matrices 2-4 enter through their antisymmetric
// parts, which the preparation forms once per call.  The density is product 0.
constexpr uint64_t kProducts = 0x00ull | (0x25ull << 8) | (0x46ull << 16) | (0x67ull << 24) | (0xEAull << 32) |
                               (0xAFull << 40) | (0xD1ull << 48);

__device__ __forceinline__ Product product_of(int k) {
  const unsigned c = static_cast<unsigned>(kProducts >> (8 * k)) & 0xFFu;
  return {static_cast<int>(c & 3u), static_cast<int>((c >> 2) & 7u), static_cast<int>((c >> 5) & 3u),
          (c >> 7) ? 2.0f : 1.0f};
}

// One CTA per pattern block q (A, B, T) (grid-stride): the FP32-pair copy
// of the block's values x (x = hi + lo within 2^-48 relative), and at
// cm_off[q] the largest |x| of each of its nf_B columns, then of each of its
// nf_A rows, rounded up to FP32.  With anti, x is the antisymmetric part
// (G - G^T)/2 in FP64, G^T read from the partner block (B, A, -T) through
// shared memory where both sides have at most 64 functions, else straight
// from memory (only that part enters the adjoint's cross-product terms).
__global__ void __launch_bounds__(128) k_prepare_blocks(DevBasis B, DevGrid G, const double* __restrict__ M,
                                                       int anti, int64_t n_blocks, const int* __restrict__ blk_row,
                                                       const int* __restrict__ blk_col,
                                                       const int64_t* __restrict__ blk_off,
                                                       const int* __restrict__ blk_T,
                                                       const int64_t* __restrict__ cm_off, float2* __restrict__ out,
                                                       float* __restrict__ cm) {
  __shared__ double sT[64 * 65];  // G^T of the block: sT[i * 65 + j] = partner (j, i)
  for (int64_t q = blockIdx.x; q < n_blocks; q += gridDim.x) {
    const int nfA = __ldg(B.sp_nfn + G.atom_sp[blk_row[q]]), nfB = __ldg(B.sp_nfn + G.atom_sp[blk_col[q]]);
    const double* X = M + blk_off[q];
    const int ne = nfA * nfB;
    const int qt = anti ? blk_T[q] : -1;
    const double* XT = qt >= 0 ? M + blk_off[qt] : nullptr;  // nfB rows x nfA columns
    const bool tile = XT && nfA <= 64 && nfB <= 64;
    if (tile) {
      __syncthreads();
      for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int r = e / nfA, c = e - r * nfA;
        sT[c * 65 + r] = XT[e];
      }
      __syncthreads();
    }
    auto val = [&](int i, int j) {
      const double x = X[static_cast<int64_t>(i) * nfB + j];
      if (!anti) return x;
      const double xt = tile ? sT[i * 65 + j] : XT ? XT[static_cast<int64_t>(j) * nfA + i] : 0.0;
      return 0.5 * (x - xt);
    };
    float2* o = out + blk_off[q];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int i = e / nfB, j = e - i * nfB;
      const double x = val(i, j);
      const float h = __double2float_rn(x);
      o[e] = make_float2(h, __double2float_rn(x - static_cast<double>(h)));
    }
    float* mx = cm + cm_off[q];
    for (int j = threadIdx.x; j < nfB; j += blockDim.x) {
      double m = 0.0;
      for (int i = 0; i < nfA; ++i) m = fmax(m, fabs(val(i, j)));
      mx[j] = __double2float_ru(m);
    }
    for (int i = threadIdx.x; i < nfA; i += blockDim.x) {
      double m = 0.0;
      for (int j = 0; j < nfB; ++j) m = fmax(m, fabs(val(i, j)));
      mx[nfB + i] = __double2float_ru(m);
    }
  }
}

__device__ __forceinline__ int fexp(float x) {  // |x| < 2^fexp(x) for x != 0
  return static_cast<int>((__float_as_uint(x) >> 23) & 0xFF) - 126;
}

// width of j-tile jt: its functions rounded up to 16 (the MMA's N
// granularity); its G' digit tiles hold that many rows
__device__ __forceinline__ int jt_width(int nb, int jt) { return (min(kTile, nb - jt * kTile) + 15) & ~15; }

// Pre-pass: one CTA per (batch, matrix).  Column exponents e_j (|G'_ij| <
// 2^e_j over the batch's i), then the six digits of every G'_ij written as
// the B operand tiles of the main kernel: block (jt, ic) (a 12 KB slot) =
// six tiles of jt_width rows (j) x 16 K (i), 32 bytes a row, in the
// no-swizzle K-major layout, back to back; padding rows and columns are 0.
// The column bound is the largest column maximum (k_prepare_blocks) of the
// blocks (a, c) of column j's centre c over the batch's active centres a,
// whose functions are exactly the batch's i.
__global__ void __launch_bounds__(256) k_gslice(DevGrid G, int64_t b0, const float2* M0,
                                                const float2* M1, const float2* M2, const float2* M3,
                                                const float2* M4, const float* C0, const float* C1,
                                                const float* C2, const float* C3, const float* C4,
                                                const int* __restrict__ pair_blk, const int64_t* __restrict__ cm_off,
                                                const int64_t* __restrict__ gsl_off, uint32_t* __restrict__ gsl) {
  __shared__ unsigned sMax[kMaxNb];  // bits of the bound of max_i |G'_ij| (non-negative floats order as integers)
  const int64_t b = b0 + blockIdx.x;
  const int m = blockIdx.y;
  const float2* M = m == 0 ? M0 : m == 1 ? M1 : m == 2 ? M2 : m == 3 ? M3 : M4;  // (no local array)
  if (M == nullptr) return;
  const float* CM = m == 0 ? C0 : m == 1 ? C1 : m == 2 ? C2 : m == 3 ? C3 : C4;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  const int* idx = G.bat_idx + G.bat_idx_ptr[b];
  const int n_jt = (nb + kTile - 1) / kTile, n_ic = (nb + kKc - 1) / kKc;
  uint32_t* out = gsl + (gsl_off[b] + static_cast<int64_t>(m) * n_jt * n_ic * kBlockB) / 4;
  // pass 1: column bounds, a thread per column over the batch's centres
  {
    const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
    const int* pb = pair_blk + G.bat_pair_ptr[b];
    const int* info = G.fn_info + G.bat_fn_ptr[b];
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      const int c = info[j] >> 16, jj = info[j] & 0xffff;
      float mx = 0.f;
      for (int a = 0; a < na; ++a) {
        const int q = pb[a * na + c];  // block (a, c): its column jj
        if (q >= 0) mx = fmaxf(mx, __ldg(CM + cm_off[q] + jj));
      }
      sMax[j] = __float_as_uint(mx);
    }
  }
  __syncthreads();
  // pass 2: the six digits of every element, in the B-operand tile layout;
  // a thread takes kU words (element pairs) at a time and issues all their
  // offset loads, then all their value loads, before slicing any
  constexpr int kU = 4;
  for (int jt = 0; jt < n_jt; ++jt) {
    const int tw = jt_width(nb, jt) * 8;  // words of one tile (one per element pair)
    const int words = n_ic * tw;
    for (int w0 = threadIdx.x; w0 < words; w0 += kU * blockDim.x) {
      int i_[kU], j_[kU], o0[kU], o1[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int w = w0 + u * blockDim.x;
        const int ic = w / tw, pos = w - ic * tw;
        // pos -> byte offset rg*SBO + kq*LBO + r8*16 + kp*4
        const int rg = pos >> 6, kq = (pos >> 5) & 1, r8 = (pos >> 2) & 7, kp = pos & 3;
        j_[u] = jt * kTile + rg * 8 + r8;
        i_[u] = ic * kKc + kq * 8 + kp * 2;
        const bool ok = w < words && j_[u] < nb;
        o0[u] = ok && i_[u] < nb ? __ldg(idx + i_[u] * nb + j_[u]) : -1;
        o1[u] = ok && i_[u] + 1 < nb ? __ldg(idx + (i_[u] + 1) * nb + j_[u]) : -1;
      }
      float2 x0[kU], x1[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        x0[u] = o0[u] < 0 ? make_float2(0.f, 0.f) : __ldg(M + o0[u]);
        x1[u] = o1[u] < 0 ? make_float2(0.f, 0.f) : __ldg(M + o1[u]);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int w = w0 + u * blockDim.x;
        if (w >= words) break;
        const int ic = w / tw, pos = w - ic * tw;
        float d0[kSlices], d1[kSlices];
        if (j_[u] < nb) {
          const unsigned mb = sMax[j_[u]];
          const float m0 = magic0(mb ? fexp(__uint_as_float(mb)) : -30000);
          slice6(x0[u].x, x0[u].y, m0, d0);
          slice6(x1[u].x, x1[u].y, m0, d1);
        } else {
#pragma unroll
          for (int s = 0; s < kSlices; ++s) d0[s] = d1[s] = 0.f;
        }
        uint32_t* o = out + static_cast<int64_t>(jt * n_ic + ic) * (kBlockB / 4) + pos;
#pragma unroll
        for (int s = 0; s < kSlices; ++s) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(d0[s], d1[s]);
          o[b_tile(s) * tw] = *reinterpret_cast<const uint32_t*>(&h2);  // [B0, B2, B4, B1, B3, B5]
        }
      }
    }
  }
}

// the work of one item (batch, 64-point tile): groups (j-tile, product, K
// segment) in order, each a K-loop over the segment's functions i in chunks
// of 16 (n_ic chunks in all, KS chunks per pipeline stage)
struct ItemInfo {
  int64_t b, bp0;
  int pt, np, ldp, nb, n_jt, n_ic, n_seg, n_stot;
  int64_t plane;
};

// pipeline stages of K segment seg
__device__ __forceinline__ int seg_stages(int n_ic, int seg, int ks) {
  return (min(kSegIc, n_ic - seg * kSegIc) + ks - 1) / ks;
}

__device__ __forceinline__ ItemInfo item_info(const DevGrid& G, int2 it) {
  ItemInfo I;
  I.b = it.x;
  I.pt = it.y;
  I.bp0 = G.pt_ptr[I.b];
  I.np = static_cast<int>(G.pt_ptr[I.b + 1] - I.bp0);
  I.ldp = (I.np + 7) & ~7;
  I.nb = static_cast<int>(G.bat_fn_ptr[I.b + 1] - G.bat_fn_ptr[I.b]);
  I.n_jt = (I.nb + kTile - 1) / kTile;
  I.n_ic = (I.nb + kKc - 1) / kKc;
  I.n_seg = (I.n_ic + kSegIc - 1) / kSegIc;
  I.plane = static_cast<int64_t>(I.nb) * I.ldp;
  return I;
}

template <int KS>
__device__ __forceinline__ int stages_per_product(const ItemInfo& I) {  // all segments of one (j-tile, product)
  return (I.n_seg - 1) * (kSegIc / KS) + seg_stages(I.n_ic, I.n_seg - 1, KS);
}

// position in an item's stage sequence (j-tile, product, K segment, stage
// within the segment), advanced without divisions
template <int KS>
struct StepIter {
  int st = 0, seg = 0, kk = 0, jt = 0;
  __device__ __forceinline__ void next(const ItemInfo& I, int n_prod) {
    if (++st == seg_stages(I.n_ic, seg, KS)) {
      st = 0;
      if (++seg == I.n_seg) {
        seg = 0;
        if (++kk == n_prod) {
          kk = 0;
          ++jt;
        }
      }
    }
  }
  // chunk of 16 functions read by K-step h of this stage
  __device__ __forceinline__ int chunk(int h) const { return seg * kSegIc + st * KS + h; }
};

// One work item = (batch, 64-point tile); its groups (j-tile, product) run
// in order, each a K-loop over the functions i.  Warp roles as in the
// integration kernel:
//   warp 17     (one thread) loads each step's box of F (64 points x 16
//               functions of the step's quantity) and, on an item's first
//               step, the points' exponents into the raw ring (raw_full
//               counts the bytes; raw_empty hands a stage back);
//   warps 0-7   per step: thread (point, 4 functions) reads its raw values,
//               waits empty[stage]; one thread starts the bulk copy of the
//               step's G' digits into the stage (its bytes complete
//               gfull[stage]);
//               all slice their F values, store the digits, arrive on
//               full[stage] and hand the raw stage back;
//   warp 16     (one thread) issues the six MMAs per step into the group's
//               accumulator set (groups alternate between two sets), commits
//               empty[stage] and, after the group's last step, accfull[set];
//   warps 8-15  read U's levels from tensor memory, dot each column with R
//               (a lane per thread, double-float), keep a running sum per lane
//               over the item's groups and write each point's result at the
//               end of the item.
// Every wait is bounded; a timeout sets the status bit and an abort flag.
template <int MODE, int KS>  // MODE 0: density, 1: adjoint; KS: K-steps per stage
__global__ void __launch_bounds__(kThreads, 1)
    k_split_rowdot(DevGrid G, const int2* __restrict__ items, int n_items, const CUtensorMap* __restrict__ maps,
                   const int64_t* __restrict__ scr_off, const double* __restrict__ scratch,
                   const int* __restrict__ rowexp, const int64_t* __restrict__ gsl_off,
                   const unsigned char* __restrict__ gsl, const unsigned char* __restrict__ gzero,
                   unsigned present, int weighted, double* __restrict__ out, unsigned* status) {
  using L = Layout<KS>;
  constexpr int kStages = L::kStages, kRaw = L::kRaw, kStage = L::kStage, kRawStage = L::kRawStage;
  constexpr int kRawExp = L::kRawExp, kSmemRaw = L::kSmemRaw, kSmemStages = L::kSmemStages;
  constexpr int kSmemY = L::kSmemY, kSmemBar = L::kSmemBar, kNumBars = L::kNumBars;
  extern __shared__ __align__(1024) unsigned char smem[];
  double* sY = reinterpret_cast<double*>(smem + kSmemY);    // [part][point]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSmemBar + kNumBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kSmemBar + kNumBars * 8 + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (smem_u32(smem) & 1023u) {  // TMA boxes and operand tiles need aligned stages
    if (tid == 0) atomicOr(status, 2u);
    return;
  }
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int st) { return bar0 + 8u * st; };
  auto empty_bar = [&](int st) { return bar0 + 8u * (kStages + st); };
  auto accfull_bar = [&](int set) { return bar0 + 8u * (2 * kStages + set); };
  auto accempty_bar = [&](int set) { return bar0 + 8u * (2 * kStages + 2 + set); };
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 4);
  auto rawfull_bar = [&](int rs) { return bar0 + 8u * (2 * kStages + 5 + rs); };
  auto rawempty_bar = [&](int rs) { return bar0 + 8u * (2 * kStages + 5 + kRaw + rs); };
  auto gfull_bar = [&](int st) { return bar0 + 8u * (2 * kStages + 5 + 2 * kRaw + st); };
  // the products whose matrix is present, in order, 3 bits each (registers only)
  unsigned plist = 0;
  int n_prod = 0;
  for (int k = 0; k < (MODE == 0 ? 1 : 7); ++k)
    if (present & (1u << product_of(k).gm)) plist |= static_cast<unsigned>(k) << (3 * n_prod++);
  auto prod_at = [&](int kk) { return product_of(static_cast<int>((plist >> (3 * kk)) & 7u)); };

  for (int i = tid; i < kStages * KS * kTileBytes / 16; i += kThreads) {  // tile Z of every K-step
    const int sh = i / (kTileBytes / 16), off = i - sh * (kTileBytes / 16);
    reinterpret_cast<uint4*>(smem + kSmemStages + sh * kHalf)[off] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();  // the zero tiles are read by the tensor cores (async proxy)
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
    for (int rs = 0; rs < kRaw; ++rs) {
      mbar_init(rawfull_bar(rs), 1);
      mbar_init(rawempty_bar(rs), kSlicers / 32);
    }
    for (int st = 0; st < kStages; ++st) mbar_init(gfull_bar(st), 1);
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
    // thread = (point p, functions 4q..4q+3 of the step); a warp takes 16
    // points and one pair of q.  Each half warp holds points 0-7 of one q and
    // points 8-15 of the other, so its 8-byte raw loads cover 128 distinct
    // bytes and its 8-byte digit stores land in distinct banks of the two
    // 8-row core matrices.
    const int sub = (lane >> 3) & 1;
    const int p = 16 * (warp >> 1) + 8 * (sub ^ (lane >> 4)) + (lane & 7), q = 2 * (warp & 1) + sub;
    const int dst_off = (p >> 3) * kSBO + (q >> 1) * kLBO + (p & 7) * 16 + (q & 1) * 8;
    bool ok = true;
    int g = 0;  // steps of this CTA
    for (int n = blockIdx.x; n < n_items; n += gridDim.x) {
      const ItemInfo I = item_info(G, items[n]);
      const bool live = I.pt * kTile + p < I.np;
      const unsigned char* gblk = gsl + gsl_off[I.b];
      const int n_steps = I.n_jt * n_prod * stages_per_product<KS>(I);
      float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;  // rounding constants of the point's four quantities
      StepIter<KS> it;
      for (int s = 0; s < n_steps; ++s, ++g) {
        const int rs = g % kRaw, st = g % kStages;
        if (!mbar_wait_abort(rawfull_bar(rs), (g / kRaw) & 1, s_abort, status, G.wait_ns)) {
          ok = false;
          break;
        }
        const unsigned char* raw = smem + kSmemRaw + rs * kRawStage;
        if (s == 0 && live) {
          const int4 e = *reinterpret_cast<const int4*>(raw + kRawExp + p * 16);
          m0 = magic0(e.x);
          m1 = magic0(e.y);
          m2 = magic0(e.z);
          m3 = magic0(e.w);
        }
        float2 x[KS][4];
#pragma unroll
        for (int h = 0; h < KS; ++h)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            x[h][k] = *reinterpret_cast<const float2*>(raw + h * kRawTile + (4 * q + k) * (kTile * 8) + p * 8);
        if (!mbar_wait_abort(empty_bar(st), ((g / kStages) & 1) ^ 1, s_abort, status, G.wait_ns)) {
          ok = false;
          break;
        }
        const Product P = prod_at(it.kk);
        unsigned char* sA = smem + kSmemStages + st * kStage;
        if (tid == 0) {  // this stage's G' digits: one block (up to 12 KB) per K-step
          const uint32_t bytes = kSlices * jt_width(I.nb, it.jt) * kRowBytes;  // the j-tile's six digit tiles
          arrive_expect_tx(gfull_bar(st), KS * bytes);
#pragma unroll
          for (int h = 0; h < KS; ++h) {
            // a K-step past the last chunk of functions (odd chunk counts,
            // KS = 2) multiplies zeros: its F box is zero-filled and its G'
            // block is the zero block
            const int ic = it.chunk(h);
            const unsigned char* src =
                ic < I.n_ic ? gblk + (static_cast<int64_t>(P.gm) * I.n_jt * I.n_ic +
                                      static_cast<int64_t>(it.jt) * I.n_ic + ic) * kBlockB
                            : gzero;
            bulk_copy(smem_u32(sA + h * kHalf + kStageA), src, bytes, gfull_bar(st));
          }
        }
        const float m = P.qf == 0 ? m0 : P.qf == 1 ? m1 : P.qf == 2 ? m2 : m3;
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          // functions (4q, 4q+1) and (4q+2, 4q+3) of K-step h as packed pairs
          float2 d01[kSlices], d23[kSlices];
          slice6x2(pk2(x[h][0].x, x[h][1].x), pk2(x[h][0].y, x[h][1].y), m, d01);
          slice6x2(pk2(x[h][2].x, x[h][3].x), pk2(x[h][2].y, x[h][3].y), m, d23);
#pragma unroll
          for (int t = 0; t < kSlices; ++t) {
            asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(
                             smem_u32(sA + h * kHalf + (1 + t) * kTileBytes + dst_off)),
                         "r"(bf16x2_exact(d01[t])), "r"(bf16x2_exact(d23[t]))
                         : "memory");
          }
        }
        fence_async_smem();
        mbar_arrive(full_bar(st));
        // Only now is the raw stage free: the digit stores above take their
        // data from the loaded values, so once they have issued the loads
        // have landed (freeing it right after issuing the loads let the next
        // TMA box overwrite values that were still on their way).
        __syncwarp();
        if (lane == 0) mbar_arrive(rawempty_bar(rs));
        it.next(I, n_prod);
      }
      // agree on stopping (a wait that gave up in one warp ends every role)
      if (bar_red_or(1, kSlicers, !ok || *s_abort)) break;
    }
    // no G' copy outlives the CTA: thread 0 issued one per completed step;
    // the last kStages of them may not have been consumed after an abort
    if (tid == 0)
      for (int h = max(0, g - kStages); h < g; ++h)
        (void)mbar_wait(gfull_bar(h % kStages), (h / kStages) & 1, status);
  } else if (warp == kProdWarp) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int n = blockIdx.x; n < n_items && ok; n += gridDim.x) {
        const ItemInfo I = item_info(G, items[n]);
        const CUtensorMap* map = maps + I.b;
        const int r0 = I.pt * kTile, rows = min(kTile, I.np - r0);
        const int n_steps = I.n_jt * n_prod * stages_per_product<KS>(I);
        StepIter<KS> it;
        for (int s = 0; s < n_steps; ++s, ++g) {
          const int rs = g % kRaw;
          if (!mbar_wait_abort(rawempty_bar(rs), ((g / kRaw) & 1) ^ 1, s_abort, status, G.wait_ns, 32)) {
            ok = false;
            break;
          }
          const uint32_t dst = smem_u32(smem + kSmemRaw + rs * kRawStage), fb = rawfull_bar(rs);
          arrive_expect_tx(fb, KS * kRawTile + (s == 0 ? rows * 16 : 0));
#pragma unroll
          for (int h = 0; h < KS; ++h)  // boxes past the last function read zeros
            tma_load_3d(dst + h * kRawTile, map, r0, it.chunk(h) * kKc, prod_at(it.kk).qf, fb);
          if (s == 0) bulk_copy(dst + kRawExp, rowexp + 4 * (I.bp0 + r0), rows * 16, fb);
          it.next(I, n_prod);
        }
      }
      // no copy outlives the CTA: the last kRaw issued steps have landed
      for (int h = max(0, g - kRaw); h < g; ++h) (void)mbar_wait(rawfull_bar(h % kRaw), (h / kRaw) & 1, status);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      int g = 0, k = 0;
      bool ok = true;
      for (int n = blockIdx.x; n < n_items && ok; n += gridDim.x) {
        const ItemInfo I = item_info(G, items[n]);
        int seg = 0, kk = 0, jt = 0;  // groups run (j-tile, product, segment) in order
        for (int grp = 0; grp < I.n_jt * n_prod * I.n_seg && ok; ++grp, ++k) {
          const int set = k & 1;
          if (!mbar_wait_abort(accempty_bar(set), ((k >> 1) & 1) ^ 1, s_abort, status, G.wait_ns, 64)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t t0 = tmem + set * kSetCols;
          const int nbj = jt_width(I.nb, jt);
          const int n_st = seg_stages(I.n_ic, seg, KS);
          if (++seg == I.n_seg) {
            seg = 0;
            if (++kk == n_prod) {
              kk = 0;
              ++jt;
            }
          }
          for (int c = 0; c < n_st; ++c, ++g) {
            const int st = g % kStages;
            if (!mbar_wait_abort(full_bar(st), (g / kStages) & 1, s_abort, status, G.wait_ns, 32) ||
                !mbar_wait_abort(gfull_bar(st), (g / kStages) & 1, s_abort, status, G.wait_ns, 32)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < KS; ++h) {
              const uint32_t a = smem_u32(smem + kSmemStages + st * kStage + h * kHalf), bb = a + kStageA;
              mma_levels(t0, a, bb, (c == 0 && h == 0) ? 0u : 1u, nbj);
            }
            mma_commit(empty_bar(st));
          }
          if (ok) mma_commit(accfull_bar(set));
        }
      }
      // every MMA issued by this thread has completed before tensor memory is freed
      mma_commit(drain_bar);
      (void)mbar_wait(drain_bar, 0, status);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    // Thread = one TMEM lane: lanes 0-63 hold levels 0, 2, 4 and lanes 64-127
    // levels 1, 3, 5 of the same 64 points.  The dot with R is linear in the
    // levels, so each lane keeps its own double-float partial sum; the two
    // halves and the two column groups meet once per item.
    const int eg = (warp - kEpiWarp0) >> 2;  // column group: 8-column chunks eg, eg + 2, ...
    const int quarter = warp & 3;            // TMEM lanes 32 quarter .. +31
    const int r = (quarter & 1) * 32 + lane, lvl = quarter >> 1;
    const uint32_t lane_base = static_cast<uint32_t>(quarter * 32) << 16;
    int k = 0;
    bool ok = true;
    for (int n = blockIdx.x; n < n_items && ok; n += gridDim.x) {
      const ItemInfo I = item_info(G, items[n]);
      const float2* base = reinterpret_cast<const float2*>(scratch) + scr_off[I.b];
      const int p = I.pt * kTile + r;
      const bool live = p < I.np;
      df y = {0.f, 0.f};  // running sum over the item's groups
      int seg = 0, kk = 0, jt = 0;
      for (int grp = 0; grp < I.n_jt * n_prod * I.n_seg; ++grp, ++k) {
        const int set = k & 1;
        const int j0 = jt * kTile;
        const Product P = prod_at(kk);
        const int N = jt_width(I.nb, jt);  // accumulator blocks are N columns wide
        const float2* Rrow = base + P.qr * I.plane + p;
        // R of this thread's point, 8 columns per chunk; the first chunk's
        // values load while the MMAs finish, later ones one chunk ahead
        auto load_R = [&](int c0, float2* R) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int j = j0 + c0 + i;
            R[i] = (live && j < I.nb) ? __ldg(Rrow + static_cast<int64_t>(j) * I.ldp) : make_float2(0.f, 0.f);
          }
        };
        float2 Rc[8], Rn[8];
        if (eg * 8 < N) load_R(eg * 8, Rc);
        ok = mbar_wait_abort(accfull_bar(set), (k >> 1) & 1, s_abort, status, G.wait_ns, 256);
        if (bar_red_or(2, kEpiThreads, !ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // this group's sum yh + yl: per column u = v0 + v1 + v2 (top lanes
        // L0 + L2 + L4 with L0, L2 exact; bottom lanes L1 + L3 + L5) as the
        // exact two-sum of v0, v1 with v2 (2^-16 and further below) folded
        // into its error; the product with R = (rh, rl) keeps its FMA error
        // term unnormalised, and the sum adds each product by a two-sum whose
        // error joins yl (all terms about 2^-24 below yh and beyond)
        float yh = 0.f, yl = 0.f;
        for (int c0 = eg * 8; c0 < N; c0 += 16) {
          if (c0 + 16 < N) load_R(c0 + 16, Rn);
          float v0[8], v1[8], v2[8];
          const uint32_t ta = tmem + lane_base + set * kSetCols + c0;
          tmem_ld8x3(ta, ta + N, ta + 2 * N, v0, v1, v2);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const df u = two_sum(v0[i], v1[i]);
            const float ul = __fadd_rn(u.lo, v2[i]);
            const float rh = Rc[i].x, rl = Rc[i].y;
            const float ph = __fmul_rn(rh, u.hi);
            float pl = __fmaf_rn(rh, u.hi, -ph);
            pl = __fmaf_rn(rh, ul, pl);
            pl = __fmaf_rn(rl, u.hi, pl);
            const df a = two_sum(yh, ph);
            yh = a.hi;
            yl = __fadd_rn(yl, __fadd_rn(a.lo, pl));
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) Rc[i] = Rn[i];
        }
        tc_fence_before();
        mbar_arrive(accempty_bar(set));
        y = df_add(y, df{P.factor * yh, P.factor * yl});  // factor 1 or 2: exact
        if (++seg == I.n_seg) {
          seg = 0;
          if (++kk == n_prod) {
            kk = 0;
            ++jt;
          }
        }
      }
      if (!ok) break;
      // the four partial sums of each point (two level halves x two column groups)
      sY[(eg * 2 + lvl) * kTile + r] = static_cast<double>(y.hi) + static_cast<double>(y.lo);
      bar_sync(2, kEpiThreads);
      if (eg == 0 && lvl == 0 && live) {
        const double val = (sY[r] + sY[kTile + r]) + (sY[2 * kTile + r] + sY[3 * kTile + r]);
        const int64_t gp = I.bp0 + p;
        out[gp] = weighted ? G.w[gp] * val : val;
      }
      bar_sync(2, kEpiThreads);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// FP32-pair copies of the present matrices into slots [slot0, slot0 + 5) of
// the grid's buffer (of the antisymmetric parts of matrices 2-4, the SO
// slots), with their per-block column and row maxima; returns the mask of
// present matrices
q4c_status prepare(const q4c_grid* g, const double* const mats[5], int slot0, const float2* mdf[5],
                   unsigned* present, cudaStream_t s) {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  *present = 0;
  KernelScope ks("split_gslice", s);
  for (int m = 0; m < 5; ++m) {
    mdf[m] = nullptr;
    if (!mats[m] || g->nnz == 0) continue;
    float2* dst = g->d_gdf + (slot0 + m) * g->nnz;
    const unsigned nblk = static_cast<unsigned>(std::min<int64_t>(g->n_blocks, 64 * n_sm));
    k_prepare_blocks<<<nblk, 128, 0, s>>>(g->tables->view(), g->view(), mats[m], m >= 2 ? 1 : 0, g->n_blocks,
                                          g->d_blk_row, g->d_blk_col, g->d_blk_off, g->d_blk_T, g->d_cm_off, dst,
                                          g->d_cm + (slot0 + m) * g->cm_total);
    mdf[m] = dst;
    *present |= 1u << m;
  }
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

// one wave [b0, b1) of the density (MODE 0) or adjoint (MODE 1): G' digit
// blocks and the row-dot kernel with KS K-steps per stage; the wave's offset
// tables and basis tiles (with per-point exponents) must already be in place
template <int MODE>
q4c_status gslice_wave(const q4c_grid* g, int wv, const float2* const mdf[5], cudaStream_t s) {
  const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
  if (b1 <= b0) return Q4C_OK;
  // each matrix's block maxima sit in the slot of its FP32-pair copy
  const float* cmp[5];
  for (int m = 0; m < 5; ++m)
    cmp[m] = mdf[m] ? g->d_cm + ((mdf[m] - g->d_gdf) / std::max<int64_t>(g->nnz, 1)) * g->cm_total : nullptr;
  KernelScope ks("split_gslice", s);
  k_gslice<<<dim3(static_cast<unsigned>(b1 - b0), MODE == 0 ? 1 : 5), 256, 0, s>>>(
      g->view(), b0, mdf[0], mdf[1], mdf[2], mdf[3], mdf[4], cmp[0], cmp[1], cmp[2], cmp[3],
      cmp[4], g->d_pair_blk, g->d_cm_off, g->d_gsl_off, reinterpret_cast<uint32_t*>(g->d_gsl));
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

// the row-dot kernel of one wave (its G' blocks in place)
template <int MODE, int KS>
q4c_status rowdot_kernel(const q4c_grid* g, int wv, unsigned present, bool weighted, double* out, cudaStream_t s,
                         const char* name) {
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  Q4C_CUDA(cudaFuncSetAttribute(k_split_rowdot<MODE, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Layout<KS>::kSmemTotal));
  const int64_t i0 = g->rd_w0[wv], i1 = g->rd_w0[wv + 1];
  const int n_items = static_cast<int>(i1 - i0);
  if (n_items == 0) return Q4C_OK;
  const int grid = std::min(n_items, n_sm);
  {
    KernelScope ks(name, s);
    k_split_rowdot<MODE, KS><<<grid, kThreads, Layout<KS>::kSmemTotal, s>>>(
        g->view(), g->d_rd_items + i0, n_items, reinterpret_cast<const CUtensorMap*>(g->d_tmaps) + g->n_batches,
        g->d_scr_off, g->d_scratch, g->d_rowexp, g->d_gsl_off, reinterpret_cast<const unsigned char*>(g->d_gsl),
        g->d_gzero, present, weighted ? 1 : 0, out, g->d_status);
  }
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

template <int MODE>
q4c_status kernel_ks(const q4c_grid* g, int wv, unsigned present, bool weighted, double* out, cudaStream_t s, int ks,
                     const char* name) {
  if (ks == 2) return rowdot_kernel<MODE, 2>(g, wv, present, weighted, out, s, name);
  return rowdot_kernel<MODE, 1>(g, wv, present, weighted, out, s, name);
}

template <int MODE>
q4c_status wave(const q4c_grid* g, int wv, const float2* const mdf[5], unsigned present, bool weighted,
                double* out, cudaStream_t s) {
  if (g->wave_b0[wv + 1] <= g->wave_b0[wv]) return Q4C_OK;
  if (q4c_status st = gslice_wave<MODE>(g, wv, mdf, s)) return st;
  return kernel_ks<MODE>(g, wv, present, weighted, out, s, g->rd_ks, MODE == 0 ? "split_density" : "split_backward");
}

template <int MODE>
q4c_status run(const q4c_tables* t, const q4c_grid* g, const double* const mats[5], double* out, cudaStream_t s,
               bool weighted) {
  if (g->max_nb > kMaxNb) {
    set_error("the split density/adjoint need at most 4096 active functions per batch");
    return Q4C_EUNSUPPORTED;
  }
  const float2* mdf[5];
  unsigned present = 0;
  if (q4c_status st = prepare(g, mats, 0, mdf, &present, s)) return st;
  const int n_waves = static_cast<int>(g->wave_b0.size()) - 1;
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_fill_idx(t, g, b0, b1, s)) return st;
    if (q4c_status st = launch_basis_df(t, g, b0, b1, nullptr, nullptr, g->d_rowexp, MODE == 0 ? 1 : 4, s)) return st;
    if (q4c_status st = wave<MODE>(g, wv, mdf, present, weighted, out, s)) return st;
  }
  return Q4C_OK;
}

}  // namespace rowdot

q4c_status rowdot_prepare(const q4c_grid* g, const double* const mats[5], int slot0, const float2* mdf[5],
                          unsigned* present, cudaStream_t s) {
  return rowdot::prepare(g, mats, slot0, mdf, present, s);
}

q4c_status rowdot_wave(const q4c_grid* g, int wv, int mode, const float2* const mdf[5], unsigned present,
                       bool weighted, double* out, cudaStream_t s) {
  return mode == 0 ? rowdot::wave<0>(g, wv, mdf, present, weighted, out, s)
                   : rowdot::wave<1>(g, wv, mdf, present, weighted, out, s);
}

// the tuner's part for the row-dot kernel: the adjoint kernel of wave 0 with
// both stage shapes (G' from zero matrices, sliced once: the kernel's work
// does not depend on the values), one untimed launch each, then three rounds
// alternating the shapes, each launch between CUDA events; the faster shape
// is kept for the grid.  The wave's offset tables and basis tiles with
// per-point exponents must be in place.
q4c_status autotune_rowdot(q4c_grid* g, double* out, cudaStream_t s) {
  g->rd_tune_ms[0] = g->rd_tune_ms[1] = -1.0;
  if (g->wave_b0.size() < 2 || g->max_nb > rowdot::kMaxNb || g->nnz == 0) return Q4C_OK;
  if (g->wave_b0[1] <= g->wave_b0[0]) return Q4C_OK;
  const float2* mdf[5];
  for (int m = 0; m < 5; ++m) mdf[m] = g->d_gdf + (5 + m) * g->nnz;
  Q4C_CUDA(cudaMemsetAsync(g->d_gdf + 5 * g->nnz, 0, sizeof(float2) * 5 * g->nnz, s));
  Q4C_CUDA(cudaMemsetAsync(g->d_cm + 5 * g->cm_total, 0, sizeof(float) * 5 * g->cm_total, s));
  if (q4c_status st = rowdot::gslice_wave<1>(g, 0, mdf, s)) return st;
  cudaEvent_t ev[2][3][2] = {};
  q4c_status status = Q4C_OK;
  for (int k = 0; k < 2; ++k)
    for (int r = 0; r < 3; ++r)
      for (int e = 0; e < 2; ++e)
        if (cudaEventCreate(&ev[k][r][e]) != cudaSuccess) status = Q4C_ECUDA;
  for (int ks = 1; ks <= 2 && status == Q4C_OK; ++ks)
    status = rowdot::kernel_ks<1>(g, 0, 31u, true, out, s, ks, "split_tune");
  for (int r = 0; r < 3 && status == Q4C_OK; ++r)
    for (int ks = 1; ks <= 2 && status == Q4C_OK; ++ks) {
      cudaEventRecord(ev[ks - 1][r][0], s);
      status = rowdot::kernel_ks<1>(g, 0, 31u, true, out, s, ks, "split_tune");
      cudaEventRecord(ev[ks - 1][r][1], s);
    }
  if (status == Q4C_OK && cudaStreamSynchronize(s) != cudaSuccess) status = Q4C_ECUDA;
  for (int k = 0; k < 2 && status == Q4C_OK; ++k) {
    double sum = 0.0;
    for (int r = 0; r < 3; ++r) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k][r][0], ev[k][r][1]) != cudaSuccess) status = Q4C_ECUDA;
      sum += ms;
    }
    g->rd_tune_ms[k] = sum / 3.0;
  }
  if (status == Q4C_OK) g->rd_ks = g->rd_tune_ms[1] < g->rd_tune_ms[0] ? 2 : 1;
  else set_error("q4c_autotune: timing of the density/adjoint kernel failed");
  for (int k = 0; k < 2; ++k)
    for (int r = 0; r < 3; ++r)
      for (int e = 0; e < 2; ++e)
        if (ev[k][r][e]) cudaEventDestroy(ev[k][r][e]);
  return status;
}

q4c_status density_split(const q4c_tables* t, const q4c_grid* g, const double* P, double* n, cudaStream_t s) {
  const double* mats[5] = {P, nullptr, nullptr, nullptr, nullptr};
  return rowdot::run<0>(t, g, mats, n, s, false);
}

q4c_status backward_split(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* Gm, double* dLdv,
                          cudaStream_t s, bool weighted) {
  const double* mats[5] = {Gm->V, Gm->W0, Gm->SOx, Gm->SOy, Gm->SOz};
  // with every slot NULL the gradient is zero
  if (!Gm->V && !Gm->W0 && !Gm->SOx && !Gm->SOy && !Gm->SOz) {
    Q4C_CUDA(cudaMemsetAsync(dLdv, 0, sizeof(double) * g->n_pts, s));
    return Q4C_OK;
  }
  return rowdot::run<1>(t, g, mats, dLdv, s, weighted);
}

}  // namespace q4c
