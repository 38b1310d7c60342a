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
// Outputs per (batch, tile pair ti <= tj; tiles of 64 functions, the B tile
// tj only as wide as its functions rounded up to 16): V = (D Phi)^T Phi,
// W0 = sum_q (D Q)^T Q (three products into one accumulator, sliced against
// a common exponent per function so that the exact levels keep one unit),
// and SO: on a diagonal pair A_yz = (D Y)^T Z, A_zx = (D Z)^T X,
// A_xy = (D X)^T Y with SO_x = A_yz - A_yz^T etc. applied while scattering,
// on an off-diagonal pair SO_x = (D Y)^T Z - (D Z)^T Y etc. directly (two
// K-concatenated products); and, as its own launch, the per-column operator
// of Eq. 19, F = (w Phi)^T Psi with Psi_pj = (v_p + eps_j - V_j) phi_j
// (output 5, every tile pair, every element into its own block).  One warp-specialised CTA per SM (slicers, one MMA
// thread, epilogue warps; 512 TMEM columns) loops over the work items; every
// mbarrier wait is bounded and sets a status bit instead of hanging.
#include <cuda.h>

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
constexpr int kProdWarp = 17;                // warp 17 issues the TMA loads of the raw operands
constexpr int kThreads = 18 * 32;
constexpr int kEpiPitch = 17;                // floats per staged TMEM lane (16 columns + pad)
constexpr int kEpiStage = 3 * 128 * kEpiPitch * 4;  // one group's staging, 26 KB
constexpr int kStageA = (kSlices + 1) * kTileBytes;  // [Z, A0..A5] of one K-step
constexpr int kStageB = kSlices * kTileBytes;        // [B0..B5] of one K-step
constexpr int kHalf = kStageA + kStageB;             // one K-step's operands, 26 KB
constexpr int kRawTile = kTile * kKc * 8;            // one 64 x 16 box of (hi, lo), 8 KB
constexpr uint32_t kTmemCols = 512;  // two accumulator sets of three blocks of up to 64 columns
constexpr uint32_t kSetCols = 256;

// Shared-memory layout of the kernel with KS K-steps of 16 points per
// pipeline stage (the stage shape the tuner chooses per batch-size bucket):
// KS = 1 keeps four operand and four raw stages, KS = 2 two of each (twice
// the points per handshake, the same points in flight).
//   raw stage:     per K-step h the A and B boxes (64 functions x 16 points
//                  of (hi, lo), 128-byte rows, swizzled) at h * 16 KB, the
//                  stage's D values (KS x 16 x 8 B) and, on an item's first
//                  stage, the item's 128 rounding constants;
//   operand stage: per K-step h the six A digit tiles after a zero tile and
//                  the six B digit tiles, at h * 26 KB.
template <int KS>
struct Layout {
  static constexpr int kStages = KS == 1 ? 4 : 2;  // ring depth of sliced operands
  static constexpr int kRaw = KS == 1 ? 4 : 2;     // ring depth of raw boxes
  static constexpr int kStage = KS * kHalf;
  static constexpr int kRawD = KS * 2 * kRawTile;              // offset of D
  static constexpr int kRawMag = kRawD + KS * kKc * 8;         // offset of the rounding constants
  static constexpr int kRawStage = ((kRawMag + 128 * 4 + 1023) / 1024) * 1024;  // 1024-aligned (swizzle atoms)
  static constexpr int kSmemRaw = 0;
  static constexpr int kSmemStages = kSmemRaw + kRaw * kRawStage;
  static constexpr int kSmemEpi = kSmemStages + kStages * kStage;  // epilogue staging, 2 x 26 KB
  static constexpr int kSmemBar = kSmemEpi + 2 * kEpiStage;
  // full, empty, accfull[2], accempty[2], drain, raw full/empty
  static constexpr int kNumBars = 2 * kStages + 5 + 2 * kRaw;
  static constexpr int kSmemTotal = kSmemBar + kNumBars * 8 + 16;
  static_assert(kSmemTotal <= 232448, "shared memory per CTA");
};
static_assert(Layout<1>::kRawStage == 17 * 1024 && Layout<1>::kStage == 26624, "the one-step layout");

// ------------------------------------------------------------ kernel
// The products of one item, K-concatenated into one accumulator: n of them,
// the A-side (D-scaled) and B-side quantities of product pr in bits
// 2pr..2pr+1 of qa and qb (0 Phi, 1 X, 2 Y, 3 Z); a two-product item
// subtracts its second product (its D is negated).
struct Products {
  int n;
  unsigned qa, qb;
  __device__ __forceinline__ int a(int pr) const { return static_cast<int>((qa >> (2 * pr)) & 3u); }
  __device__ __forceinline__ int b(int pr) const { return static_cast<int>((qb >> (2 * pr)) & 3u); }
};

// Items cover the tile pairs ti <= tj of a batch.  SO_k is the antisymmetric
// part of A_k (A_yz = (D Y)^T Z, A_zx = (D Z)^T X, A_xy = (D X)^T Y): on a
// diagonal tile pair the item computes A_k and the epilogue takes
// A_k(i, j) - A_k(j, i); on an off-diagonal pair (ti < tj) it computes
// SO_k itself, e.g. SO_x(ti, tj) = (D Y_ti)^T Z_tj - (D Z_ti)^T Y_tj, since
// A_yz(j, i) = (D Z_i)^T Y_j: every item then keeps its full 64-function
// tile on the M side and the narrower tile tj on the N side.
__device__ __forceinline__ Products products_of(int o, bool offdiag) {
  switch (o) {
    case 0: return {1, 0u, 0u};                                 // V
    case 1: return {3, 0x39u, 0x39u};                           // W0: (X, X), (Y, Y), (Z, Z)
    case 2: return offdiag ? Products{2, 0xEu, 0xBu} : Products{1, 2u, 3u};  // SO_x: (Y, Z) - (Z, Y)
    case 3: return offdiag ? Products{2, 0x7u, 0xDu} : Products{1, 3u, 1u};  // SO_y: (Z, X) - (X, Z)
    case 4: return offdiag ? Products{2, 0x9u, 0x6u} : Products{1, 1u, 2u};  // SO_z: (X, Y) - (Y, X)
    default: return {1, 0u, 1u};                                // per-column operator: (w Phi)^T Psi
  }
}

__device__ __forceinline__ Products item_products(const int4& item) {
  return products_of(item.y, item.y >= 2 && item.y <= 4 && item.z != item.w);
}

// B-tile width of an item: the functions of tile tj rounded up to 16 (the
// MMA's N granularity)
__device__ __forceinline__ int item_nb(int nb, int tj) { return (min(kTile, nb - tj * kTile) + 15) & ~15; }

// Rounding constants of one item's rows: 0..63 the A side (column exponents
// of the D-scaled quantity), 64..127 the B side.  An item with several
// K-concatenated products (W0, off-diagonal SO) slices them against one
// exponent per function (the maximum over its products), so that they share
// units.
__global__ void k_item_prep(DevGrid G, const int4* __restrict__ items, const int* __restrict__ colexp,
                            float* __restrict__ mag) {
  const int n = blockIdx.x;
  const int4 item = items[n];
  const int64_t b = item.x;
  const int t = threadIdx.x, side = t >> 6, r = t & 63;
  const int64_t fn0 = G.bat_fn_ptr[b];
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - fn0);
  const int* cexp = colexp + 8 * fn0;
  const int f = (side ? item.w : item.z) * kTile + r;
  int e = -30000;
  if (f < nb) {
    const int base = side ? 4 : 0;
    const Products P = item_products(item);
    for (int pr = 0; pr < P.n; ++pr) e = max(e, cexp[(base + (side ? P.b(pr) : P.a(pr))) * nb + f]);
  }
  mag[static_cast<int64_t>(n) * 128 + t] = magic0(e);
}

__device__ __forceinline__ float4 lds128(const unsigned char* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ void sts64(unsigned char* p, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(smem_u32(p)), "r"(a), "r"(b) : "memory");
}


// One work item = (batch, output, tile pair).  Its K dimension is a stream
// of steps of 16 points; W0 and the off-diagonal SO items interleave their
// products step by step (a K-concatenation into one accumulator, common
// exponents; the subtracted SO product slices -D).
//
// Warp roles (one CTA per SM, items strided over the CTAs):
//   warp 17     (one thread) loads step g's raw operands into raw stage
//               g mod 4 once the slicers have read it (raw_empty): two TMA
//               boxes (A and B rows of the step's quantities, zeros past n_p
//               and n_b), the step's 16 D values and, on an item's first
//               step, the item's rounding constants; one mbarrier (raw_full)
//               counts the bytes;
//   warps 0-7   thread (row r, points 4q..4q+3) reads its raw values, forms
//               the D-scaled A values in double-float, slices both sides
//               (the B side only on the item's B rows) into six BF16 digits
//               and stores them (8 bytes per slice and side) into operand
//               stage g mod 4 once the MMAs that last read it have completed
//               (empty[stage], a tcgen05.commit), arrives on full[stage] and
//               frees the raw stage;
//   warp 16     (one thread) waits full[stage], issues the six MMAs into the
//               item's accumulator set (items alternate between two sets of
//               up to 192 TMEM columns), commits empty[stage], and after an item's
//               last step commits accfull[set];
//   warps 8-15  wait accfull[set], read the six levels, combine and scatter
//               (two groups of four warps take alternate 16-column chunks;
//               the scatter offsets come from the batch's dense offset
//               table), then arrive on accempty[set] so the set can take
//               item k + 2.
// Every wait is bounded; a role that times out sets the status bit and an
// abort flag that ends the other roles' waits, and the MMA thread drains its
// outstanding MMAs (bounded) before tensor memory is freed.
template <int KS>
__global__ void __launch_bounds__(kThreads, 1)
    k_split_products(DevGrid G, const int4* __restrict__ items, int n_items,
                     const CUtensorMap* __restrict__ maps, const float2* __restrict__ dpad,
                     const float* __restrict__ mag, double* V, double* W0, double* SOx, double* SOy, double* SOz,
                     unsigned* status) {
  using L = Layout<KS>;
  constexpr int kStages = L::kStages, kRaw = L::kRaw, kStage = L::kStage, kRawStage = L::kRawStage;
  constexpr int kRawD = L::kRawD, kRawMag = L::kRawMag, kSmemRaw = L::kSmemRaw, kSmemStages = L::kSmemStages;
  constexpr int kSmemEpi = L::kSmemEpi, kSmemBar = L::kSmemBar, kNumBars = L::kNumBars;
  // stages of KS x 16 points per item: the batch's points, times the products
  // the item K-concatenates
  auto item_stages = [&](const int4& it) {
    const int np = static_cast<int>(G.pt_ptr[it.x + 1] - G.pt_ptr[it.x]);
    return (np + KS * kKc - 1) / (KS * kKc) * item_products(it).n;
  };
  extern __shared__ __align__(1024) unsigned char smem[];
  float* stage = reinterpret_cast<float*>(smem + kSmemEpi);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSmemBar + kNumBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + kSmemBar + kNumBars * 8 + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (smem_u32(smem) & 1023u) {  // the swizzled TMA boxes need 1024-byte aligned stages
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

  // zero tile Z at the head of each K-step's A tiles (never overwritten)
  for (int i = tid; i < kStages * KS * kTileBytes / 16; i += kThreads) {
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
    // row, points 4q..4q+3 of the step.  A quarter warp takes one q on rows
    // 0-7 (its 16-byte raw chunks 2q ^ row are then eight distinct banks
    // groups) and a half warp one K-half on rows 0-7 (its 8-byte digit slots
    // fill one 128-byte core-matrix pair without a bank conflict).
    const int r = warp * 8 + (lane & 7), q = lane >> 3;
    // byte offsets: swizzled 16-byte chunks 2q, 2q+1 of row r in a raw box;
    // the 8-byte slot of (r, 4q) in a K-major core-matrix operand tile
    const int rc0 = r * 128 + (((2 * q) ^ (r & 7)) << 4), rc1 = r * 128 + (((2 * q + 1) ^ (r & 7)) << 4);
    const int dst_off = (r >> 3) * kSBO + (q >> 1) * kLBO + (r & 7) * 16 + (q & 1) * 8;
    int g = 0;  // stages sliced by this CTA
    for (int n = blockIdx.x; n < n_items; n += gridDim.x) {
      const int4 item = items[n];
      const int n_steps = item_stages(item);
      const int nbB = item_nb(static_cast<int>(G.bat_fn_ptr[item.x + 1] - G.bat_fn_ptr[item.x]), item.w);
      const int n_prod = item_products(item).n;
      const bool b_row = r < nbB;  // this warp's rows of the B tile exist (nbB is a multiple of 16)
      float mA = 0.f, mB = 0.f;
      bool ok = true;
      for (int s = 0, pr = 0; s < n_steps; ++s, ++g, pr = (pr + 1 == n_prod) ? 0 : pr + 1) {
        const int rs = g % kRaw, st = g % kStages;
        if (!mbar_wait_abort(rawfull_bar(rs), (g / kRaw) & 1, s_abort, status, G.wait_ns)) {
          ok = false;
          break;
        }
        const unsigned char* raw = smem + kSmemRaw + rs * kRawStage;
        if (s == 0) {
          mA = reinterpret_cast<const float*>(raw + kRawMag)[r];
          mB = reinterpret_cast<const float*>(raw + kRawMag)[64 + r];
        }
        float4 a01[KS], a23[KS], b01[KS], b23[KS], d01[KS], d23[KS];
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          const unsigned char* box = raw + h * 2 * kRawTile;
          a01[h] = lds128(box + rc0);
          a23[h] = lds128(box + rc1);
          b01[h] = b23[h] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (b_row) {
            b01[h] = lds128(box + kRawTile + rc0);
            b23[h] = lds128(box + kRawTile + rc1);
          }
          d01[h] = lds128(raw + kRawD + h * kKc * 8 + q * 32);
          d23[h] = lds128(raw + kRawD + h * kKc * 8 + q * 32 + 16);
          if (pr == 1 && n_prod == 2) {  // the subtracted product of an off-diagonal SO item: -D (exact)
            d01[h] = make_float4(-d01[h].x, -d01[h].y, -d01[h].z, -d01[h].w);
            d23[h] = make_float4(-d23[h].x, -d23[h].y, -d23[h].z, -d23[h].w);
          }
        }
        if (!mbar_wait_abort(empty_bar(st), ((g / kStages) & 1) ^ 1, s_abort, status, G.wait_ns)) {
          ok = false;
          break;
        }
#pragma unroll
        for (int h = 0; h < KS; ++h) {
          unsigned char* sA = smem + kSmemStages + st * kStage + h * kHalf;
          unsigned char* sB = sA + kStageA;
          // points (4q, 4q+1) and (4q+2, 4q+3) of K-step h as packed pairs
          {  // A side: D-scaled values in double-float
            float2 xh01, xl01, xh23, xl23;
            df_mul2(pk2(a01[h].x, a01[h].z), pk2(a01[h].y, a01[h].w), pk2(d01[h].x, d01[h].z),
                    pk2(d01[h].y, d01[h].w), pk2(-d01[h].x, -d01[h].z), xh01, xl01);
            df_mul2(pk2(a23[h].x, a23[h].z), pk2(a23[h].y, a23[h].w), pk2(d23[h].x, d23[h].z),
                    pk2(d23[h].y, d23[h].w), pk2(-d23[h].x, -d23[h].z), xh23, xl23);
            float2 e01[kSlices], e23[kSlices];
            slice6x2(xh01, xl01, mA, e01);
            slice6x2(xh23, xl23, mA, e23);
#pragma unroll
            for (int t = 0; t < kSlices; ++t)  // A: [Z, A0..A5]
              sts64(sA + (1 + t) * kTileBytes + dst_off, bf16x2_exact(e01[t]), bf16x2_exact(e23[t]));
          }
          if (b_row) {  // B side: tiles of nbB rows
            float2 e01[kSlices], e23[kSlices];
            slice6x2(pk2(b01[h].x, b01[h].z), pk2(b01[h].y, b01[h].w), mB, e01);
            slice6x2(pk2(b23[h].x, b23[h].z), pk2(b23[h].y, b23[h].w), mB, e23);
#pragma unroll
            for (int t = 0; t < kSlices; ++t)  // B: [B0, B2, B4, B1, B3, B5]
              sts64(sB + b_tile(t) * nbB * kRowBytes + dst_off, bf16x2_exact(e01[t]), bf16x2_exact(e23[t]));
          }
        }
        fence_async_smem();
        mbar_arrive(full_bar(st));
        // Only now is the raw stage free: the digit stores above take their
        // data from the loaded values, so once they have issued the loads
        // have landed (the next TMA box may not overwrite values in flight).
        __syncwarp();
        if (lane == 0) mbar_arrive(rawempty_bar(rs));
      }
      // agree on stopping (a wait that gave up in one warp ends every role)
      if (bar_red_or(1, kSlicers, !ok || *s_abort)) break;
    }
  } else if (warp == kProdWarp) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      int g = 0;
      for (int n = blockIdx.x; n < n_items; n += gridDim.x) {
        const int4 item = items[n];
        const int n_steps = item_stages(item);
        const Products P = item_products(item);
        const CUtensorMap* map = maps + item.x;
        const float2* drow = dpad + static_cast<int64_t>(item.x) * kDPitch;
        const int i0 = item.z * kTile, j0 = item.w * kTile;
        bool ok = true;
        for (int s = 0; s < n_steps; ++s, ++g) {
          const int rs = g % kRaw;
          if (!mbar_wait_abort(rawempty_bar(rs), ((g / kRaw) & 1) ^ 1, s_abort, status, G.wait_ns, 32)) {
            ok = false;
            break;
          }
          const int c = P.n == 1 ? s : s / P.n, pr = s - c * P.n;  // c: this stage's chunk of KS x 16 points
          const uint32_t dst = smem_u32(smem + kSmemRaw + rs * kRawStage);
          const uint32_t fb = rawfull_bar(rs);
          arrive_expect_tx(fb, KS * (2 * kRawTile + kKc * 8) + (s == 0 ? 128 * 4 : 0));
#pragma unroll
          for (int h = 0; h < KS; ++h) {
            const int x = (c * KS + h) * kKc;  // first point of K-step h (16-byte aligned coordinate)
            tma_load_3d(dst + h * 2 * kRawTile, map, x, i0, P.a(pr), fb);
            tma_load_3d(dst + h * 2 * kRawTile + kRawTile, map, x, j0, P.b(pr), fb);
          }
          bulk_copy(dst + kRawD, drow + c * KS * kKc, KS * kKc * 8, fb);
          if (s == 0) bulk_copy(dst + kRawMag, mag + static_cast<int64_t>(n) * 128, 128 * 4, fb);
        }
        if (!ok) break;
      }
      // no copy outlives the CTA: the last kRaw issued steps have landed
      // (immediately true unless a wait gave up; bounded either way)
      for (int h = max(0, g - kRaw); h < g; ++h) (void)mbar_wait(rawfull_bar(h % kRaw), (h / kRaw) & 1, status);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------- MMA issue
    if (lane == 0) {
      int g = 0, k = 0;
      for (int n = blockIdx.x; n < n_items; n += gridDim.x, ++k) {
        const int4 item = items[n];
        const int n_steps = item_stages(item);
        const int nbB = item_nb(static_cast<int>(G.bat_fn_ptr[item.x + 1] - G.bat_fn_ptr[item.x]), item.w);
        const int set = k & 1;
        if (!mbar_wait_abort(accempty_bar(set), ((k >> 1) & 1) ^ 1, s_abort, status, G.wait_ns, 64)) break;
        tc_fence_after();
        const uint32_t t0 = tmem + set * kSetCols;
        bool ok = true;
        for (int s = 0; s < n_steps; ++s, ++g) {
          const int st = g % kStages;
          if (!mbar_wait_abort(full_bar(st), (g / kStages) & 1, s_abort, status, G.wait_ns, 32)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int h = 0; h < KS; ++h) {
            const uint32_t a = smem_u32(smem + kSmemStages + st * kStage + h * kHalf), bb = a + kStageA;
            mma_levels(t0, a, bb, (s == 0 && h == 0) ? 0u : 1u, nbB);
          }
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
      bool ok = mbar_wait_abort(accfull_bar(set), (k >> 1) & 1, s_abort, status, G.wait_ns, 256);
      if (bar_red_or(2, kEpiThreads, !ok)) break;
      tc_fence_after();
      const int4 item = items[n];
      const int64_t b = item.x;
      const int o = item.y, i0 = item.z * kTile, j0 = item.w * kTile;
      const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
      const int N = item_nb(nb, item.w);  // accumulator blocks are N columns wide
      const int* idx = G.bat_idx + G.bat_idx_ptr[b];
      double* out = (o == 0 || o == 5) ? V : o == 1 ? W0 : o == 2 ? SOx : o == 3 ? SOy : SOz;
      for (int c0 = eg * 16; c0 < N; c0 += 32) {
#pragma unroll
        for (int blk = 0; blk < 3; ++blk) {
          float vv[16];
          tmem_ld16(tmem + lane_base + set * kSetCols + blk * N + c0, vv);
#pragma unroll
          for (int i = 0; i < 16; ++i) stg[(blk * 128 + et) * kEpiPitch + i] = vv[i];
        }
        bar_sync(3 + eg, 128);
        // thread -> (column, rows): a warp covers 16 consecutive columns of two rows
        const int col = et & 15, j = j0 + c0 + col;
#pragma unroll 2
        for (int qr = 0; qr < 8; ++qr) {
          const int r = (et >> 4) + 8 * qr, i = i0 + r;
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
          if (o == 5) {
            // not symmetric: every (i, j) into its own block
          } else if (o <= 1) {
            if (i > j) continue;
          } else {
            // SO: a diagonal tile pair holds A_k, so A_k(i, j) - A_k(j, i) goes
            // to (i, j), i < j; an off-diagonal one holds SO_k itself (i < j)
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

namespace {

// one launch of the products kernel with KS K-steps per stage over items
// [i0, i0 + n): a persistent grid of at most one CTA per SM
template <int KS>
q4c_status launch_products(const q4c_grid* g, const int4* items, int n, const float* mag, double* V, double* W0,
                           double* SOx, double* SOy, double* SOz, const char* name, cudaStream_t s) {
  using L = split::Layout<KS>;
  Q4C_CUDA(cudaFuncSetAttribute(split::k_split_products<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                L::kSmemTotal));
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  KernelScope ks(name, s);
  split::k_split_products<KS><<<std::min(n, n_sm), split::kThreads, L::kSmemTotal, s>>>(
      g->view(), items, n, reinterpret_cast<const CUtensorMap*>(g->d_tmaps), g->d_dpad, mag, V, W0, SOx, SOy, SOz,
      g->d_status);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

// items[0, n) with their rounding constants mag[128 n]
q4c_status launch_products_ks(int ks, const q4c_grid* g, const int4* items, int n, const float* mag, double* V,
                              double* W0, double* SOx, double* SOy, double* SOz, const char* name, cudaStream_t s) {
  if (n <= 0) return Q4C_OK;
  return ks == 2 ? launch_products<2>(g, items, n, mag, V, W0, SOx, SOy, SOz, name, s)
                 : launch_products<1>(g, items, n, mag, V, W0, SOx, SOy, SOz, name, s);
}

// items of one wave: rounding constants of all of them, then one launch per
// batch-size bucket with the stage shape chosen for that bucket
q4c_status products_items(const q4c_grid* g, const int4* d_items, const std::vector<int64_t>& bucket_w0, int wv,
                          double* V, double* W0, double* SOx, double* SOy, double* SOz, const char* name,
                          cudaStream_t s) {
  const int64_t* r = bucket_w0.data() + static_cast<size_t>(wv) * (kTileBuckets + 1);
  const int64_t i0 = r[0], i1 = r[kTileBuckets];
  if (i1 <= i0) return Q4C_OK;
  {
    KernelScope ks("split_prep", s);
    split::k_item_prep<<<static_cast<unsigned>(i1 - i0), 128, 0, s>>>(g->view(), d_items + i0, g->d_colexp,
                                                                       g->d_split_mag);
  }
  Q4C_CUDA(cudaGetLastError());
  // the rounding constants of item n sit at mag[(n - i0) * 128]; each bucket
  // launch gets its own item list and the constants of its first item
  for (int k = 0; k < kTileBuckets; ++k) {
    const int64_t b0 = r[k], b1 = r[k + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_products_ks(g->split_ks[k], g, d_items + b0, static_cast<int>(b1 - b0),
                                           g->d_split_mag + (b0 - i0) * 128, V, W0, SOx, SOy, SOz, name, s))
      return st;
  }
  return Q4C_OK;
}

}  // namespace

// the products of one wave: rounding constants and the products kernels
// over the wave's items; the wave's offset tables, basis tiles, column
// exponents and D row must already be in place
q4c_status products_wave(const q4c_grid* g, int wv, const q4c_matrices* out, cudaStream_t s) {
  return products_items(g, g->d_split_items, g->split_bw0, wv, out->V, out->W0, out->SOx, out->SOy, out->SOz,
                        "split_products", s);
}

q4c_status integrate_split(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* out,
                           cudaStream_t s) {
  if (g->max_np > 341) {  // exactness bound of the level sums (and the D buffer)
    set_error("q4c_integrate: the split path needs batches of at most 341 points");
    return Q4C_EUNSUPPORTED;
  }
  double* outs[5] = {out->V, out->W0, out->SOx, out->SOy, out->SOz};
  for (double* o : outs) Q4C_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * g->nnz, s));
  const int n_waves = static_cast<int>(g->wave_b0.size()) - 1;
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_fill_idx(t, g, b0, b1, s)) return st;
    if (q4c_status st = launch_basis_df(t, g, b0, b1, v, g->d_colexp, nullptr, 4, s, g->d_dpad)) return st;
    if (q4c_status st = products_wave(g, wv, out, s)) return st;
  }
  return mirror_and_spinor(g, out, s);
}

// The per-column operator of Eq. 19 on the split path: per wave the offset
// tables, the tiles Phi and Psi with D = w (k_basis_df<2>), the rounding
// constants and one products launch over every tile pair; F is written
// element by element (no mirror: it is not symmetric).
q4c_status integrate_columns_split(const q4c_tables* t, const q4c_grid* g, const double* v, double* F,
                                   cudaStream_t s) {
  if (g->max_np > 341) {
    set_error("q4c_integrate_columns: the split path needs batches of at most 341 points");
    return Q4C_EUNSUPPORTED;
  }
  Q4C_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * g->nnz, s));
  const int n_waves = static_cast<int>(g->wave_b0.size()) - 1;
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_fill_idx(t, g, b0, b1, s)) return st;
    if (q4c_status st = launch_basis_df(t, g, b0, b1, v, g->d_colexp, nullptr, 2, s, g->d_dpad)) return st;
    if (q4c_status st = products_items(g, g->d_col_items, g->col_bw0, wv, F, nullptr, nullptr, nullptr, nullptr,
                                       "split_columns", s))
      return st;
  }
  return Q4C_OK;
}

// Tile-shape tuner: on the first wave, with the wave's tables, tiles and
// rounding constants in place, each batch-size bucket's items run with one
// and with two K-steps per stage (one untimed launch, then three timed by
// CUDA events on the stream) into scratch outputs; the faster shape is kept
// for the bucket.  The density/adjoint kernel's shape is chosen the same way
// (one per grid) on the same tiles.
q4c_status autotune_split(const q4c_tables* t, q4c_grid* g, const double* v, cudaStream_t s) {
  if (g->max_np > 341 || g->wave_b0.size() < 2) return Q4C_OK;
  for (int k = 0; k < kTileBuckets; ++k) g->tune_ms[k][0] = g->tune_ms[k][1] = -1.0;
  const int64_t b0 = g->wave_b0[0], b1 = g->wave_b0[1];
  if (b1 <= b0) return Q4C_OK;
  if (q4c_status st = launch_fill_idx(t, g, b0, b1, s)) return st;
  if (q4c_status st = launch_basis_df(t, g, b0, b1, v, g->d_colexp, g->d_rowexp, 4, s, g->d_dpad)) return st;
  {  // the density/adjoint kernel's shape (one per grid), on the same tiles
    double* out = nullptr;
    Q4C_CUDA(cudaMalloc(&out, sizeof(double) * std::max<int64_t>(g->n_pts, 1)));
    const q4c_status st = autotune_rowdot(g, out, s);
    cudaStreamSynchronize(s);
    cudaFree(out);
    if (st) return st;
  }
  const int64_t* r = g->split_bw0.data();
  const int64_t i0 = r[0], i1 = r[kTileBuckets];
  if (i1 <= i0) return Q4C_OK;
  split::k_item_prep<<<static_cast<unsigned>(i1 - i0), 128, 0, s>>>(g->view(), g->d_split_items + i0, g->d_colexp,
                                                                     g->d_split_mag);
  Q4C_CUDA(cudaGetLastError());
  double* scratch = nullptr;
  Q4C_CUDA(cudaMalloc(&scratch, sizeof(double) * 5 * std::max<int64_t>(g->nnz, 1)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  q4c_status status = Q4C_OK;
  auto fail = [&](q4c_status st) { status = st; };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("q4c_autotune: cudaEventCreate failed");
    status = Q4C_ECUDA;
  }
  double* o[5];
  for (int m = 0; m < 5; ++m) o[m] = scratch + m * std::max<int64_t>(g->nnz, 1);
  for (int k = 0; k < kTileBuckets && status == Q4C_OK; ++k) {
    const int64_t c0 = r[k], c1 = r[k + 1];
    if (c1 <= c0) continue;
    const float* mag = g->d_split_mag + (c0 - i0) * 128;
    for (int ks = 1; ks <= 2 && status == Q4C_OK; ++ks) {
      float ms = 0.f;
      if (q4c_status st = launch_products_ks(ks, g, g->d_split_items + c0, static_cast<int>(c1 - c0), mag, o[0],
                                             o[1], o[2], o[3], o[4], "split_tune", s)) {
        fail(st);
        break;
      }
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && status == Q4C_OK; ++rep)
        if (q4c_status st = launch_products_ks(ks, g, g->d_split_items + c0, static_cast<int>(c1 - c0), mag, o[0],
                                               o[1], o[2], o[3], o[4], "split_tune", s))
          fail(st);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        set_error("q4c_autotune: timing failed");
        fail(Q4C_ECUDA);
        break;
      }
      g->tune_ms[k][ks - 1] = ms / 3.0;
    }
    if (status == Q4C_OK) g->split_ks[k] = g->tune_ms[k][1] >= 0.0 && g->tune_ms[k][1] < g->tune_ms[k][0] ? 2 : 1;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(scratch);
  return status;
}

}  // namespace q4c
