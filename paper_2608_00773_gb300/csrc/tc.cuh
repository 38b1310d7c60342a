// tcgen05 helpers shared by the split-precision kernels: shared-memory
// matrix and instruction descriptors, MMA issue/commit, bounded mbarrier
// waits, tensor-memory loads and the six-digit BF16 splitting of FP64 values.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace q4c {
namespace tc {

constexpr int kSlices = 6;
constexpr int kLBO = 128;                         // core matrices adjacent in K
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s of wall clock per drain wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, no-swizzle shared-memory matrix descriptor (tcgen05 format);
// sbo = byte distance between 8-row groups
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((kLBO >> 4) & 0x3FFF) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version for tcgen05
  return d;                              // base offset 0, swizzle none
}

// kind::f16 instruction descriptor: BF16 x BF16 -> FP32, both K-major
__device__ __forceinline__ uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// ---- the 21 slice products of one K-step (s + t <= 5) as six MMAs
// Operand tiles are 64 rows x 16 K BF16 (2 KB, no-swizzle K-major).  A is
// stored as seven tiles [Z, A0..A5] (Z zeros), so the M = 128 operand starting
// at tile q is [A_(q-1); A_q]; B is stored as [B0, B2, B4, B1, B3, B5].  An MMA
// of [A_a; A_(a+1)] with the consecutive B tiles B_t, B_(t+2), ... (a + t even)
// adds level a + t + 2c to the top lanes and level a + t + 2c + 1 to the bottom
// lanes of the 64-column block (a + t)/2 + c, so the three blocks [L0;L1],
// [L2;L3], [L4;L5] at tmem receive exactly the pairs of their levels:
//   [A0;A1] x [B0,B2,B4]  -> blocks 0-2   (6 pairs)
//   [Z;A0]  x [B1,B3,B5]  -> blocks 0-2   (3 pairs, bottom lanes)
//   [A2;A3] x [B0,B2]     -> blocks 1-2   (4 pairs)
//   [A1;A2] x [B1,B3]     -> blocks 1-2   (4 pairs)
//   [A4;A5] x B0          -> block 2      (2 pairs)
//   [A3;A4] x B1          -> block 2      (2 pairs)
constexpr int kLevelTile = 2048;     // bytes per 64-row operand tile
constexpr uint32_t kLevelSBO = 256;  // bytes between 8-row groups
constexpr int kRowBytes = 32;        // one row of 16 K values (BF16)

// tile position of B slice t in the stage
__host__ __device__ constexpr int b_tile(int t) { return (t & 1) ? 3 + (t >> 1) : (t >> 1); }

// a, b: shared addresses of tile Z of A (64-row tiles) and of the first B
// tile; the six B tiles hold nb rows each (nb a multiple of 16, <= 64;
// tile pos at b + pos * nb * 32), so the three accumulator blocks are nb
// columns wide ([L0;L1] at tmem, [L2;L3] at tmem + nb, [L4;L5] at tmem +
// 2 nb); acc = 0 starts the accumulators (the first MMA covers all three)
__device__ __forceinline__ void mma_levels(uint32_t tmem, uint32_t a, uint32_t b, uint32_t acc, int nb) {
  auto A = [&](int q) { return make_desc(a + q * kLevelTile, kLevelSBO); };
  auto Bt = [&](int pos) { return make_desc(b + pos * nb * kRowBytes, kLevelSBO); };
  mma_bf16(tmem, A(1), Bt(0), make_idesc(128, 3 * nb), acc);
  mma_bf16(tmem, A(0), Bt(3), make_idesc(128, 3 * nb), 1u);
  mma_bf16(tmem + nb, A(3), Bt(0), make_idesc(128, 2 * nb), 1u);
  mma_bf16(tmem + nb, A(2), Bt(3), make_idesc(128, 2 * nb), 1u);
  mma_bf16(tmem + 2 * nb, A(5), Bt(0), make_idesc(128, nb), 1u);
  mma_bf16(tmem + 2 * nb, A(4), Bt(3), make_idesc(128, nb), 1u);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait; returns false (and sets the status bit) once 1 s has passed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) break;
  }
  atomicOr(status, 1u);
  return false;
}

// bounded wait of a working role (limit_ns of wall clock, the grid's work
// wait limit) that also gives up as soon as another role of the CTA has set
// *abort (a role that times out sets it and the status bit); the drain waits
// before a CTA exits keep the fixed 1 s limit of mbar_wait
// (sleep_ns > 0: back off between polls, for roles whose waits are long and
// whose polling would take issue slots from the working warps)
__device__ __forceinline__ bool mbar_wait_abort(uint32_t bar, uint32_t parity, volatile int* abort,
                                                unsigned* status, uint64_t limit_ns, unsigned sleep_ns = 0) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (sleep_ns) __nanosleep(sleep_ns);
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > limit_ns) {
      *abort = 1;
      atomicOr(status, 1u);
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

// named barrier over n threads
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// named barrier over n threads that returns the OR of p over them
__device__ __forceinline__ bool bar_red_or(int id, int n, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(p)), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// the phase of an mbarrier also waits for `bytes` of asynchronous copies
__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bulk global -> shared copy (16-byte aligned addresses, size a multiple of
// 16) that completes `bytes` of transactions on the mbarrier
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// arrive on the mbarrier and add `bytes` to the transactions its phase waits for
__device__ __forceinline__ void arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// tiled TMA load of one box of a 3-D tensor map (in global memory) at
// element coordinates (x, y, z); completes the box's bytes on the mbarrier.
// x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM loads: the destination registers of tcgen05.ld are defined only
// after tcgen05.wait::ld, so each helper issues its loads and the wait in ONE
// asm statement; its outputs then exist only after the wait, and no use of
// them can be scheduled ahead of it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// three 8-column loads (one per address) under a single wait
__device__ __forceinline__ void tmem_ld8x3(uint32_t t0, uint32_t t1, uint32_t t2, float* v0, float* v1, float* v2) {
  uint32_t a[8], b[8], c[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
        "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
      : "r"(t0), "r"(t1), "r"(t2)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v0[i] = __uint_as_float(a[i]);
    v1[i] = __uint_as_float(b[i]);
    v2[i] = __uint_as_float(c[i]);
  }
}

// ------------------------------------------------------------ slicing
// The split of a value x against a column exponent e (|x| <= 2^e):
//   x = sum_s d_s 2^(e - 6 - 8 s) + O(2^(e - 47)),  s = 0..5,
// with balanced digits, each exact in BF16.

// Rounding constant of the leading digit for column exponent e: 1.5 2^(e + 17).
// Adding and subtracting 1.5 2^(23 + u) in FP32 rounds x to the nearest
// multiple of 2^u, exactly, whenever |x| < 2^(22 + u).  An empty column
// (e < -1000) gets 0; e is clamped to [-80, 100] so that every digit weight
// 2^(e - 6 - 8s) stays a normal FP32 and BF16 number.
__device__ __forceinline__ float magic0(int e) {
  if (e < -1000) return 0.0f;
  e = min(max(e, -80), 100);
  return __int_as_float(((e + 17 + 127) << 23) | 0x400000);
}

// Six balanced digits of the double-float value h + l (|h + l| <= 2^e) with
// m0 = magic0(e): digit s is returned already multiplied by its weight
// 2^(e - 6 - 8s).  Digits 0-2 come from h exactly (|d| <= 64, 128, 128); l
// joins the residual (|r| <= 2^(e - 23)) before digit 3, rounded at most
// 2^(e - 48), so |d3| <= 160 and |d4|, |d5| <= 128, all exact in BF16, and
// the six digits represent h + l within 2^(e - 46).
__device__ __forceinline__ void slice6(float h, float l, float m0, float d[kSlices]) {
  float x = h, m = m0;
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    if (s == 3) x = __fadd_rn(x, l);
    const float t = __fsub_rn(__fadd_rn(x, m), m);
    d[s] = t;
    x = __fsub_rn(x, t);
    m = __fmul_rn(m, 0x1p-8f);
  }
}

// ------------------------------------------------------------ pairs
// Two FP32 values operated on by the packed float2 instructions of sm_100
// and later (CUDA's __fadd2_rn, __fmul2_rn, __ffma2_rn): each half is
// rounded on its own exactly as the scalar instruction would, and one
// instruction does the work of two (the slicers are bound by instruction
// issue, not by FP32 lanes).  a - b is fma(b, -1, a), one rounding of the
// exact difference, as the scalar subtraction.
__device__ __forceinline__ float2 pk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }  // a b + c

// BF16 pair (low half = .x) of two FP32 values that are exact in BF16 (their
// low 16 bits are zero): the upper halves, by byte permute
__device__ __forceinline__ uint32_t bf16x2_exact(float2 v) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(r) : "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)));
  return r;
}

// double-float products of two pairs (x = xh + xl, y = yh + yl per half),
// the same operations as df_mul: p = xh yh, e = fma(xh, yh, -p) (with
// -p = xh (-yh) rounded, nyh = -yh), e = fma(xh, yl, e), e = fma(xl, yh, e),
// then the fast two-sum of p and e
__device__ __forceinline__ void df_mul2(float2 xh, float2 xl, float2 yh, float2 yl, float2 nyh, float2& rh,
                                        float2& rl) {
  const float2 p = mul2(xh, yh);
  float2 e = fma2(xh, yh, mul2(xh, nyh));
  e = fma2(xh, yl, e);
  e = fma2(xl, yh, e);
  rh = add2(p, e);
  rl = sub2(e, sub2(rh, p));
}

// slice6 on a pair of values (h + l per half) against the same rounding
// constant m0 for both: d[s] holds digit s of both halves, weighted
__device__ __forceinline__ void slice6x2(float2 h, float2 l, float m0, float2 d[kSlices]) {
  float2 x = h;
  float m = m0;
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    if (s == 3) x = add2(x, l);
    const float2 mm = pk2(m, m);
    const float2 t = sub2(add2(x, mm), mm);
    d[s] = t;
    if (s + 1 < kSlices) x = sub2(x, t);
    m = __fmul_rn(m, 0x1p-8f);
  }
}

}  // namespace tc
}  // namespace q4c
