// Basis tiles for the split-precision path in double-float arithmetic.
//
// Same values as k_basis_tiles (phi = g S_lm, grad phi = g' d/r S + g grad S,
// Eq. 12 and Appendix B), to about 2^-44 relative instead of FP64's 2^-53,
// computed on the FP32 pipes (GB300's FP64 rate is 1/58 of FP32).  The
// split path slices every value into 47-bit digits against per-column
// exponents and reaches ~1e-12 relative error of the matrices with these
// inputs, far inside its 1e-9 bound.
//
// The log-grid coordinate t = ln(r/r_min)/h is split as t = k + s with k from
// an FP32 logarithm and s = ln(r/r_k)/h from the atanh series
// ln q = 2 (z + z^3/3 + z^5/5 + ...), z = (q - 1)/(q + 1), |z| < 0.03.
//
// One warp handles one active atom and 32 consecutive points of the batch, so
// the loops over the atom's functions are warp-uniform and the per-function
// column maxima reduce across the warp before one shared-memory atomic.
// Outputs (per batch): tiles Phi, X, Y, Z as float2 (hi, lo) in the FP64
// tile layout [4][n_b][ceil8(n_p)]; column exponents (slots 0..3: upper bounds
// for the D-scaled values, D = w v; 4..7: the values) and per-point exponents
// of the four quantities (max over functions).  NQ = 1 computes and stores
// Phi alone (the density contracts Phi only).  NQ = 2 is the per-column
// operator of Eq. 19: Phi and Psi_pj = (v_p + eps_j - V_j(r_pj)) phi_j(p) in
// the planes of Phi and X, with D = w (V_j the column potential splined on
// the radial knots, eps_j its eigenvalue, per radial function).
#include <algorithm>

#include "df.cuh"
#include "internal.h"

namespace q4c {
namespace bdf {

struct cdf {
  float hi, lo;
};
constexpr cdf mk(double c) { return {static_cast<float>(c), static_cast<float>(c - static_cast<double>(static_cast<float>(c)))}; }
__device__ __forceinline__ df D(cdf c) { return {c.hi, c.lo}; }

constexpr cdf c00 = mk(0.28209479177387814);
constexpr cdf c1 = mk(0.4886025119029199);
constexpr cdf c2a = mk(1.0925484305920792);
constexpr cdf c20 = mk(0.31539156525252005);
constexpr cdf c22 = mk(0.5462742152960396);
constexpr cdf c33 = mk(0.5900435899266435);
constexpr cdf c32a = mk(2.890611442640554);
constexpr cdf c31 = mk(0.4570457994644658);
constexpr cdf c30 = mk(0.3731763325901154);
constexpr cdf c32b = mk(1.445305721320277);
constexpr cdf c44a = mk(2.5033429417967046);   // (3/4) sqrt(35/pi)
constexpr cdf c43 = mk(1.7701307697799304);    // (3/4) sqrt(35/(2 pi))
constexpr cdf c42a = mk(0.9461746957575601);   // (3/4) sqrt(5/pi)
constexpr cdf c41 = mk(0.6690465435572892);    // (3/4) sqrt(5/(2 pi))
constexpr cdf c40 = mk(0.10578554691520431);   // (3/16) / sqrt(pi)
constexpr cdf c42b = mk(0.47308734787878004);  // (3/8) sqrt(5/pi)
constexpr cdf c44b = mk(0.6258357354491761);   // (3/16) sqrt(35/pi)
constexpr cdf two_thirds = mk(2.0 / 3.0);

__device__ __forceinline__ int fexp(float x) {  // |x| < 2^fexp(x) for x != 0
  return static_cast<int>((__float_as_uint(x) >> 23) & 0xFF) - 126;
}

__device__ __forceinline__ df split_d(double x) {  // x as an FP32 pair
  const float h = static_cast<float>(x);
  return {h, static_cast<float>(x - static_cast<double>(h))};
}

__device__ __forceinline__ int dexp(double x) {
  return static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF) - 1022;
}

// S_lm and grad S_lm for l <= lmax (index l*l + m + l), Appendix B signs;
// LM is the largest l the caller's arrays hold (3 or 4)
template <int LM>
__device__ __forceinline__ void harmonics(df x, df y, df z, int lmax, df* S, df* dS) {
  const df zero = {0.f, 0.f};
  S[0] = D(c00);
  dS[0] = dS[1] = dS[2] = zero;
  if (lmax < 1) return;
  const df n1 = df_neg(D(c1));
  S[1] = df_mul(n1, y); dS[3] = zero; dS[4] = n1; dS[5] = zero;
  S[2] = df_mul(D(c1), z); dS[6] = zero; dS[7] = zero; dS[8] = D(c1);
  S[3] = df_mul(n1, x); dS[9] = n1; dS[10] = zero; dS[11] = zero;
  if (lmax < 2) return;
  const df xx = df_mul(x, x), yy = df_mul(y, y), zz = df_mul(z, z);
  const df xy = df_mul(x, y), yz = df_mul(y, z), xz = df_mul(x, z);
  const df na = df_neg(D(c2a));
  S[4] = df_mul(D(c2a), xy); dS[12] = df_mul(D(c2a), y); dS[13] = df_mul(D(c2a), x); dS[14] = zero;
  S[5] = df_mul(na, yz); dS[15] = zero; dS[16] = df_mul(na, z); dS[17] = df_mul(na, y);
  const df t20 = df_sub(df_mul_f(zz, 2.f), df_add(xx, yy));  // 2 z^2 - x^2 - y^2
  S[6] = df_mul(D(c20), t20);
  dS[18] = df_mul_f(df_mul(D(c20), x), -2.f);
  dS[19] = df_mul_f(df_mul(D(c20), y), -2.f);
  dS[20] = df_mul_f(df_mul(D(c20), z), 4.f);
  S[7] = df_mul(na, xz); dS[21] = df_mul(na, z); dS[22] = zero; dS[23] = df_mul(na, x);
  const df xmy = df_sub(xx, yy);
  S[8] = df_mul(D(c22), xmy);
  dS[24] = df_mul_f(df_mul(D(c22), x), 2.f);
  dS[25] = df_mul_f(df_mul(D(c22), y), -2.f);
  dS[26] = zero;
  if (lmax < 3) return;
  const df n33 = df_neg(D(c33)), n31 = df_neg(D(c31));
  // m = -3: -c33 y (3x^2 - y^2)
  const df t3a = df_sub(df_mul_f(xx, 3.f), yy);
  S[9] = df_mul(n33, df_mul(y, t3a));
  dS[27] = df_mul_f(df_mul(n33, xy), 6.f);
  dS[28] = df_mul_f(df_mul(n33, xmy), 3.f);
  dS[29] = zero;
  // m = -2: c32a x y z
  S[10] = df_mul(D(c32a), df_mul(xy, z));
  dS[30] = df_mul(D(c32a), yz); dS[31] = df_mul(D(c32a), xz); dS[32] = df_mul(D(c32a), xy);
  // m = -1: -c31 y (4z^2 - x^2 - y^2)
  const df q4 = df_sub(df_mul_f(zz, 4.f), df_add(xx, yy));
  S[11] = df_mul(n31, df_mul(y, q4));
  dS[33] = df_mul_f(df_mul(D(c31), xy), 2.f);
  dS[34] = df_mul(n31, df_sub(df_sub(df_mul_f(zz, 4.f), xx), df_mul_f(yy, 3.f)));
  dS[35] = df_mul_f(df_mul(n31, yz), 8.f);
  // m = 0: c30 z (2z^2 - 3x^2 - 3y^2)
  const df xy2 = df_add(xx, yy);
  S[12] = df_mul(D(c30), df_mul(z, df_sub(df_mul_f(zz, 2.f), df_mul_f(xy2, 3.f))));
  dS[36] = df_mul_f(df_mul(D(c30), xz), -6.f);
  dS[37] = df_mul_f(df_mul(D(c30), yz), -6.f);
  dS[38] = df_mul(D(c30), df_sub(df_mul_f(zz, 6.f), df_mul_f(xy2, 3.f)));
  // m = 1: -c31 x (4z^2 - x^2 - y^2)
  S[13] = df_mul(n31, df_mul(x, q4));
  dS[39] = df_mul(n31, df_sub(df_sub(df_mul_f(zz, 4.f), df_mul_f(xx, 3.f)), yy));
  dS[40] = df_mul_f(df_mul(D(c31), xy), 2.f);
  dS[41] = df_mul_f(df_mul(n31, xz), 8.f);
  // m = 2: c32b z (x^2 - y^2)
  S[14] = df_mul(D(c32b), df_mul(z, xmy));
  dS[42] = df_mul_f(df_mul(D(c32b), xz), 2.f);
  dS[43] = df_mul_f(df_mul(D(c32b), yz), -2.f);
  dS[44] = df_mul(D(c32b), xmy);
  // m = 3: -c33 x (x^2 - 3y^2)
  S[15] = df_mul(n33, df_mul(x, df_sub(xx, df_mul_f(yy, 3.f))));
  dS[45] = df_mul_f(df_mul(n33, xmy), 3.f);
  dS[46] = df_mul_f(df_mul(D(c33), xy), 6.f);
  dS[47] = zero;
  if constexpr (LM >= 4) {
    if (lmax < 4) return;
    // l = 4 (rho = r^2), the same polynomials as the FP64 path
    const df n43 = df_neg(D(c43)), n41 = df_neg(D(c41));
    const df rho = df_add(xy2, zz), xyz = df_mul(xy, z);
    const df q2 = df_sub(df_mul_f(zz, 7.f), rho);                    // 7 z^2 - rho
    const df q1 = df_sub(df_mul_f(zz, 7.f), df_mul_f(rho, 3.f));     // 7 z^2 - 3 rho
    const df q5 = df_sub(df_mul_f(zz, 5.f), rho);                    // 5 z^2 - rho
    const df t3b = df_sub(xx, df_mul_f(yy, 3.f));                    // x^2 - 3 y^2
    const df z3 = df_mul_f(zz, 3.f), z6 = df_mul_f(zz, 6.f);
    S[16] = df_mul(D(c44a), df_mul(xy, xmy));
    dS[48] = df_mul(D(c44a), df_mul(y, t3a));
    dS[49] = df_mul(D(c44a), df_mul(x, t3b));
    dS[50] = zero;
    S[17] = df_mul(n43, df_mul(yz, t3a));
    dS[51] = df_mul_f(df_mul(n43, xyz), 6.f);
    dS[52] = df_mul_f(df_mul(n43, df_mul(z, xmy)), 3.f);
    dS[53] = df_mul(n43, df_mul(y, t3a));
    S[18] = df_mul(D(c42a), df_mul(xy, q2));
    dS[54] = df_mul(D(c42a), df_mul(y, df_sub(df_sub(z6, df_mul_f(xx, 3.f)), yy)));
    dS[55] = df_mul(D(c42a), df_mul(x, df_sub(df_sub(z6, xx), df_mul_f(yy, 3.f))));
    dS[56] = df_mul_f(df_mul(D(c42a), xyz), 12.f);
    S[19] = df_mul(n41, df_mul(yz, q1));
    dS[57] = df_mul_f(df_mul(D(c41), xyz), 6.f);
    dS[58] = df_mul(n41, df_mul(z, df_sub(q1, df_mul_f(yy, 6.f))));
    dS[59] = df_mul_f(df_mul(n41, df_mul(y, q5)), 3.f);
    S[20] = df_mul(D(c40), df_add(df_sub(df_mul_f(df_mul(zz, zz), 35.f), df_mul_f(df_mul(zz, rho), 30.f)),
                                  df_mul_f(df_mul(rho, rho), 3.f)));
    dS[60] = df_mul_f(df_mul(D(c40), df_mul(x, q5)), -12.f);
    dS[61] = df_mul_f(df_mul(D(c40), df_mul(y, q5)), -12.f);
    dS[62] = df_mul_f(df_mul(D(c40), df_mul(z, df_sub(df_mul_f(zz, 5.f), df_mul_f(rho, 3.f)))), 16.f);
    S[21] = df_mul(n41, df_mul(xz, q1));
    dS[63] = df_mul(n41, df_mul(z, df_sub(q1, df_mul_f(xx, 6.f))));
    dS[64] = df_mul_f(df_mul(D(c41), xyz), 6.f);
    dS[65] = df_mul_f(df_mul(n41, df_mul(x, q5)), 3.f);
    S[22] = df_mul(D(c42b), df_mul(xmy, q2));
    dS[66] = df_mul_f(df_mul(D(c42b), df_mul(x, df_sub(z3, xx))), 4.f);
    dS[67] = df_mul_f(df_mul(D(c42b), df_mul(y, df_sub(z3, yy))), -4.f);
    dS[68] = df_mul_f(df_mul(D(c42b), df_mul(z, xmy)), 12.f);
    S[23] = df_mul(n43, df_mul(xz, t3b));
    dS[69] = df_mul_f(df_mul(n43, df_mul(z, xmy)), 3.f);
    dS[70] = df_mul_f(df_mul(D(c43), xyz), 6.f);
    dS[71] = df_mul(n43, df_mul(x, t3b));
    S[24] = df_mul(D(c44b), df_add(df_sub(df_mul(xx, xx), df_mul_f(df_mul(xx, yy), 6.f)), df_mul(yy, yy)));
    dS[72] = df_mul_f(df_mul(D(c44b), df_mul(x, t3b)), 4.f);
    dS[73] = df_mul_f(df_mul(D(c44b), df_mul(y, df_sub(yy, df_mul_f(xx, 3.f)))), 4.f);
    dS[74] = zero;
  }
}

// S_lm alone for l <= lmax (the same polynomials as harmonics)
template <int LM>
__device__ __forceinline__ void harmonics_s(df x, df y, df z, int lmax, df* S) {
  S[0] = D(c00);
  if (lmax < 1) return;
  const df n1 = df_neg(D(c1));
  S[1] = df_mul(n1, y);
  S[2] = df_mul(D(c1), z);
  S[3] = df_mul(n1, x);
  if (lmax < 2) return;
  const df xx = df_mul(x, x), yy = df_mul(y, y), zz = df_mul(z, z);
  const df xy = df_mul(x, y), yz = df_mul(y, z), xz = df_mul(x, z);
  const df na = df_neg(D(c2a));
  S[4] = df_mul(D(c2a), xy);
  S[5] = df_mul(na, yz);
  S[6] = df_mul(D(c20), df_sub(df_mul_f(zz, 2.f), df_add(xx, yy)));
  S[7] = df_mul(na, xz);
  const df xmy = df_sub(xx, yy);
  S[8] = df_mul(D(c22), xmy);
  if (lmax < 3) return;
  const df n33 = df_neg(D(c33)), n31 = df_neg(D(c31));
  S[9] = df_mul(n33, df_mul(y, df_sub(df_mul_f(xx, 3.f), yy)));
  S[10] = df_mul(D(c32a), df_mul(xy, z));
  const df q4 = df_sub(df_mul_f(zz, 4.f), df_add(xx, yy));
  S[11] = df_mul(n31, df_mul(y, q4));
  S[12] = df_mul(D(c30), df_mul(z, df_sub(df_mul_f(zz, 2.f), df_mul_f(df_add(xx, yy), 3.f))));
  S[13] = df_mul(n31, df_mul(x, q4));
  S[14] = df_mul(D(c32b), df_mul(z, xmy));
  S[15] = df_mul(n33, df_mul(x, df_sub(xx, df_mul_f(yy, 3.f))));
  if constexpr (LM >= 4) {
    if (lmax < 4) return;
    const df n43 = df_neg(D(c43)), n41 = df_neg(D(c41));
    const df rho = df_add(df_add(xx, yy), zz);
    const df q2 = df_sub(df_mul_f(zz, 7.f), rho);
    const df q1 = df_sub(df_mul_f(zz, 7.f), df_mul_f(rho, 3.f));
    S[16] = df_mul(D(c44a), df_mul(xy, xmy));
    S[17] = df_mul(n43, df_mul(yz, df_sub(df_mul_f(xx, 3.f), yy)));
    S[18] = df_mul(D(c42a), df_mul(xy, q2));
    S[19] = df_mul(n41, df_mul(yz, q1));
    S[20] = df_mul(D(c40), df_add(df_sub(df_mul_f(df_mul(zz, zz), 35.f), df_mul_f(df_mul(zz, rho), 30.f)),
                                  df_mul_f(df_mul(rho, rho), 3.f)));
    S[21] = df_mul(n41, df_mul(xz, q1));
    S[22] = df_mul(D(c42b), df_mul(xmy, q2));
    S[23] = df_mul(n43, df_mul(xz, df_sub(xx, df_mul_f(yy, 3.f))));
    S[24] = df_mul(D(c44b), df_add(df_sub(df_mul(xx, xx), df_mul_f(df_mul(xx, yy), 6.f)), df_mul(yy, yy)));
  }
}

template <int NQ, int LM>
__global__ void __launch_bounds__(256, 4) k_basis_df(DevBasis B, DevGrid G, DfTables T, int64_t b0,
                                                  const int64_t* __restrict__ scr_off, float2* __restrict__ scratch,
                                                  const double* __restrict__ v, int* __restrict__ colexp,
                                                  int* __restrict__ rowexp, float2* __restrict__ dpad,
                                                  const float4* __restrict__ ccoef, const double* __restrict__ ceps) {
  extern __shared__ int sm[];  // [8][nb] column exponents, then [4][np] point exponents
  const int64_t b = b0 + blockIdx.x;
  const int64_t p0 = G.pt_ptr[b];
  const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
  const int ldp = (np + 7) & ~7;
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  float2* base = scratch + scr_off[b];
  const int64_t plane = static_cast<int64_t>(nb) * ldp;
  int* s_col = sm;
  int* s_row = sm + 8 * nb;
  for (int i = threadIdx.x; i < 8 * nb + 4 * np; i += blockDim.x) sm[i] = -30000;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int n_chunks = (np + 31) / 32;
  for (int wi = warp; wi < na * n_chunks; wi += nwarps) {
    const int a = wi / n_chunks, p = (wi - a * n_chunks) * 32 + lane;
    const bool live = p < np;
    const int A = G.bat_atoms[a0 + a];
    const int f0 = G.bat_atom_fn0[a0 + a];
    const int sp = G.c_sp[A];
    const int r0 = __ldg(B.sp_rad0 + sp), nr = __ldg(B.sp_nrad + sp);
    const int pp = live ? p : 0;
    const df dx = df_sub(T.pts[3 * (p0 + pp)], T.atoms[3 * A]);
    const df dy = df_sub(T.pts[3 * (p0 + pp) + 1], T.atoms[3 * A + 1]);
    const df dz = df_sub(T.pts[3 * (p0 + pp) + 2], T.atoms[3 * A + 2]);
    const df r2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
    // inside the cutoff sphere, below the first knot: in FP32 away from the
    // two spheres; within FP32 rounding of either (where the gradient jumps),
    // from the FP64 coordinates as the FP64 path decides
    bool in = live && r2.hi < T.rc2, below = r2.hi < T.rmin2;
    if (live && (fabsf(r2.hi - T.rc2) <= T.rc2 * 0x1p-18f || fabsf(r2.hi - T.rmin2) <= T.rmin2 * 0x1p-18f)) {
      const double r64 = centre_distance(G.x[p0 + p] - G.c_xyz[3 * A], G.y[p0 + p] - G.c_xyz[3 * A + 1],
                                         G.z[p0 + p] - G.c_xyz[3 * A + 2]);
      in = r64 < B.r_c;
      below = r64 < B.r_min;
    }
    int eD = -30000;
    if (colexp && live) {
      const double Dp = NQ == 2 ? G.w[p0 + p] : G.w[p0 + p] * v[p0 + p];
      if (Dp != 0.0) eD = dexp(Dp);
      if (dpad && a == 0) {  // D = w v as (hi, lo), once per point
        const float h = static_cast<float>(Dp);
        dpad[b * kDPitch + p] = make_float2(h, static_cast<float>(Dp - static_cast<double>(h)));
      }
    } else if (dpad && a == 0 && p < ((np + 31) & ~31)) {
      dpad[b * kDPitch + p] = make_float2(0.f, 0.f);  // stages of 16 or 32 points read zeros past n_p
    }
    const df vdf = (NQ == 2 && live) ? split_d(v[p0 + p]) : df{0.f, 0.f};
    int lmax = 0;
    for (int q = 0; q < nr; ++q) lmax = max(lmax, __ldg(B.rad_l + r0 + q));
    df S[(LM + 1) * (LM + 1)], dS[NQ == 4 ? 3 * (LM + 1) * (LM + 1) : 1];
    if (NQ != 4)
      harmonics_s<LM>(dx, dy, dz, lmax, S);
    else
      harmonics<LM>(dx, dy, dz, lmax, S, dS);
    const bool pos = in && r2.hi > 0.f;  // a point on the nucleus has r = 0 and 1/r taken as 0
    const df r = pos ? df_sqrt(r2) : df{0.f, 0.f};
    const df ir = pos ? df_div(df{1.f, 0.f}, r) : df{0.f, 0.f};
    const df ux = df_mul(dx, ir), uy = df_mul(dy, ir), uz = df_mul(dz, ir);
    // log-grid interval and local coordinate s (shared by the atom's radials)
    int k = 0;
    df s = {0.f, 0.f};
    if (in && !below) {
      const float tf = __logf(r.hi * T.inv_rmin) * T.inv_h;
      k = min(max(static_cast<int>(tf), 0), B.n_log - 2);
      const df qv = df_mul(r, T.inv_knot[k]);
      const df w = df_sub(qv, df{1.f, 0.f});
      const df zq = df_div(w, df_add(w, df{2.f, 0.f}));
      const df z2 = df_mul(zq, zq);
      const float z2f = z2.hi;
      const float tail = 0.4f + z2f * (0.2857142857f + z2f * 0.2222222222f);  // 2/5 + 2/7 z^2 + 2/9 z^4
      df ln = df_add(df_mul_f(zq, 2.f), df_mul(df_mul(zq, z2), D(two_thirds)));
      ln = df_add(ln, df_mul_f(df_mul(zq, z2), z2f * tail));
      s = df_mul(ln, T.inv_h_df);
    }
    int fl = 0;
    float rmax[4] = {-1.f, -1.f, -1.f, -1.f};  // largest |hi| per quantity over this atom's functions
    for (int q = 0; q < nr; ++q) {
      const int rad = r0 + q;
      const int l = __ldg(B.rad_l + rad);
      df g = {0.f, 0.f}, gp = {0.f, 0.f};
      df psi = {0.f, 0.f};  // NQ = 2: v_p + eps_j - V_j(r)
      if (NQ == 2 && in) {
        const float4* vp = ccoef + (static_cast<int64_t>(rad) * (B.n_log - 1) + (below ? 0 : k)) * 2;
        const float4 v01 = __ldg(vp), v23 = __ldg(vp + 1);
        const df V0 = {v01.x, v01.y}, V1 = {v01.z, v01.w}, V2 = {v23.x, v23.y}, V3 = {v23.z, v23.w};
        const df Vr = below ? V0 : df_add(df_mul(df_add(df_mul(df_add(df_mul(V3, s), V2), s), V1), s), V0);
        psi = df_sub(df_add(vdf, split_d(__ldg(ceps + rad))), Vr);
      }
      if (in) {
        if (below) {
          g = T.g0[rad];
        } else {
          const float4* cp = T.coef + (static_cast<int64_t>(rad) * (B.n_log - 1) + k) * 2;
          const float4 c01 = __ldg(cp), c23 = __ldg(cp + 1);
          const df C0 = {c01.x, c01.y}, C1 = {c01.z, c01.w}, C2 = {c23.x, c23.y}, C3 = {c23.z, c23.w};
          const df u = df_add(df_mul(df_add(df_mul(df_add(df_mul(C3, s), C2), s), C1), s), C0);
          const df du = df_add(df_mul(df_add(df_mul(df_mul_f(C3, 3.f), s), df_mul_f(C2, 2.f)), s), C1);
          df irl = ir;
          for (int t = 0; t < l; ++t) irl = df_mul(irl, ir);
          g = df_mul(u, irl);
          if (NQ == 4)
            gp = df_mul(df_mul(df_sub(df_mul(du, T.inv_h_df), df_mul_f(u, static_cast<float>(l + 1))), ir), irl);
        }
      }
      const df gx = df_mul(gp, ux), gy = df_mul(gp, uy), gz = df_mul(gp, uz);
      for (int m = 0; m < 2 * l + 1; ++m, ++fl) {
        const int idx = l * l + m;
        df vals[4];
        vals[0] = df_mul(g, S[idx]);
        if (NQ == 4) {
          vals[1] = df_add(df_mul(gx, S[idx]), df_mul(g, dS[3 * idx]));
          vals[2] = df_add(df_mul(gy, S[idx]), df_mul(g, dS[3 * idx + 1]));
          vals[3] = df_add(df_mul(gz, S[idx]), df_mul(g, dS[3 * idx + 2]));
        } else if (NQ == 2) {
          vals[1] = df_mul(psi, vals[0]);
        }
        const int f = f0 + fl;
        if (live) {
          float2* o = base + static_cast<int64_t>(f) * ldp + p;
#pragma unroll
          for (int c = 0; c < NQ; ++c) o[c * plane] = make_float2(vals[c].hi, vals[c].lo);
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) rmax[c] = fmaxf(rmax[c], fabsf(vals[c].hi));
        if (colexp) {
#pragma unroll
          for (int c = 0; c < NQ; ++c) {
            const float h = vals[c].hi;
            const int e = (live && h != 0.f) ? fexp(h) : -30000;
            const int ea = (e > -30000 && eD > -30000) ? e + eD : -30000;
            const int mb = __reduce_max_sync(0xffffffffu, e);
            const int ma = __reduce_max_sync(0xffffffffu, ea);
            if (lane == 0) {
              if (mb > -30000) atomicMax(&s_col[(4 + c) * nb + f], mb);
              if (ma > -30000) atomicMax(&s_col[c * nb + f], ma);
            }
          }
        }
      }
    }
    if (rowexp && live) {
#pragma unroll
      for (int c = 0; c < NQ; ++c)
        if (rmax[c] > 0.f) atomicMax(&s_row[c * np + p], fexp(rmax[c]));
    }
  }
  __syncthreads();
  if (colexp) {
    int* out = colexp + 8 * G.bat_fn_ptr[b];
    for (int i = threadIdx.x; i < 8 * nb; i += blockDim.x) out[i] = s_col[i];
  }
  if (rowexp) {
    for (int i = threadIdx.x; i < 4 * np; i += blockDim.x) {
      const int c = i / np, p = i - c * np;
      rowexp[4 * (p0 + p) + c] = s_row[i];
    }
  }
}

}  // namespace bdf

q4c_status launch_basis_df(const q4c_tables* t, const q4c_grid* g, int64_t b0, int64_t b1, const double* v,
                           int* colexp, int* rowexp, int nq, cudaStream_t s, float2* dpad) {
  if (nq == 2 && !(t->d_col_coef_df && t->d_col_eps && v)) {
    set_error("launch_basis_df: the per-column operator needs the column potentials and v");
    return Q4C_EINVAL;
  }
  const size_t smem = sizeof(int) * (8 * std::max(g->max_nb, 1) + 4 * std::max(g->max_np, 1));
  // the l <= 3 instantiations keep the smaller harmonic arrays (registers and stack)
  const bool l4 = !t->rad_l.empty() && *std::max_element(t->rad_l.begin(), t->rad_l.end()) >= 4;
  auto kern = nq == 1   ? (l4 ? bdf::k_basis_df<1, 4> : bdf::k_basis_df<1, 3>)
              : nq == 2 ? (l4 ? bdf::k_basis_df<2, 4> : bdf::k_basis_df<2, 3>)
                        : (l4 ? bdf::k_basis_df<4, 4> : bdf::k_basis_df<4, 3>);
  if (nq != 1 && nq != 2 && nq != 4) {
    set_error("launch_basis_df: nq must be 1, 2 or 4");
    return Q4C_EINVAL;
  }
  if (smem > 48 * 1024)
    Q4C_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  DfTables T = t->df_view();
  T.pts = g->d_pts_df;
  T.atoms = g->d_atoms_df;
  KernelScope ks("basis_df", s);
  kern<<<static_cast<unsigned>(b1 - b0), 256, smem, s>>>(t->view(), g->view(), T, b0, g->d_scr_off,
                                                                     reinterpret_cast<float2*>(g->d_scratch), v,
                                                                     colexp, rowexp, dpad, t->d_col_coef_df,
                                                                     t->d_col_eps);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

}  // namespace q4c
