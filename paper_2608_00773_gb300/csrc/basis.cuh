// Device evaluation of the NAO basis phi = u_l(r)/r * Y_lm (Eq. 12a) and its
// gradient, in FP64.
//
// phi = g(r) S_lm(d), g = u/r^(l+1), S_lm = r^l Y_lm a homogeneous polynomial
// in d = r - R_atom; grad phi = g'(r) (d/r) S_lm + g grad S_lm.
// Y_lm follows Appendix B (Eqs. B1-B3) literally: the (-1)^m of B1 times a
// phase-free associated Legendre function, which makes the m = +-1, +-3
// polynomials below the negatives of the phase-free real harmonics.
#pragma once

#include "internal.h"

namespace q4c {

// cubic spline on the logarithmic grid: g = u/r^(l+1) and dg/dr, r < r_c
__device__ __forceinline__ void radial_g(const DevBasis& B, int rad, int l, double r, double inv_r, double& g,
                                         double& gp) {
  if (r < B.r_min) {  // u = u(r_min) (r/r_min)^(l+1): g constant
    g = __ldg(B.g0 + rad);
    gp = 0.0;
    return;
  }
  const double t = log(r * B.inv_rmin) * B.inv_h;
  int k = static_cast<int>(t);
  if (k > B.n_log - 2) k = B.n_log - 2;
  const double s = t - k;
  const double2* c2 = reinterpret_cast<const double2*>(B.coef + (static_cast<size_t>(rad) * (B.n_log - 1) + k) * 4);
  const double2 c01 = __ldg(c2), c23 = __ldg(c2 + 1);
  const double u = c01.x + s * (c01.y + s * (c23.x + s * c23.y));
  const double du_ds = c01.y + s * (2.0 * c23.x + 3.0 * s * c23.y);
  double irl1 = inv_r;
  for (int q = 0; q < l; ++q) irl1 *= inv_r;
  g = u * irl1;
  gp = (du_ds * B.inv_h - (l + 1) * u) * inv_r * irl1;
}

// S_lm and grad S_lm for l <= lmax (lmax <= 4), index l*l + (m + l)
__device__ __forceinline__ void solid_harmonics(double x, double y, double z, int lmax, double* S, double* dS) {
  constexpr double c00 = 0.28209479177387814;   // 1/(2 sqrt(pi))
  constexpr double c1 = 0.4886025119029199;     // sqrt(3/(4 pi))
  constexpr double c2a = 1.0925484305920792;    // sqrt(15/pi)/2
  constexpr double c20 = 0.31539156525252005;   // sqrt(5/pi)/4
  constexpr double c22 = 0.5462742152960396;    // sqrt(15/pi)/4
  constexpr double c33 = 0.5900435899266435;    // sqrt(35/(2 pi))/4
  constexpr double c32a = 2.890611442640554;    // sqrt(105/pi)/2
  constexpr double c31 = 0.4570457994644658;    // sqrt(21/(2 pi))/4
  constexpr double c30 = 0.3731763325901154;    // sqrt(7/pi)/4
  constexpr double c32b = 1.445305721320277;    // sqrt(105/pi)/4
  constexpr double c44a = 2.5033429417967046;   // (3/4) sqrt(35/pi)
  constexpr double c43 = 1.7701307697799304;    // (3/4) sqrt(35/(2 pi))
  constexpr double c42a = 0.9461746957575601;   // (3/4) sqrt(5/pi)
  constexpr double c41 = 0.6690465435572892;    // (3/4) sqrt(5/(2 pi))
  constexpr double c40 = 0.10578554691520431;   // (3/16) / sqrt(pi)
  constexpr double c42b = 0.47308734787878004;  // (3/8) sqrt(5/pi)
  constexpr double c44b = 0.6258357354491761;   // (3/16) sqrt(35/pi)
  S[0] = c00;
  dS[0] = dS[1] = dS[2] = 0.0;
  if (lmax < 1) return;
  // l = 1: m = -1, 0, 1 -> -c y, c z, -c x
  S[1] = -c1 * y; dS[3] = 0.0; dS[4] = -c1; dS[5] = 0.0;
  S[2] = c1 * z;  dS[6] = 0.0; dS[7] = 0.0; dS[8] = c1;
  S[3] = -c1 * x; dS[9] = -c1; dS[10] = 0.0; dS[11] = 0.0;
  if (lmax < 2) return;
  const double xx = x * x, yy = y * y, zz = z * z;
  // l = 2
  S[4] = c2a * x * y;              dS[12] = c2a * y; dS[13] = c2a * x; dS[14] = 0.0;
  S[5] = -c2a * y * z;             dS[15] = 0.0; dS[16] = -c2a * z; dS[17] = -c2a * y;
  S[6] = c20 * (2.0 * zz - xx - yy); dS[18] = -2.0 * c20 * x; dS[19] = -2.0 * c20 * y; dS[20] = 4.0 * c20 * z;
  S[7] = -c2a * x * z;             dS[21] = -c2a * z; dS[22] = 0.0; dS[23] = -c2a * x;
  S[8] = c22 * (xx - yy);          dS[24] = 2.0 * c22 * x; dS[25] = -2.0 * c22 * y; dS[26] = 0.0;
  if (lmax < 3) return;
  // l = 3
  S[9] = -c33 * y * (3.0 * xx - yy);
  dS[27] = -c33 * 6.0 * x * y; dS[28] = -c33 * 3.0 * (xx - yy); dS[29] = 0.0;
  S[10] = c32a * x * y * z;
  dS[30] = c32a * y * z; dS[31] = c32a * x * z; dS[32] = c32a * x * y;
  S[11] = -c31 * y * (4.0 * zz - xx - yy);
  dS[33] = c31 * 2.0 * x * y; dS[34] = -c31 * (4.0 * zz - xx - 3.0 * yy); dS[35] = -c31 * 8.0 * y * z;
  S[12] = c30 * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
  dS[36] = -c30 * 6.0 * x * z; dS[37] = -c30 * 6.0 * y * z; dS[38] = c30 * (6.0 * zz - 3.0 * xx - 3.0 * yy);
  S[13] = -c31 * x * (4.0 * zz - xx - yy);
  dS[39] = -c31 * (4.0 * zz - 3.0 * xx - yy); dS[40] = c31 * 2.0 * x * y; dS[41] = -c31 * 8.0 * x * z;
  S[14] = c32b * z * (xx - yy);
  dS[42] = c32b * 2.0 * x * z; dS[43] = -c32b * 2.0 * y * z; dS[44] = c32b * (xx - yy);
  S[15] = -c33 * x * (xx - 3.0 * yy);
  dS[45] = -c33 * 3.0 * (xx - yy); dS[46] = c33 * 6.0 * x * y; dS[47] = 0.0;
  if (lmax < 4) return;
  // l = 4 (rho = r^2); the sign (-1)^|m| of Appendix B on every m != 0 term
  const double rho = xx + yy + zz, xyz = x * y * z;
  const double q2 = 7.0 * zz - rho, q1 = 7.0 * zz - 3.0 * rho, q5 = 5.0 * zz - rho;
  S[16] = c44a * x * y * (xx - yy);
  dS[48] = c44a * y * (3.0 * xx - yy); dS[49] = c44a * x * (xx - 3.0 * yy); dS[50] = 0.0;
  S[17] = -c43 * y * z * (3.0 * xx - yy);
  dS[51] = -6.0 * c43 * xyz; dS[52] = -3.0 * c43 * z * (xx - yy); dS[53] = -c43 * y * (3.0 * xx - yy);
  S[18] = c42a * x * y * q2;
  dS[54] = c42a * y * (6.0 * zz - 3.0 * xx - yy); dS[55] = c42a * x * (6.0 * zz - xx - 3.0 * yy);
  dS[56] = 12.0 * c42a * xyz;
  S[19] = -c41 * y * z * q1;
  dS[57] = 6.0 * c41 * xyz; dS[58] = -c41 * z * (q1 - 6.0 * yy); dS[59] = -3.0 * c41 * y * q5;
  S[20] = c40 * (35.0 * zz * zz - 30.0 * zz * rho + 3.0 * rho * rho);
  dS[60] = -12.0 * c40 * x * q5; dS[61] = -12.0 * c40 * y * q5; dS[62] = 16.0 * c40 * z * (5.0 * zz - 3.0 * rho);
  S[21] = -c41 * x * z * q1;
  dS[63] = -c41 * z * (q1 - 6.0 * xx); dS[64] = 6.0 * c41 * xyz; dS[65] = -3.0 * c41 * x * q5;
  S[22] = c42b * (xx - yy) * q2;
  dS[66] = 4.0 * c42b * x * (3.0 * zz - xx); dS[67] = -4.0 * c42b * y * (3.0 * zz - yy);
  dS[68] = 12.0 * c42b * z * (xx - yy);
  S[23] = -c43 * x * z * (xx - 3.0 * yy);
  dS[69] = -3.0 * c43 * z * (xx - yy); dS[70] = 6.0 * c43 * xyz; dS[71] = -c43 * x * (xx - 3.0 * yy);
  S[24] = c44b * (xx * xx - 6.0 * xx * yy + yy * yy);
  dS[72] = 4.0 * c44b * x * (xx - 3.0 * yy); dS[73] = 4.0 * c44b * y * (yy - 3.0 * xx); dS[74] = 0.0;
}

// Evaluates every function of one atom at one point.  out(k, phi, gx, gy, gz)
// is called for k = 0..nf-1 in the basis order (radial, then m = -l..l).
template <typename Out>
__device__ __forceinline__ void atom_functions(const DevBasis& B, int species, double dx, double dy, double dz,
                                               Out&& out) {
  const int r0 = __ldg(B.sp_rad0 + species), nr = __ldg(B.sp_nrad + species);
  const double r = centre_distance(dx, dy, dz);
  if (!(r < B.r_c)) {
    int k = 0;
    for (int q = 0; q < nr; ++q) {
      const int l = __ldg(B.rad_l + r0 + q);
      for (int m = 0; m < 2 * l + 1; ++m) out(k++, 0.0, 0.0, 0.0, 0.0);
    }
    return;
  }
  int lmax = 0;
  for (int q = 0; q < nr; ++q) lmax = max(lmax, __ldg(B.rad_l + r0 + q));
  double S[(kMaxL + 1) * (kMaxL + 1)], dS[3 * (kMaxL + 1) * (kMaxL + 1)];
  solid_harmonics(dx, dy, dz, lmax, S, dS);
  const double inv_r = r > 0.0 ? 1.0 / r : 0.0;
  const double ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
  int k = 0;
  for (int q = 0; q < nr; ++q) {
    const int l = __ldg(B.rad_l + r0 + q);
    double g, gp;
    radial_g(B, r0 + q, l, r, inv_r, g, gp);
    for (int m = 0; m < 2 * l + 1; ++m) {
      const int idx = l * l + m;
      const double s = S[idx];
      out(k++, g * s, gp * ux * s + g * dS[3 * idx], gp * uy * s + g * dS[3 * idx + 1],
          gp * uz * s + g * dS[3 * idx + 2]);
    }
  }
}

}  // namespace q4c
