/*
 * q4c_oracle.c -- plain, slow, FP64 CPU oracle for the Q4C real-space
 * integration path.  TEST INFRASTRUCTURE ONLY: it is used by tests/, by
 * __graft_entry__.smoke() and by bench.py's cpu_baseline / reference arm,
 * never by the product path.  It shares no code, header or table with the
 * CUDA library; the two meet only through the seeded inputs in workloads/.
 *
 * Everything here is the definition written out, one loop per sum, with no
 * batching, screening beyond exact zeros, blocking or reordering:
 *
 *   V_ij    = sum_p w_p v_p phi_i(p) phi_j(p)                  (Eqs. 29-30,
 *             grid sum of a matrix element with F = v)
 *   W0_ij   = sum_p w_p v_p grad phi_i . grad phi_j            (kinetic-balance
 *   SOk_ij  = sum_p w_p v_p (grad phi_i x grad phi_j)_k         small-component
 *             reading of the SS block of Eq. 16: (s.a)(s.b) = a.b + i s.(a x b))
 *   n_p     = sum_ij P_ij phi_i(p) phi_j(p)                    (Eqs. 39-40)
 *   dL/dv_p = w_p sum_M sum_ij G^M_ij f^M_ij(p)                (adjoint of the
 *             linear map v -> (V, W0, SOx, SOy, SOz); the paper has no gradients)
 *
 * Basis (Eq. 12a): phi = u_l(r)/r * Y_lm, Y_lm real spherical harmonics of
 * Appendix B (Eqs. B1-B3) taken literally: the (-1)^m of B1 multiplies an
 * associated Legendre function defined in B2 without a phase.
 * Radial functions are tabulated on a logarithmic grid and interpolated by a
 * natural cubic spline in the grid index (the paper only says "numerically
 * on one-dimensional logarithmic grids", Eq. 12).
 * Integration grid: overlapping atom-centred grids with a partition of unity
 * (Section III A); Becke's partition (Becke 1988, three iterations of
 * f(mu) = 1.5 mu - 0.5 mu^3), radial Gauss-Chebyshev of the second kind with
 * Becke's map, angular Gauss-Legendre x uniform product grid.
 *
 * Sums use Neumaier's compensated summation in double so that results do
 * not depend on the host's long double format.
 *
 * Parity pins (tests/test_oracle_*.py): Gaussian overlap and kinetic closed
 * forms, the one-centre erf-potential integral, one-atom spin-orbit radial
 * integral, Y_lm against scipy's complex harmonics and Eq. 13, orthonormality,
 * Becke partition of unity, spline against scipy's natural CubicSpline,
 * symmetry, translation invariance, Tr(PS) = sum_p w_p n_p, adjoint linearity.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* compensated accumulator (Neumaier 1974)                              */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } orc_acc;
static void acc_add(orc_acc* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double acc_get(const orc_acc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* quadrature                                                           */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1], Newton's method
 * on P_n with the three-term recurrence. */
int orc_gauss_legendre(int n, double* x, double* w) {
  if (n < 1) return -1;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn = 0.0, pm = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      /* P_n(z) and P_{n-1}(z) by (k) P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2} */
      pn = z; pm = 1.0;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
        pm = pn; pn = pk;
      }
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    pn = z; pm = 1.0;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
      pm = pn; pn = pk;
    }
    dp = n * (z * pn - pm) / (z * z - 1.0);
    /* the initial guesses descend; store ascending */
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* Radial shells: Gauss-Chebyshev of the second kind, x_i = cos(i pi/(N+1)),
 * i = 1..N, mapped by r = R (1+x)/(1-x).  The weight integrates
 * int_0^inf F(r) r^2 dr:  w_i = pi/(N+1) sin(theta_i) r_i^2 2R/(1-x_i)^2. */
void orc_radial_shells(int N, double R, double* r, double* w) {
  for (int i = 1; i <= N; ++i) {
    double th = i * M_PI / (N + 1);
    double x = cos(th);
    double ri = R * (1.0 + x) / (1.0 - x);
    r[i - 1] = ri;
    w[i - 1] = M_PI / (N + 1) * sin(th) * ri * ri * 2.0 * R / ((1.0 - x) * (1.0 - x));
  }
}

/* ------------------------------------------------------------------ */
/* radial functions                                                     */
/* ------------------------------------------------------------------ */

/* smooth cutoff: 1 below r_on, 0 from r_c on, quintic smoothstep between */
double orc_cutoff(double r, double r_on, double r_c) {
  if (r <= r_on) return 1.0;
  if (r >= r_c) return 0.0;
  double s = (r - r_on) / (r_c - r_on);
  return 1.0 - (10.0 * s * s * s - 15.0 * s * s * s * s + 6.0 * s * s * s * s * s);
}

/* Knots r_k = r_min (r_c/r_min)^(k/(n-1)), values u_k = r^(l+1) e^(-alpha r^2) c(r),
 * and the natural cubic spline second derivatives M_k in the index variable
 * t = k (unit spacing): M_{k-1} + 4 M_k + M_{k+1} = 6 (u_{k+1} - 2u_k + u_{k-1}),
 * M_0 = M_{n-1} = 0, solved by plain Gaussian elimination of the
 * tridiagonal system. */
/* Second derivatives M_k (in the knot index) of the natural cubic spline
 * through u_0..u_{n-1}: M_0 = M_{n-1} = 0, M_{k-1} + 4 M_k + M_{k+1} =
 * 6 (u_{k+1} - 2 u_k + u_{k-1}). */
static void orc_natural_M(int n, const double* u, double* M) {
  int m = n - 2; /* unknowns M_1..M_{n-2} */
  double* diag = (double*)malloc(sizeof(double) * m);
  double* rhs = (double*)malloc(sizeof(double) * m);
  for (int i = 0; i < m; ++i) {
    int k = i + 1;
    diag[i] = 4.0;
    rhs[i] = 6.0 * (u[k + 1] - 2.0 * u[k] + u[k - 1]);
  }
  /* forward elimination with unit off-diagonals */
  for (int i = 1; i < m; ++i) {
    double f = 1.0 / diag[i - 1];
    diag[i] -= f;
    rhs[i] -= f * rhs[i - 1];
  }
  M[0] = 0.0;
  M[n - 1] = 0.0;
  M[m] = rhs[m - 1] / diag[m - 1];
  for (int i = m - 2; i >= 0; --i) M[i + 1] = (rhs[i] - M[i + 2]) / diag[i];
  free(diag);
  free(rhs);
}

/* The same second derivatives for radial values given at the knots (the
 * small-component radials Q(r) of Eq. 12b enter this way). */
int orc_spline_second(int n, const double* u, double* M) {
  if (n < 3) return -1;
  orc_natural_M(n, u, M);
  return 0;
}

int orc_tabulate(int l, double alpha, int n, double r_min, double r_c, double r_on,
                 double* r, double* u, double* M) {
  if (n < 3) return -1;
  for (int k = 0; k < n; ++k) {
    double rk = r_min * pow(r_c / r_min, (double)k / (double)(n - 1));
    r[k] = rk;
    u[k] = pow(rk, l + 1) * exp(-alpha * rk * rk) * orc_cutoff(rk, r_on, r_c);
  }
  orc_natural_M(n, u, M);
  return 0;
}

/* Spline value u(r) and du/dr.  t = ln(r/r_min)/h, h = ln(r_c/r_min)/(n-1);
 * on [k, k+1] with s = t - k:
 *   u = (1-s) u_k + s u_{k+1} + ((1-s)^3 - (1-s)) M_k/6 + (s^3 - s) M_{k+1}/6.
 * Below r_min: u = u_0 (r/r_min)^(l+1).  From r_c on: 0. */
void orc_spline_eval(int l, int n, double r_min, double r_c, const double* u, const double* M,
                     double r, double* uval, double* dudr) {
  if (r >= r_c) { *uval = 0.0; *dudr = 0.0; return; }
  if (r < r_min) {
    double q = pow(r / r_min, l);
    *uval = u[0] * q * (r / r_min);
    *dudr = u[0] * (l + 1) * q / r_min;
    return;
  }
  double h = log(r_c / r_min) / (n - 1);
  double t = log(r / r_min) / h;
  int k = (int)floor(t);
  if (k > n - 2) k = n - 2;
  if (k < 0) k = 0;
  double s = t - k, a = 1.0 - s;
  double val = a * u[k] + s * u[k + 1] + (a * a * a - a) * M[k] / 6.0 + (s * s * s - s) * M[k + 1] / 6.0;
  double dt = -u[k] + u[k + 1] + (-3.0 * a * a + 1.0) * M[k] / 6.0 + (3.0 * s * s - 1.0) * M[k + 1] / 6.0;
  *uval = val;
  *dudr = dt / (h * r);
}

/* ------------------------------------------------------------------ */
/* real spherical harmonics, Appendix B                                 */
/* ------------------------------------------------------------------ */

static double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}
static double binom(int a, int b) { return factorial(a) / (factorial(b) * factorial(a - b)); }

/* K_l^m of Eq. B3 */
double orc_K(int l, int m) {
  int am = abs(m);
  return sqrt((2.0 * l + 1.0) * factorial(l - am) / (4.0 * M_PI * factorial(l + am)));
}

/* Coefficients a_k of the m-th derivative of the Legendre polynomial P_l:
 * d^m/dt^m P_l(t) = sum_k a[k] t^k, k = 0..l-m.  From the explicit sum
 * P_l(t) = 2^-l sum_j (-1)^j C(l,j) C(2l-2j,l) t^(l-2j). */
static void legendre_deriv_coeffs(int l, int m, double* a) {
  for (int k = 0; k <= l; ++k) a[k] = 0.0;
  for (int j = 0; 2 * j <= l; ++j) {
    int p = l - 2 * j;
    if (p < m) continue;
    double c = ldexp(1.0, -l) * ((j & 1) ? -1.0 : 1.0) * binom(l, j) * binom(2 * l - 2 * j, l);
    c *= factorial(p) / factorial(p - m);
    a[p - m] += c;
  }
}

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

/* Y_l^m(theta, phi) straight from Eqs. B1-B3 (used by the pins). */
double orc_ylm_spherical(int l, int m, double theta, double phi) {
  int am = abs(m);
  double a[16];
  legendre_deriv_coeffs(l, am, a);
  double ct = cos(theta), st = sin(theta);
  double dP = 0.0;
  for (int k = 0; k <= l - am; ++k) dP += a[k] * ipow(ct, k);
  double Plm = ipow(st, am) * dP; /* Eq. B2: (sin)^m d^m/dx^m P_l */
  double sgn = (am & 1) ? -1.0 : 1.0;
  if (m > 0) return sgn * sqrt(2.0) * orc_K(l, m) * cos(m * phi) * Plm;
  if (m == 0) return orc_K(l, 0) * Plm;
  return sgn * sqrt(2.0) * orc_K(l, m) * sin(am * phi) * Plm;
}

/* Solid harmonic S_lm = r^l Y_lm and its Cartesian gradient.
 * r^l Y_lm = N * A_m(x,y) * Pi_lm(z, r^2) with
 *   A_m = Re (x+iy)^|m| (m > 0), Im (x+iy)^|m| (m < 0), 1 (m = 0),
 *   Pi  = r^(l-|m|) (d^|m| P_l)(z/r) = sum_k a_k z^k (r^2)^((l-|m|-k)/2),
 *   N   = (-1)^m sqrt(2) K_l^m (m != 0), K_l^0 (m = 0). */
void orc_solid_harmonic(int l, int m, double x, double y, double z, double* S, double* dS) {
  int am = abs(m);
  double a[16];
  legendre_deriv_coeffs(l, am, a);
  double rho = x * x + y * y + z * z;
  /* A_m and its partials via (x+iy)^m recurrences */
  double C = 1.0, Sn = 0.0, Cm1 = 0.0, Sm1 = 0.0;
  for (int k = 1; k <= am; ++k) {
    Cm1 = C; Sm1 = Sn;
    double c2 = x * C - y * Sn, s2 = x * Sn + y * C;
    C = c2; Sn = s2;
  }
  double A, Ax, Ay;
  if (m > 0) { A = C; Ax = am * Cm1; Ay = -am * Sm1; }
  else if (m < 0) { A = Sn; Ax = am * Sm1; Ay = am * Cm1; }
  else { A = 1.0; Ax = 0.0; Ay = 0.0; }
  int q = l - am;
  double Pi = 0.0, dPi_drho = 0.0, dPi_dz = 0.0;
  for (int k = 0; k <= q; ++k) {
    if (a[k] == 0.0) continue;
    int e = (q - k) / 2; /* (q-k) is even whenever a[k] != 0 */
    Pi += a[k] * ipow(z, k) * ipow(rho, e);
    if (e > 0) dPi_drho += a[k] * ipow(z, k) * e * ipow(rho, e - 1);
    if (k > 0) dPi_dz += a[k] * k * ipow(z, k - 1) * ipow(rho, e);
  }
  double N = (m == 0) ? orc_K(l, 0) : (((am & 1) ? -1.0 : 1.0) * sqrt(2.0) * orc_K(l, m));
  *S = N * A * Pi;
  dS[0] = N * (Ax * Pi + A * dPi_drho * 2.0 * x);
  dS[1] = N * (Ay * Pi + A * dPi_drho * 2.0 * y);
  dS[2] = N * (A * (dPi_dz + dPi_drho * 2.0 * z));
}

/* ------------------------------------------------------------------ */
/* basis                                                                */
/* ------------------------------------------------------------------ */

typedef struct {
  int n_atoms;
  const double* xyz;        /* [n_atoms][3] Bohr */
  const int* species;       /* [n_atoms] */
  int n_species;
  const int* n_rad;         /* [n_species] radial functions per species */
  const int* rad_l;         /* [sum n_rad] species-major */
  const double* rad_alpha;  /* [sum n_rad] */
  int n_log;
  double r_min, r_c, r_on;
  const double* tab_u;      /* [sum n_rad][n_log] knot values (spline mode) */
  const double* tab_M;      /* [sum n_rad][n_log] second derivatives */
  int analytic;             /* 1: u = r^(l+1) exp(-alpha r^2), no cutoff (closed-form pins) */
  const double* lattice;    /* [3][3] lattice vectors as rows (periodic cell), NULL for a molecule */
  int n_shell;              /* periodic images T in [-n_shell, n_shell]^3 */
} orc_basis;

/* ------------------------------------------------------------------ */
/* centres: the atoms and, in a periodic cell, their images (Eqs. 24-25) */
/* ------------------------------------------------------------------ */
/* Centre c = cell * n_atoms + A, cells in lexicographic order of
 * T = (t1, t2, t3) in [-s, s]^3 (s = n_shell; s = 0 for a molecule), at
 * R_A + t1 a1 + t2 a2 + t3 a3. */
static int orc_cell_side(const double* lattice, int n_shell) { return lattice ? 2 * n_shell + 1 : 1; }

static void orc_cell_T(int side, int cell, int T[3]) {
  int s = side / 2;
  T[0] = cell / (side * side) - s;
  T[1] = (cell / side) % side - s;
  T[2] = cell % side - s;
}

static void orc_shift(const double* lattice, const int T[3], double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (!lattice) return;
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) out[d] += T[k] * lattice[3 * k + d];
}

/* positions of all centres: out [side^3 * n_atoms][3]; returns their number */
static int orc_centres(int n_atoms, const double* xyz, const double* lattice, int n_shell, double** out) {
  int side = orc_cell_side(lattice, n_shell), nc = side * side * side * n_atoms;
  double* c = (double*)malloc(sizeof(double) * 3 * (size_t)nc);
  for (int cell = 0; cell < side * side * side; ++cell) {
    int T[3];
    double sh[3];
    orc_cell_T(side, cell, T);
    orc_shift(lattice, T, sh);
    for (int A = 0; A < n_atoms; ++A)
      for (int d = 0; d < 3; ++d) c[3 * ((size_t)cell * n_atoms + A) + d] = xyz[3 * A + d] + sh[d];
  }
  *out = c;
  return nc;
}

/* Function table: atom a, radial k of its species, m = -l..l (radial-major). */
int orc_count_functions(const orc_basis* b) {
  int n = 0;
  for (int a = 0; a < b->n_atoms; ++a) {
    int s = b->species[a], off = 0;
    for (int t = 0; t < s; ++t) off += b->n_rad[t];
    for (int k = 0; k < b->n_rad[s]; ++k) n += 2 * b->rad_l[off + k] + 1;
  }
  return n;
}
void orc_function_table(const orc_basis* b, int* fn_atom, int* fn_rad, int* fn_l, int* fn_m) {
  int n = 0;
  for (int a = 0; a < b->n_atoms; ++a) {
    int s = b->species[a], off = 0;
    for (int t = 0; t < s; ++t) off += b->n_rad[t];
    for (int k = 0; k < b->n_rad[s]; ++k) {
      int l = b->rad_l[off + k];
      for (int m = -l; m <= l; ++m) {
        fn_atom[n] = a; fn_rad[n] = off + k; fn_l[n] = l; fn_m[n] = m; ++n;
      }
    }
  }
}

/* g(r) = u(r)/r^(l+1) and g'(r) */
static void radial_g(const orc_basis* b, int rad, int l, double r, double* g, double* gp) {
  if (b->analytic) {
    if (r >= b->r_c) { *g = 0.0; *gp = 0.0; return; }
    double al = b->rad_alpha[rad];
    double e = exp(-al * r * r);
    *g = e;
    *gp = -2.0 * al * r * e;
    return;
  }
  if (r >= b->r_c) { *g = 0.0; *gp = 0.0; return; }
  const double* u = b->tab_u + (size_t)rad * b->n_log;
  const double* M = b->tab_M + (size_t)rad * b->n_log;
  if (r < b->r_min) { /* u = u_0 (r/r_min)^(l+1): g constant */
    *g = u[0] / ipow(b->r_min, l + 1);
    *gp = 0.0;
    return;
  }
  double uv, du;
  orc_spline_eval(l, b->n_log, b->r_min, b->r_c, u, M, r, &uv, &du);
  double rl1 = ipow(r, l + 1);
  *g = uv / rl1;
  *gp = (du - (l + 1) * uv / r) / rl1;
}

/* phi_i and grad phi_i at point p for the function centred at atom position c */
static void phi_at(const orc_basis* b, int rad, int l, int m, const double c[3], const double p[3],
                   double* phi, double grad[3]) {
  double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (r >= b->r_c) { *phi = 0.0; grad[0] = grad[1] = grad[2] = 0.0; return; }
  double g, gp, S, dS[3];
  radial_g(b, rad, l, r, &g, &gp);
  orc_solid_harmonic(l, m, d[0], d[1], d[2], &S, dS);
  *phi = g * S;
  for (int k = 0; k < 3; ++k) grad[k] = (r > 0.0 ? gp * d[k] / r * S : 0.0) + g * dS[k];
}

/* evaluate one basis function (global index, centred in the 0-cell) at points */
void orc_basis_eval(const orc_basis* b, int n_pts, const double* xyz, int n_fn, const int* fns,
                    double* phi, double* grad) {
  int nf = orc_count_functions(b);
  int* fa = (int*)malloc(sizeof(int) * nf);
  int* fr = (int*)malloc(sizeof(int) * nf);
  int* fl = (int*)malloc(sizeof(int) * nf);
  int* fm = (int*)malloc(sizeof(int) * nf);
  orc_function_table(b, fa, fr, fl, fm);
  for (int q = 0; q < n_fn; ++q) {
    int i = fns[q];
    for (int p = 0; p < n_pts; ++p) {
      phi_at(b, fr[i], fl[i], fm[i], b->xyz + 3 * fa[i], xyz + 3 * (size_t)p,
             &phi[(size_t)q * n_pts + p], &grad[((size_t)q * n_pts + p) * 3]);
    }
  }
  free(fa); free(fr); free(fl); free(fm);
}

/* ------------------------------------------------------------------ */
/* integration grid and Becke partition                                 */
/* ------------------------------------------------------------------ */

static double becke_s(double mu) {
  double f = mu;
  for (int k = 0; k < 3; ++k) f = 1.5 * f - 0.5 * f * f * f;
  return 0.5 * (1.0 - f);
}

/* Stratmann, Scuseria and Frisch (1996) cell function, without size
 * adjustment: s(mu) = (1 - g(mu))/2 with the odd degree-7 polynomial
 * g(x) = (35 x - 35 x^3 + 21 x^5 - 5 x^7)/16 of x = mu/a, a = 0.64, on
 * |mu| <= a, and g = -1 below, +1 above (so s is exactly 1 near its own
 * centre and 0 near the other). */
static double stratmann_s(double mu) {
  const double a = 0.64;
  if (mu <= -a) return 1.0;
  if (mu >= a) return 0.0;
  const double x = mu / a, x2 = x * x;
  const double g = x * (35.0 - x2 * (35.0 - x2 * (21.0 - 5.0 * x2))) / 16.0;
  return 0.5 * (1.0 - g);
}

/* Partition weight p_owner(r) over the neighbour set N(r) = {B : |r - R_B| < r_nb},
 * scheme 0 Becke's cell function, 1 Stratmann's.
 * centres: [n_c][3] (atoms, and periodic images if any). */
double orc_partition_weight(int n_c, const double* centres, int owner, const double p[3], double r_nb,
                            int scheme) {
  if (owner < 0 || owner >= n_c) return 0.0;
  double* dist = (double*)malloc(sizeof(double) * n_c);
  int* in = (int*)calloc(n_c, sizeof(int));
  for (int B = 0; B < n_c; ++B) {
    double dx = p[0] - centres[3 * B], dy = p[1] - centres[3 * B + 1], dz = p[2] - centres[3 * B + 2];
    dist[B] = sqrt(dx * dx + dy * dy + dz * dz);
    in[B] = dist[B] < r_nb;
  }
  double result = 0.0;
  if (in[owner]) {
    double sum = 0.0, Pown = 0.0;
    for (int A = 0; A < n_c; ++A) {
      if (!in[A]) continue;
      double PA = 1.0;
      for (int B = 0; B < n_c; ++B) {
        if (B == A || !in[B]) continue;
        double dx = centres[3 * A] - centres[3 * B], dy = centres[3 * A + 1] - centres[3 * B + 1],
               dz = centres[3 * A + 2] - centres[3 * B + 2];
        double RAB = sqrt(dx * dx + dy * dy + dz * dz);
        const double mu = (dist[A] - dist[B]) / RAB;
        PA *= scheme == 1 ? stratmann_s(mu) : becke_s(mu);
      }
      sum += PA;
      if (A == owner) Pown = PA;
    }
    result = Pown / sum;
  }
  free(dist);
  free(in);
  return result;
}

double orc_becke_weight(int n_c, const double* centres, int owner, const double p[3], double r_nb) {
  return orc_partition_weight(n_c, centres, owner, p, r_nb, 0);
}

/* Raw grid of every (0-cell) atom, partition weights, pruning.
 * Raw point id = ((atom*n_rad + i)*n_theta + a)*n_phi + b; i radial shell
 * (i = 1..N of x_i = cos(i pi/(N+1)), so decreasing r), a Gauss-Legendre node in cos(theta)
 * (ascending), b azimuth phi_b = (b + 1/2) 2 pi / n_phi.
 * The Becke partition runs over all centres (atoms and, in a periodic cell,
 * their images) within r_nb; the owner is the generating atom in cell 0.
 * Keep p iff some centre lies strictly within r_c of p and w_p != 0.
 * stride > 1 keeps only raw ids divisible by stride (a uniform sample used
 * to time the oracle on a bounded share of a large workload).
 * Returns the number of kept points; out arrays must hold the raw count. */
long orc_grid_cell(int n_atoms, const double* xyz, const double* lattice, int n_shell, int n_rad, double R,
                   int n_theta, int n_phi, double r_c, double r_nb, int scheme, long long stride,
                   double* out_xyz, double* out_w, long long* out_id) {
  double* rr = (double*)malloc(sizeof(double) * n_rad);
  double* wr = (double*)malloc(sizeof(double) * n_rad);
  double* ct = (double*)malloc(sizeof(double) * n_theta);
  double* wt = (double*)malloc(sizeof(double) * n_theta);
  orc_radial_shells(n_rad, R, rr, wr);
  orc_gauss_legendre(n_theta, ct, wt);
  double* cen = NULL;
  int side = orc_cell_side(lattice, n_shell);
  int nc = orc_centres(n_atoms, xyz, lattice, n_shell, &cen);
  int cell0 = (side * side * side - 1) / 2; /* T = (0, 0, 0) */
  double* nbr = (double*)malloc(sizeof(double) * 3 * (size_t)nc);
  long kept = 0;
  for (int A = 0; A < n_atoms; ++A) {
    for (int i = 0; i < n_rad; ++i) {
      for (int a = 0; a < n_theta; ++a) {
        double st = sqrt(1.0 - ct[a] * ct[a]);
        for (int bb = 0; bb < n_phi; ++bb) {
          long long id = (((long long)A * n_rad + i) * n_theta + a) * n_phi + bb;
          if (stride > 1 && id % stride != 0) continue; /* uniform sample of the raw grid */
          double ph = (bb + 0.5) * 2.0 * M_PI / n_phi;
          double p[3] = {xyz[3 * A] + rr[i] * st * cos(ph), xyz[3 * A + 1] + rr[i] * st * sin(ph),
                         xyz[3 * A + 2] + rr[i] * ct[a]};
          int near = 0;
          for (int B = 0; B < nc && !near; ++B) {
            double dx = p[0] - cen[3 * B], dy = p[1] - cen[3 * B + 1], dz = p[2] - cen[3 * B + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < r_c) near = 1;
          }
          if (!near) continue;
          /* the weight depends only on the centres within r_nb of p, in
           * ascending order: it is taken over exactly that list */
          int nn = 0, own_n = -1;
          for (int B = 0; B < nc; ++B) {
            double dx = p[0] - cen[3 * B], dy = p[1] - cen[3 * B + 1], dz = p[2] - cen[3 * B + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < r_nb) {
              if (B == cell0 * n_atoms + A) own_n = nn;
              for (int d = 0; d < 3; ++d) nbr[3 * nn + d] = cen[3 * B + d];
              ++nn;
            }
          }
          if (own_n < 0) continue; /* the owner is not a neighbour: weight 0 */
          double w = wr[i] * wt[a] * (2.0 * M_PI / n_phi) * orc_partition_weight(nn, nbr, own_n, p, r_nb, scheme);
          if (w == 0.0) continue;
          out_xyz[3 * kept] = p[0]; out_xyz[3 * kept + 1] = p[1]; out_xyz[3 * kept + 2] = p[2];
          out_w[kept] = w;
          out_id[kept] = id;
          ++kept;
        }
      }
    }
  }
  free(rr); free(wr); free(ct); free(wt); free(cen); free(nbr);
  return kept;
}

/* The kept points of orc_grid_cell (stride 1) that lie within r_c of at
 * least one of n_t target positions, with the same weights and raw ids, in
 * raw id order.  They are found on two restricted sets, both exact: a kept
 * point lies within r_nb of its generating atom (the partition weight is 0
 * otherwise), so only atoms within r_c + r_nb of a target generate one; and
 * every centre within r_nb of such a point lies within r_c + r_nb of that
 * target.  The partition weight depends only on the centres within r_nb of
 * the point, in ascending order, so it is taken over exactly that list
 * (the same neighbour set in the same order as over the full list).
 * Returns the number of points (at most max_out are written), or -1 if a
 * target is farther than r_c from every centre (it would keep nothing). */
long orc_grid_near(int n_atoms, const double* xyz, const double* lattice, int n_shell, int n_rad, double R,
                   int n_theta, int n_phi, double r_c, double r_nb, int scheme, int n_t, const double* targets,
                   long max_out, double* out_xyz, double* out_w, long long* out_id) {
  double* rr = (double*)malloc(sizeof(double) * n_rad);
  double* wr = (double*)malloc(sizeof(double) * n_rad);
  double* ct = (double*)malloc(sizeof(double) * n_theta);
  double* wt = (double*)malloc(sizeof(double) * n_theta);
  orc_radial_shells(n_rad, R, rr, wr);
  orc_gauss_legendre(n_theta, ct, wt);
  double* cen = NULL;
  int side = orc_cell_side(lattice, n_shell);
  int nc = orc_centres(n_atoms, xyz, lattice, n_shell, &cen);
  int cell0 = (side * side * side - 1) / 2;
  /* centres within r_c + r_nb of some target, ascending */
  double* sub = (double*)malloc(sizeof(double) * 3 * (size_t)nc);
  int* sub_id = (int*)malloc(sizeof(int) * nc);
  int ns = 0;
  for (int c = 0; c < nc; ++c) {
    for (int t = 0; t < n_t; ++t) {
      double dx = cen[3 * c] - targets[3 * t], dy = cen[3 * c + 1] - targets[3 * t + 1],
             dz = cen[3 * c + 2] - targets[3 * t + 2];
      if (sqrt(dx * dx + dy * dy + dz * dz) < r_c + r_nb) {
        for (int d = 0; d < 3; ++d) sub[3 * ns + d] = cen[3 * c + d];
        sub_id[ns++] = c;
        break;
      }
    }
  }
  double* nbr = (double*)malloc(sizeof(double) * 3 * (size_t)(ns > 0 ? ns : 1));
  long kept = 0;
  for (int A = 0; A < n_atoms; ++A) {
    int own = -1; /* the generating atom (cell 0) in the restricted list */
    for (int k = 0; k < ns; ++k)
      if (sub_id[k] == cell0 * n_atoms + A) own = k;
    if (own < 0) continue; /* farther than r_c + r_nb from every target */
    for (int i = 0; i < n_rad; ++i) {
      for (int a = 0; a < n_theta; ++a) {
        double st = sqrt(1.0 - ct[a] * ct[a]);
        for (int bb = 0; bb < n_phi; ++bb) {
          long long id = (((long long)A * n_rad + i) * n_theta + a) * n_phi + bb;
          double ph = (bb + 0.5) * 2.0 * M_PI / n_phi;
          double p[3] = {xyz[3 * A] + rr[i] * st * cos(ph), xyz[3 * A + 1] + rr[i] * st * sin(ph),
                         xyz[3 * A + 2] + rr[i] * ct[a]};
          int close = 0;
          for (int t = 0; t < n_t && !close; ++t) {
            double dx = p[0] - targets[3 * t], dy = p[1] - targets[3 * t + 1], dz = p[2] - targets[3 * t + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < r_c) close = 1;
          }
          if (!close) continue;
          int near = 0;
          for (int B = 0; B < ns && !near; ++B) {
            double dx = p[0] - sub[3 * B], dy = p[1] - sub[3 * B + 1], dz = p[2] - sub[3 * B + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < r_c) near = 1;
          }
          if (!near) continue;
          /* the centres within r_nb of p, ascending, and the owner among them */
          int nn = 0, own_n = -1;
          for (int B = 0; B < ns; ++B) {
            double dx = p[0] - sub[3 * B], dy = p[1] - sub[3 * B + 1], dz = p[2] - sub[3 * B + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < r_nb) {
              if (B == own) own_n = nn;
              for (int d = 0; d < 3; ++d) nbr[3 * nn + d] = sub[3 * B + d];
              ++nn;
            }
          }
          if (own_n < 0) continue; /* the owner is not a neighbour: weight 0 */
          double w = wr[i] * wt[a] * (2.0 * M_PI / n_phi) * orc_partition_weight(nn, nbr, own_n, p, r_nb, scheme);
          if (w == 0.0) continue;
          if (kept < max_out) {
            out_xyz[3 * kept] = p[0]; out_xyz[3 * kept + 1] = p[1]; out_xyz[3 * kept + 2] = p[2];
            out_w[kept] = w;
            out_id[kept] = id;
          }
          ++kept;
        }
      }
    }
  }
  free(rr); free(wr); free(ct); free(wt); free(cen); free(sub); free(sub_id); free(nbr);
  return kept;
}

/* the molecular grid (no lattice) */
long orc_grid(int n_atoms, const double* xyz, int n_rad, double R, int n_theta, int n_phi,
              double r_c, double r_nb, long long stride, double* out_xyz, double* out_w, long long* out_id) {
  return orc_grid_cell(n_atoms, xyz, NULL, 0, n_rad, R, n_theta, n_phi, r_c, r_nb, 0, stride, out_xyz, out_w,
                       out_id);
}

/* ------------------------------------------------------------------ */
/* block pattern (molecule): block (A,B) iff |R_A - R_B| < 2 r_c         */
/* CSR over atom rows; blocks dense row-major nf_A x nf_B                */
/* ------------------------------------------------------------------ */
static int species_nfn(const orc_basis* b, int s) {
  int off = 0, n = 0;
  for (int t = 0; t < s; ++t) off += b->n_rad[t];
  for (int k = 0; k < b->n_rad[s]; ++k) n += 2 * b->rad_l[off + k] + 1;
  return n;
}

/* Block (A, B, T) exists iff |R_A - R_B - T.L| < 2 r_c (strict), T an
 * integer lattice triple in [-2s, 2s]^3 (T = 0 for a molecule): the real-space
 * H(T) blocks <phi_(A,0)| . |phi_(B,T)> (Eqs. 24-25).  Rows A, then B, then T
 * lexicographic.  Returns the number of blocks; if blk_ptr != NULL fills CSR
 * (blk_ptr[n_atoms+1], blk_col[nb], blk_T[nb][3] if not NULL, blk_off[nb+1]). */
long orc_pattern(const orc_basis* b, long long* blk_ptr, int* blk_col, int* blk_T, long long* blk_off) {
  long nb = 0;
  long long off = 0;
  int s2 = b->lattice ? 2 * b->n_shell : 0, side = 2 * s2 + 1;
  if (blk_ptr) blk_ptr[0] = 0;
  for (int A = 0; A < b->n_atoms; ++A) {
    for (int B = 0; B < b->n_atoms; ++B) {
      for (int cell = 0; cell < side * side * side; ++cell) {
        int T[3];
        double sh[3];
        orc_cell_T(side, cell, T);
        orc_shift(b->lattice, T, sh);
        double dx = b->xyz[3 * A] - b->xyz[3 * B] - sh[0], dy = b->xyz[3 * A + 1] - b->xyz[3 * B + 1] - sh[1],
               dz = b->xyz[3 * A + 2] - b->xyz[3 * B + 2] - sh[2];
        if (sqrt(dx * dx + dy * dy + dz * dz) < 2.0 * b->r_c) {
          if (blk_col) {
            blk_col[nb] = B;
            blk_off[nb] = off;
            if (blk_T) { blk_T[3 * nb] = T[0]; blk_T[3 * nb + 1] = T[1]; blk_T[3 * nb + 2] = T[2]; }
          }
          off += (long long)species_nfn(b, b->species[A]) * species_nfn(b, b->species[B]);
          ++nb;
        }
      }
    }
    if (blk_ptr) blk_ptr[A + 1] = nb;
  }
  if (blk_off) blk_off[nb] = off;
  return nb;
}

/* ------------------------------------------------------------------ */
/* per-point evaluation of all functions (zero where inactive)          */
/* ------------------------------------------------------------------ */
typedef struct {
  int nf;
  int *fa, *fr, *fl, *fm, *afirst; /* afirst[atom] = first function index */
} ftab;

static void ftab_init(const orc_basis* b, ftab* t) {
  t->nf = orc_count_functions(b);
  t->fa = (int*)malloc(sizeof(int) * (t->nf + 1));
  t->fr = (int*)malloc(sizeof(int) * (t->nf + 1));
  t->fl = (int*)malloc(sizeof(int) * (t->nf + 1));
  t->fm = (int*)malloc(sizeof(int) * (t->nf + 1));
  t->afirst = (int*)malloc(sizeof(int) * (b->n_atoms + 1));
  orc_function_table(b, t->fa, t->fr, t->fl, t->fm);
  int i = 0;
  for (int a = 0; a <= b->n_atoms; ++a) {
    while (i < t->nf && t->fa[i] < a) ++i;
    t->afirst[a] = i;
  }
}
static void ftab_free(ftab* t) { free(t->fa); free(t->fr); free(t->fl); free(t->fm); free(t->afirst); }


/* ------------------------------------------------------------------ */
/* matrix elements                                                      */
/* ------------------------------------------------------------------ */

/* Listed pairs (global function indices): out arrays [n_pairs]. */
void orc_matrix_pairs(const orc_basis* b, long n_pts, const double* xyz, const double* w, const double* v,
                      long n_pairs, const int* pi, const int* pj,
                      double* V, double* W0, double* SOx, double* SOy, double* SOz) {
  ftab t;
  ftab_init(b, &t);
  /* unique functions touched */
  int* used = (int*)calloc(t.nf, sizeof(int));
  for (long q = 0; q < n_pairs; ++q) { used[pi[q]] = 1; used[pj[q]] = 1; }
  int nu = 0;
  int* list = (int*)malloc(sizeof(int) * t.nf);
  for (int i = 0; i < t.nf; ++i) if (used[i]) list[nu++] = i;
  double* phi = (double*)calloc(t.nf, sizeof(double));
  double* grad = (double*)calloc(3 * (size_t)t.nf, sizeof(double));
  orc_acc* acc = (orc_acc*)calloc(5 * (size_t)n_pairs, sizeof(orc_acc));
  for (long p = 0; p < n_pts; ++p) {
    const double* P = xyz + 3 * p;
    for (int q = 0; q < nu; ++q) {
      int i = list[q];
      phi_at(b, t.fr[i], t.fl[i], t.fm[i], b->xyz + 3 * t.fa[i], P, &phi[i], &grad[3 * i]);
    }
    double wv = w[p] * v[p];
    for (long q = 0; q < n_pairs; ++q) {
      int i = pi[q], j = pj[q];
      const double* a = &grad[3 * i];
      const double* c = &grad[3 * j];
      acc_add(&acc[5 * q + 0], wv * (phi[i] * phi[j]));
      acc_add(&acc[5 * q + 1], wv * (a[0] * c[0] + a[1] * c[1] + a[2] * c[2]));
      acc_add(&acc[5 * q + 2], wv * (a[1] * c[2] - a[2] * c[1]));
      acc_add(&acc[5 * q + 3], wv * (a[2] * c[0] - a[0] * c[2]));
      acc_add(&acc[5 * q + 4], wv * (a[0] * c[1] - a[1] * c[0]));
    }
  }
  for (long q = 0; q < n_pairs; ++q) {
    V[q] = acc_get(&acc[5 * q + 0]);
    W0[q] = acc_get(&acc[5 * q + 1]);
    SOx[q] = acc_get(&acc[5 * q + 2]);
    SOy[q] = acc_get(&acc[5 * q + 3]);
    SOz[q] = acc_get(&acc[5 * q + 4]);
  }
  free(used); free(list); free(phi); free(grad); free(acc);
  ftab_free(&t);
}

/* Listed elements of the block matrices, periodic images included: element
 * q is (i, j) of block (A, B, T) (i, j local function indices of atoms A
 * and B, T = ET[3q..3q+2]), the sum over the points and over the cells T_a
 * of the centre set with T_a + T in it of w v times the integrand of
 * phi_i centred at R_A + T_a L and phi_j at R_B + (T_a + T) L (the restricted
 * real-space sum of Eqs. 24-25 with Eqs. 29-30 and the SS reading: what
 * orc_matrix_blocks accumulates into that element). */
void orc_matrix_entries(const orc_basis* b, long n_pts, const double* xyz, const double* w, const double* v,
                        long n_e, const int* EA, const int* EB, const int* ET, const int* Ei, const int* Ej,
                        double* V, double* W0, double* SOx, double* SOy, double* SOz) {
  ftab t;
  ftab_init(b, &t);
  int side = orc_cell_side(b->lattice, b->n_shell), s = side / 2, ncell = side * side * side;
  orc_acc* acc = (orc_acc*)calloc(5 * (size_t)n_e, sizeof(orc_acc));
  /* per point, the cells T_a with R_A + T_a L within r_c of it, for each
   * atom A that heads an element (phi_i vanishes at the other cells) */
  int* close = (int*)malloc(sizeof(int) * (size_t)b->n_atoms * ncell);
  int* nclose = (int*)calloc(b->n_atoms, sizeof(int));
  int* is_row = (int*)calloc(b->n_atoms, sizeof(int));
  for (long q = 0; q < n_e; ++q) is_row[EA[q]] = 1;
  for (long p = 0; p < n_pts; ++p) {
    const double* P = xyz + 3 * p;
    double wv = w[p] * v[p];
    for (int A = 0; A < b->n_atoms; ++A) {
      if (!is_row[A]) continue;
      nclose[A] = 0;
      for (int cell = 0; cell < ncell; ++cell) {
        int Ta[3];
        double sa[3];
        orc_cell_T(side, cell, Ta);
        orc_shift(b->lattice, Ta, sa);
        double dx = P[0] - (b->xyz[3 * A] + sa[0]), dy = P[1] - (b->xyz[3 * A + 1] + sa[1]),
               dz = P[2] - (b->xyz[3 * A + 2] + sa[2]);
        if (sqrt(dx * dx + dy * dy + dz * dz) < b->r_c) close[(size_t)A * ncell + nclose[A]++] = cell;
      }
    }
    for (long q = 0; q < n_e; ++q) {
      int A = EA[q], B = EB[q];
      int i = t.afirst[A] + Ei[q], j = t.afirst[B] + Ej[q];
      for (int k = 0; k < nclose[A]; ++k) {
        const int cell = close[(size_t)A * ncell + k];
        int Ta[3], Tb[3];
        orc_cell_T(side, cell, Ta);
        int inside = 1;
        for (int k = 0; k < 3; ++k) {
          Tb[k] = Ta[k] + ET[3 * q + k];
          if (Tb[k] < -s || Tb[k] > s) inside = 0;
        }
        if (!inside) continue;
        double sa[3], sb[3], ca[3], cb[3];
        orc_shift(b->lattice, Ta, sa);
        orc_shift(b->lattice, Tb, sb);
        for (int d = 0; d < 3; ++d) {
          ca[d] = b->xyz[3 * A + d] + sa[d];
          cb[d] = b->xyz[3 * B + d] + sb[d];
        }
        double pi, pj, gi[3], gj[3];
        phi_at(b, t.fr[i], t.fl[i], t.fm[i], ca, P, &pi, gi);
        phi_at(b, t.fr[j], t.fl[j], t.fm[j], cb, P, &pj, gj);
        acc_add(&acc[5 * q + 0], wv * (pi * pj));
        acc_add(&acc[5 * q + 1], wv * (gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2]));
        acc_add(&acc[5 * q + 2], wv * (gi[1] * gj[2] - gi[2] * gj[1]));
        acc_add(&acc[5 * q + 3], wv * (gi[2] * gj[0] - gi[0] * gj[2]));
        acc_add(&acc[5 * q + 4], wv * (gi[0] * gj[1] - gi[1] * gj[0]));
      }
    }
  }
  for (long q = 0; q < n_e; ++q) {
    V[q] = acc_get(&acc[5 * q + 0]);
    W0[q] = acc_get(&acc[5 * q + 1]);
    SOx[q] = acc_get(&acc[5 * q + 2]);
    SOy[q] = acc_get(&acc[5 * q + 3]);
    SOz[q] = acc_get(&acc[5 * q + 4]);
  }
  free(acc); free(close); free(nclose); free(is_row);
  ftab_free(&t);
}

/* locate block (A, B, T) in the CSR pattern, -1 if absent (blk_T NULL: all T = 0) */
static long find_block(const long long* blk_ptr, const int* blk_col, const int* blk_T, int A, int B,
                       const int T[3]) {
  for (long long q = blk_ptr[A]; q < blk_ptr[A + 1]; ++q) {
    if (blk_col[q] != B) continue;
    if (!blk_T) {
      if (T[0] == 0 && T[1] == 0 && T[2] == 0) return (long)q;
      continue;
    }
    if (blk_T[3 * q] == T[0] && blk_T[3 * q + 1] == T[1] && blk_T[3 * q + 2] == T[2]) return (long)q;
  }
  return -1;
}

/* centres within r_c of X: their indices, atoms and cells; the values and
 * gradients of their functions at X (phi[slot*nmax + k], grad[3*(...)]) */
typedef struct {
  int n, nc, side, nmax;
  double* cen;
  int *c, *atom, *cell;
  double *phi, *grad;
} orc_active;

static void active_init(const orc_basis* b, orc_active* a) {
  a->side = orc_cell_side(b->lattice, b->n_shell);
  a->nc = orc_centres(b->n_atoms, b->xyz, b->lattice, b->n_shell, &a->cen);
  a->nmax = 0;
  for (int A = 0; A < b->n_atoms; ++A) {
    int nf = species_nfn(b, b->species[A]);
    if (nf > a->nmax) a->nmax = nf;
  }
  a->c = (int*)malloc(sizeof(int) * a->nc);
  a->atom = (int*)malloc(sizeof(int) * a->nc);
  a->cell = (int*)malloc(sizeof(int) * a->nc);
  a->phi = (double*)calloc((size_t)a->nc * a->nmax, sizeof(double));
  a->grad = (double*)calloc(3 * (size_t)a->nc * a->nmax, sizeof(double));
}
static void active_free(orc_active* a) {
  free(a->cen); free(a->c); free(a->atom); free(a->cell); free(a->phi); free(a->grad);
}

static void active_at(const orc_basis* b, const ftab* t, orc_active* a, const double X[3]) {
  a->n = 0;
  for (int c = 0; c < a->nc; ++c) {
    double dx = X[0] - a->cen[3 * c], dy = X[1] - a->cen[3 * c + 1], dz = X[2] - a->cen[3 * c + 2];
    if (sqrt(dx * dx + dy * dy + dz * dz) >= b->r_c) continue;
    int A = c % b->n_atoms, s = a->n++;
    a->c[s] = c; a->atom[s] = A; a->cell[s] = c / b->n_atoms;
    for (int i = t->afirst[A]; i < t->afirst[A + 1]; ++i) {
      int k = i - t->afirst[A];
      phi_at(b, t->fr[i], t->fl[i], t->fm[i], a->cen + 3 * c, X, &a->phi[(size_t)s * a->nmax + k],
             &a->grad[3 * ((size_t)s * a->nmax + k)]);
    }
  }
}

/* block of the centre pair (slot sa, slot sb): (A, B, T_b - T_a) */
static long pair_block(const orc_active* a, int sa, int sb, const long long* blk_ptr, const int* blk_col,
                       const int* blk_T) {
  int Ta[3], Tb[3], T[3];
  orc_cell_T(a->side, a->cell[sa], Ta);
  orc_cell_T(a->side, a->cell[sb], Tb);
  for (int k = 0; k < 3; ++k) T[k] = Tb[k] - Ta[k];
  return find_block(blk_ptr, blk_col, blk_T, a->atom[sa], a->atom[sb], T);
}

/* Full matrices on the block pattern (Eqs. 29-30 with F = v and the SS
 * reading): outputs [blk_off[nb]] each.  Every pair of centres active at a
 * point adds into its block (A, B, T_b - T_a) (the restricted real-space sum
 * of Eqs. 24-25; one block (A, B, 0) per pair for a molecule). */
int orc_matrix_blocks(const orc_basis* b, long n_pts, const double* xyz, const double* w, const double* v,
                      const long long* blk_ptr, const int* blk_col, const int* blk_T, const long long* blk_off,
                      double* V, double* W0, double* SOx, double* SOy, double* SOz) {
  ftab t;
  ftab_init(b, &t);
  orc_active a;
  active_init(b, &a);
  long long nnz = blk_off[blk_ptr[b->n_atoms]];
  orc_acc* acc = (orc_acc*)calloc(5 * (size_t)nnz, sizeof(orc_acc));
  int missing = 0;
  for (long p = 0; p < n_pts; ++p) {
    active_at(b, &t, &a, xyz + 3 * p);
    double wv = w[p] * v[p];
    for (int sa = 0; sa < a.n; ++sa) {
      for (int sb = 0; sb < a.n; ++sb) {
        long q = pair_block(&a, sa, sb, blk_ptr, blk_col, blk_T);
        if (q < 0) { missing = 1; continue; }
        int nfA = species_nfn(b, b->species[a.atom[sa]]), nfB = species_nfn(b, b->species[a.atom[sb]]);
        for (int i = 0; i < nfA; ++i) {
          for (int j = 0; j < nfB; ++j) {
            long long e = blk_off[q] + (long long)i * nfB + j;
            double pi = a.phi[(size_t)sa * a.nmax + i], pj = a.phi[(size_t)sb * a.nmax + j];
            const double* gi = &a.grad[3 * ((size_t)sa * a.nmax + i)];
            const double* gj = &a.grad[3 * ((size_t)sb * a.nmax + j)];
            acc_add(&acc[5 * e + 0], wv * (pi * pj));
            acc_add(&acc[5 * e + 1], wv * (gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2]));
            acc_add(&acc[5 * e + 2], wv * (gi[1] * gj[2] - gi[2] * gj[1]));
            acc_add(&acc[5 * e + 3], wv * (gi[2] * gj[0] - gi[0] * gj[2]));
            acc_add(&acc[5 * e + 4], wv * (gi[0] * gj[1] - gi[1] * gj[0]));
          }
        }
      }
    }
  }
  for (long long e = 0; e < nnz; ++e) {
    V[e] = acc_get(&acc[5 * e + 0]);
    W0[e] = acc_get(&acc[5 * e + 1]);
    SOx[e] = acc_get(&acc[5 * e + 2]);
    SOy[e] = acc_get(&acc[5 * e + 3]);
    SOz[e] = acc_get(&acc[5 * e + 4]);
  }
  free(acc);
  active_free(&a);
  ftab_free(&t);
  return missing;
}

/* The per-column operator of Eq. 19 (large component, scalar form):
 *   F_ij = sum_p w_p phi_i(p) [eps_j - V_j(|p - R_j|) + v_p] phi_j(p)
 * with eps_j and V_j those of the radial function of column function j
 * (eps[rad], knots[rad][n_log]: V at the log knots r_k of the radial
 * tables; natural cubic spline in the knot index, the first knot's value
 * below r_min, the last one's from r_c on, where phi_j vanishes anyway) and
 * R_j the centre of j.  Not symmetric.  Output F[blk_off[nb]]. */
void orc_matrix_columns(const orc_basis* b, long n_pts, const double* xyz, const double* w, const double* v,
                        const double* eps, const double* knots, const long long* blk_ptr, const int* blk_col,
                        const int* blk_T, const long long* blk_off, double* F) {
  ftab t;
  ftab_init(b, &t);
  orc_active a;
  active_init(b, &a);
  int n_rad_tot = 0;
  for (int s = 0; s < b->n_species; ++s) n_rad_tot += b->n_rad[s];
  const int n = b->n_log;
  double* M = (double*)malloc(sizeof(double) * (size_t)n_rad_tot * n);
  for (int k = 0; k < n_rad_tot; ++k) orc_natural_M(n, knots + (size_t)k * n, M + (size_t)k * n);
  const double h = log(b->r_c / b->r_min) / (n - 1);
  long long nnz = blk_off[blk_ptr[b->n_atoms]];
  orc_acc* acc = (orc_acc*)calloc((size_t)nnz, sizeof(orc_acc));
  double* col = (double*)malloc(sizeof(double) * (size_t)a.nmax);
  for (long p = 0; p < n_pts; ++p) {
    const double* X = xyz + 3 * p;
    active_at(b, &t, &a, X);
    for (int sb = 0; sb < a.n; ++sb) {
      int B = a.atom[sb], nfB = species_nfn(b, b->species[B]);
      const double* cB = a.cen + 3 * a.c[sb];
      double dx = X[0] - cB[0], dy = X[1] - cB[1], dz = X[2] - cB[2];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      /* the column factor w (eps_j - V_j(r) + v) phi_j of every function of centre sb */
      for (int j = 0; j < nfB; ++j) {
        int rad = t.fr[t.afirst[B] + j];
        const double* u = knots + (size_t)rad * n;
        const double* Mk = M + (size_t)rad * n;
        double Vr;
        if (r < b->r_min) {
          Vr = u[0];
        } else if (r >= b->r_c) {
          Vr = u[n - 1];
        } else {
          double tt = log(r / b->r_min) / h;
          int k = (int)floor(tt);
          if (k > n - 2) k = n - 2;
          if (k < 0) k = 0;
          double s = tt - k, q = 1.0 - s;
          Vr = q * u[k] + s * u[k + 1] + (q * q * q - q) * Mk[k] / 6.0 + (s * s * s - s) * Mk[k + 1] / 6.0;
        }
        col[j] = w[p] * (eps[rad] - Vr + v[p]) * a.phi[(size_t)sb * a.nmax + j];
      }
      for (int sa = 0; sa < a.n; ++sa) {
        long q = pair_block(&a, sa, sb, blk_ptr, blk_col, blk_T);
        if (q < 0) continue;
        int nfA = species_nfn(b, b->species[a.atom[sa]]);
        for (int i = 0; i < nfA; ++i) {
          double pi = a.phi[(size_t)sa * a.nmax + i];
          for (int j = 0; j < nfB; ++j) acc_add(&acc[blk_off[q] + (long long)i * nfB + j], pi * col[j]);
        }
      }
    }
  }
  for (long long e = 0; e < nnz; ++e) F[e] = acc_get(&acc[e]);
  free(acc); free(col); free(M);
  active_free(&a);
  ftab_free(&t);
}

/* Density n_p = sum_ij P_ij phi_i phi_j with P on the block pattern (Eq. 39),
 * the pairs of active centres taking P from their block (A, B, T_b - T_a). */
void orc_density(const orc_basis* b, long n_pts, const double* xyz,
                 const long long* blk_ptr, const int* blk_col, const int* blk_T, const long long* blk_off,
                 const double* P, double* n_out) {
  ftab t;
  ftab_init(b, &t);
  orc_active a;
  active_init(b, &a);
  for (long p = 0; p < n_pts; ++p) {
    active_at(b, &t, &a, xyz + 3 * p);
    orc_acc acc = {0.0, 0.0};
    for (int sa = 0; sa < a.n; ++sa) {
      for (int sb = 0; sb < a.n; ++sb) {
        long q = pair_block(&a, sa, sb, blk_ptr, blk_col, blk_T);
        if (q < 0) continue;
        int nfA = species_nfn(b, b->species[a.atom[sa]]), nfB = species_nfn(b, b->species[a.atom[sb]]);
        for (int i = 0; i < nfA; ++i)
          for (int j = 0; j < nfB; ++j)
            acc_add(&acc, P[blk_off[q] + (long long)i * nfB + j] * a.phi[(size_t)sa * a.nmax + i] *
                              a.phi[(size_t)sb * a.nmax + j]);
      }
    }
    n_out[p] = acc_get(&acc);
  }
  active_free(&a);
  ftab_free(&t);
}

/* Adjoint: dL/dv_p = w_p sum_M sum_ij G^M_ij f^M_ij(p), M = V, W0, SOx, SOy, SOz,
 * each G^M on the block pattern (a NULL slot counts as zero). */
void orc_adjoint(const orc_basis* b, long n_pts, const double* xyz, const double* w,
                 const long long* blk_ptr, const int* blk_col, const int* blk_T, const long long* blk_off,
                 const double* GV, const double* GW, const double* Gx, const double* Gy, const double* Gz,
                 double* dLdv) {
  ftab t;
  ftab_init(b, &t);
  orc_active a;
  active_init(b, &a);
  for (long p = 0; p < n_pts; ++p) {
    active_at(b, &t, &a, xyz + 3 * p);
    orc_acc acc = {0.0, 0.0};
    for (int sa = 0; sa < a.n; ++sa) {
      for (int sb = 0; sb < a.n; ++sb) {
        long q = pair_block(&a, sa, sb, blk_ptr, blk_col, blk_T);
        if (q < 0) continue;
        int nfA = species_nfn(b, b->species[a.atom[sa]]), nfB = species_nfn(b, b->species[a.atom[sb]]);
        for (int i = 0; i < nfA; ++i) {
          for (int j = 0; j < nfB; ++j) {
            long long e = blk_off[q] + (long long)i * nfB + j;
            double pi = a.phi[(size_t)sa * a.nmax + i], pj = a.phi[(size_t)sb * a.nmax + j];
            const double* gi = &a.grad[3 * ((size_t)sa * a.nmax + i)];
            const double* gj = &a.grad[3 * ((size_t)sb * a.nmax + j)];
            if (GV) acc_add(&acc, GV[e] * pi * pj);
            if (GW) acc_add(&acc, GW[e] * (gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2]));
            if (Gx) acc_add(&acc, Gx[e] * (gi[1] * gj[2] - gi[2] * gj[1]));
            if (Gy) acc_add(&acc, Gy[e] * (gi[2] * gj[0] - gi[0] * gj[2]));
            if (Gz) acc_add(&acc, Gz[e] * (gi[0] * gj[1] - gi[1] * gj[0]));
          }
        }
      }
    }
    dLdv[p] = w[p] * acc_get(&acc);
  }
  active_free(&a);
  ftab_free(&t);
}

/* k-pattern: the atom pairs (A, B) that have at least one block (A, B, T);
 * returns their number; if kblk_ptr != NULL fills CSR (kblk_ptr[n_atoms+1],
 * kblk_col[], kblk_off[nkb+1]). */
long orc_kpattern(const orc_basis* b, const long long* blk_ptr, const int* blk_col, long long* kblk_ptr,
                  int* kblk_col, long long* kblk_off) {
  long nkb = 0;
  long long off = 0;
  if (kblk_ptr) kblk_ptr[0] = 0;
  for (int A = 0; A < b->n_atoms; ++A) {
    for (int B = 0; B < b->n_atoms; ++B) {
      int present = 0;
      for (long long q = blk_ptr[A]; q < blk_ptr[A + 1] && !present; ++q) present = blk_col[q] == B;
      if (!present) continue;
      if (kblk_col) {
        kblk_col[nkb] = B;
        kblk_off[nkb] = off;
      }
      off += (long long)species_nfn(b, b->species[A]) * species_nfn(b, b->species[B]);
      ++nkb;
    }
    if (kblk_ptr) kblk_ptr[A + 1] = nkb;
  }
  if (kblk_off) kblk_off[nkb] = off;
  return nkb;
}

/* k-phase fold of real-space blocks (Eqs. 24-26): for each k in reduced
 * coordinates (fractions of the reciprocal lattice vectors),
 *   H(k)_AB = sum_T exp(2 pi i k.T) H(T)_AB
 * over the pattern blocks (A, B, T) (blk_T NULL: T = 0).  out: complex
 * interleaved (re, im) [n_k][nnz_k] on the k-pattern. */
void orc_kfold(const orc_basis* b, const long long* blk_ptr, const int* blk_col, const int* blk_T,
               const long long* blk_off, const double* H, int n_k, const double* k, const long long* kblk_ptr,
               const int* kblk_col, const long long* kblk_off, double* out) {
  long long nnz_k = kblk_off[kblk_ptr[b->n_atoms]];
  for (int ik = 0; ik < n_k; ++ik) {
    double* o = out + 2 * (size_t)ik * nnz_k;
    for (long long e = 0; e < 2 * nnz_k; ++e) o[e] = 0.0;
    for (int A = 0; A < b->n_atoms; ++A) {
      int nfA = species_nfn(b, b->species[A]);
      for (long long q = blk_ptr[A]; q < blk_ptr[A + 1]; ++q) {
        int B = blk_col[q], nfB = species_nfn(b, b->species[B]);
        long long kq = -1;
        for (long long r = kblk_ptr[A]; r < kblk_ptr[A + 1]; ++r)
          if (kblk_col[r] == B) kq = r;
        double t = 0.0;
        if (blk_T)
          t = k[3 * ik] * blk_T[3 * q] + k[3 * ik + 1] * blk_T[3 * q + 1] + k[3 * ik + 2] * blk_T[3 * q + 2];
        double c = cos(2.0 * M_PI * t), sn = sin(2.0 * M_PI * t);
        for (long long e = 0; e < (long long)nfA * nfB; ++e) {
          double h = H[blk_off[q] + e];
          o[2 * (kblk_off[kq] + e)] += h * c;
          o[2 * (kblk_off[kq] + e) + 1] += h * sn;
        }
      }
    }
  }
}

/* Spinor SS block assembly (Eq. 16 with the kinetic-balance reading):
 * each scalar element (i,j) becomes the 2x2 complex block
 *   [[W0 + i SOz,  SOy + i SOx], [-SOy + i SOx, W0 - i SOz]],
 * stored per pattern block as a row-major (2 nf_A) x (2 nf_B) complex matrix
 * with row 2i+s, column 2j+s' (interleaved re, im doubles). */
void orc_spinor_ss(const orc_basis* b, const long long* blk_ptr, const int* blk_col, const long long* blk_off,
                   const double* W0, const double* SOx, const double* SOy, const double* SOz, double* SS) {
  for (int A = 0; A < b->n_atoms; ++A) {
    int nfA = species_nfn(b, b->species[A]);
    for (long long q = blk_ptr[A]; q < blk_ptr[A + 1]; ++q) {
      int B = blk_col[q];
      int nfB = species_nfn(b, b->species[B]);
      for (int i = 0; i < nfA; ++i) {
        for (int j = 0; j < nfB; ++j) {
          long long e = blk_off[q] + (long long)i * nfB + j;
          double w0 = W0[e], x = SOx[e], y = SOy[e], z = SOz[e];
          /* complex entries (re, im) of the 2x2 block */
          double blk[2][2][2] = {{{w0, z}, {y, x}}, {{-y, x}, {w0, -z}}};
          for (int s = 0; s < 2; ++s)
            for (int s2 = 0; s2 < 2; ++s2) {
              long long o = 4 * blk_off[q] + (long long)(2 * i + s) * (2 * nfB) + (2 * j + s2);
              SS[2 * o] = blk[s][s2][0];
              SS[2 * o + 1] = blk[s][s2][1];
            }
        }
      }
    }
  }
}
