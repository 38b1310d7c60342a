// nao_tabulate: FP64 spline tables of the NAO radial functions (Eq. 12).
//
// The radial function u_l(r) = r^(l+1) exp(-alpha r^2) c(r) is sampled on the
// logarithmic knots r_k = r_min (r_c/r_min)^(k/(n-1)) and interpolated by a
// natural cubic spline in the knot index t = ln(r/r_min)/h.  The kernels read
// the spline as one cubic polynomial in s = t - k per interval, so the table
// stores (c0, c1, c2, c3) per interval: 32 bytes, one aligned double4 load.
#include <cmath>
#include <mutex>
#include <thread>

#include "internal.h"

namespace q4c {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

// 1 below r_on, 0 from r_c on, 1 - (10 s^3 - 15 s^4 + 6 s^5) in between
static double smooth_cut(double r, double r_on, double r_c) {
  if (r <= r_on) return 1.0;
  if (r >= r_c) return 0.0;
  const double s = (r - r_on) / (r_c - r_on);
  return 1.0 - s * s * s * (10.0 + s * (-15.0 + 6.0 * s));
}

// Natural cubic spline through y[0..n-1] at unit spacing: second derivatives
// m[k] from m[k-1] + 4 m[k] + m[k+1] = 6 (y[k+1] - 2 y[k] + y[k-1]),
// m[0] = m[n-1] = 0 (Thomas algorithm), then per-interval cubic coefficients.
static void natural_spline_coefficients(const std::vector<double>& y, double* coef) {
  const int n = static_cast<int>(y.size());
  std::vector<double> c(n, 0.0), d(n, 0.0), m(n, 0.0);
  // forward sweep over the interior unknowns 1..n-2
  for (int k = 1; k <= n - 2; ++k) {
    const double rhs = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]);
    const double denom = 4.0 - (k > 1 ? c[k - 1] : 0.0);
    c[k] = 1.0 / denom;
    d[k] = (rhs - (k > 1 ? d[k - 1] : 0.0)) / denom;
  }
  for (int k = n - 2; k >= 1; --k) m[k] = d[k] - c[k] * m[k + 1];
  for (int k = 0; k + 1 < n; ++k) {
    // u(s) = y_k (1-s) + y_{k+1} s + m_k ((1-s)^3 - (1-s))/6 + m_{k+1} (s^3 - s)/6
    coef[4 * k + 0] = y[k];
    coef[4 * k + 1] = (y[k + 1] - y[k]) - m[k] / 3.0 - m[k + 1] / 6.0;
    coef[4 * k + 2] = 0.5 * m[k];
    coef[4 * k + 3] = (m[k + 1] - m[k]) / 6.0;
  }
}

}  // namespace q4c

using namespace q4c;

DevBasis q4c_tables::view() const {
  DevBasis b;
  b.coef = d_coef;
  b.g0 = d_g0;
  b.rad_l = d_rad_l;
  b.sp_rad0 = d_sp_rad0;
  b.sp_nrad = d_sp_nrad;
  b.sp_nfn = d_sp_nfn;
  b.r_c = r_c;
  b.r_min = r_min;
  b.inv_rmin = 1.0 / r_min;
  b.inv_h = 1.0 / h;
  b.n_log = n_log;
  return b;
}

DfTables q4c_tables::df_view() const {
  DfTables d{};
  d.coef = d_coef_df;
  d.g0 = d_g0_df;
  d.inv_knot = d_inv_knot_df;
  const double ih = 1.0 / h;
  d.inv_h_df = df{static_cast<float>(ih), static_cast<float>(ih - static_cast<float>(ih))};
  d.inv_h = static_cast<float>(ih);
  d.inv_rmin = static_cast<float>(1.0 / r_min);
  d.rmin2 = static_cast<float>(r_min * r_min);
  d.rc2 = static_cast<float>(r_c * r_c);
  return d;
}

template <typename T>
static q4c_status upload(T** dst, const std::vector<T>& src) {
  Q4C_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * (src.empty() ? 1 : src.size())));
  if (!src.empty()) Q4C_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return Q4C_OK;
}

// Radial functions from (l, alpha) (knots == NULL) or from their values at
// the knots (knots [sum n_rad][n_log], alpha unused).
static q4c_status tabulate(const q4c_basis_desc* desc, const double* knots, q4c_tables** out) {
  Q4C_CHECK_ARG(desc && out, "nao_tabulate: NULL argument");
  *out = nullptr;
  Q4C_CHECK_ARG(desc->n_species >= 1 && desc->n_rad && desc->l && (desc->alpha || knots),
                "nao_tabulate: empty basis");
  Q4C_CHECK_ARG(desc->n_log >= 4, "nao_tabulate: n_log must be >= 4");
  Q4C_CHECK_ARG(desc->r_min > 0 && desc->r_on > desc->r_min && desc->r_cut > desc->r_on,
                "nao_tabulate: need 0 < r_min < r_on < r_cut");
  auto* t = new q4c_tables();
  t->n_species = desc->n_species;
  int tot = 0;
  for (int s = 0; s < desc->n_species; ++s) {
    if (desc->n_rad[s] < 1) {
      delete t;
      set_error("nao_tabulate: every species needs a radial function");
      return Q4C_EINVAL;
    }
    t->rad0.push_back(tot);
    t->n_rad.push_back(desc->n_rad[s]);
    int nf = 0;
    for (int k = 0; k < desc->n_rad[s]; ++k) {
      const int l = desc->l[tot + k];
      const double a = knots ? 0.0 : desc->alpha[tot + k];
      if (l < 0 || (!knots && !(a > 0.0))) {
        delete t;
        set_error("nao_tabulate: need l >= 0 and alpha > 0");
        return Q4C_EINVAL;
      }
      if (l > kMaxL) {
        delete t;
        set_error("nao_tabulate: l > 4 is not supported");
        return Q4C_EUNSUPPORTED;
      }
      nf += 2 * l + 1;
      t->rad_l.push_back(l);
      t->alpha.push_back(a);
    }
    t->nfn.push_back(nf);
    tot += desc->n_rad[s];
  }
  t->r_c = desc->r_cut;
  t->r_on = desc->r_on;
  t->r_min = desc->r_min;
  t->n_log = desc->n_log;
  t->h = std::log(desc->r_cut / desc->r_min) / (desc->n_log - 1);
  const int n = desc->n_log;
  t->h_coef.assign(static_cast<size_t>(tot) * (n - 1) * 4, 0.0);
  t->h_g0.assign(tot, 0.0);
  std::vector<double> y(n);
  for (int k = 0; k < tot; ++k) {
    const int l = t->rad_l[k];
    for (int j = 0; j < n; ++j) {
      const double r = desc->r_min * std::exp(j * t->h);
      // the last knot is r_c itself, where the cutoff vanishes
      const double rr = (j == n - 1) ? desc->r_cut : r;
      y[j] = knots ? knots[static_cast<size_t>(k) * n + j]
                   : std::pow(rr, l + 1) * std::exp(-t->alpha[k] * rr * rr) * smooth_cut(rr, desc->r_on, desc->r_cut);
    }
    natural_spline_coefficients(y, &t->h_coef[static_cast<size_t>(k) * (n - 1) * 4]);
    t->h_g0[k] = y[0] / std::pow(desc->r_min, l + 1);
  }
  // double-float copies: coefficient pairs, g below r_min, inverse knots
  auto split = [](double x) { const float h = static_cast<float>(x); return df{h, static_cast<float>(x - h)}; };
  std::vector<float4> coef_df(static_cast<size_t>(tot) * (n - 1) * 2);
  for (size_t iv = 0; iv < static_cast<size_t>(tot) * (n - 1); ++iv) {
    const df c0 = split(t->h_coef[4 * iv]), c1 = split(t->h_coef[4 * iv + 1]), c2 = split(t->h_coef[4 * iv + 2]),
             c3 = split(t->h_coef[4 * iv + 3]);
    coef_df[2 * iv] = make_float4(c0.hi, c0.lo, c1.hi, c1.lo);
    coef_df[2 * iv + 1] = make_float4(c2.hi, c2.lo, c3.hi, c3.lo);
  }
  std::vector<df> g0_df(tot), inv_knot(n);
  for (int k = 0; k < tot; ++k) g0_df[k] = split(t->h_g0[k]);
  for (int j = 0; j < n; ++j) inv_knot[j] = split(1.0 / (desc->r_min * std::exp(j * t->h)));
  cudaGetDevice(&t->device);
  q4c_status st;
  if ((st = upload(&t->d_coef, t->h_coef)) || (st = upload(&t->d_g0, t->h_g0)) ||
      (st = upload(&t->d_rad_l, t->rad_l)) || (st = upload(&t->d_sp_rad0, t->rad0)) ||
      (st = upload(&t->d_sp_nrad, t->n_rad)) || (st = upload(&t->d_sp_nfn, t->nfn)) ||
      (st = upload(&t->d_coef_df, coef_df)) || (st = upload(&t->d_g0_df, g0_df)) ||
      (st = upload(&t->d_inv_knot_df, inv_knot)) || (st = build_spinor_tables(t))) {
    q4c_tables_destroy(t);
    return st;
  }
  *out = t;
  return Q4C_OK;
}

extern "C" q4c_status nao_tabulate(const q4c_basis_desc* desc, q4c_tables** out) {
  return tabulate(desc, nullptr, out);
}

extern "C" q4c_status nao_tabulate_knots(const q4c_basis_desc* desc, const double* knots, q4c_tables** out) {
  Q4C_CHECK_ARG(knots, "nao_tabulate_knots: NULL knots");
  return tabulate(desc, knots, out);
}

extern "C" void q4c_tables_destroy(q4c_tables* t) {
  if (!t) return;
  cudaFree(t->d_coef);
  cudaFree(t->d_g0);
  cudaFree(t->d_rad_l);
  cudaFree(t->d_sp_rad0);
  cudaFree(t->d_sp_nrad);
  cudaFree(t->d_sp_nfn);
  cudaFree(t->d_coef_df);
  cudaFree(t->d_g0_df);
  cudaFree(t->d_inv_knot_df);
  cudaFree(t->d_col_eps);
  cudaFree(t->d_col_coef);
  cudaFree(t->d_spn0);
  cudaFree(t->d_spn_col);
  cudaFree(t->d_spn_row);
  cudaFree(t->d_ss0);
  cudaFree(t->d_col_coef_df);
  delete t;
}

extern "C" q4c_status q4c_tables_set_columns(q4c_tables* t, const double* eps, const double* knots) {
  Q4C_CHECK_ARG(t && eps && knots, "q4c_tables_set_columns: NULL argument");
  const int n_tot = static_cast<int>(t->rad_l.size()), n = t->n_log;
  std::vector<double> coef(static_cast<size_t>(n_tot) * (n - 1) * 4), y(n);
  for (int k = 0; k < n_tot; ++k) {
    for (int j = 0; j < n; ++j) y[j] = knots[static_cast<size_t>(k) * n + j];
    natural_spline_coefficients(y, &coef[static_cast<size_t>(k) * (n - 1) * 4]);
  }
  std::vector<double> e(eps, eps + n_tot);
  auto split = [](double x) { const float h = static_cast<float>(x); return std::make_pair(h, static_cast<float>(x - h)); };
  std::vector<float4> coef_df(static_cast<size_t>(n_tot) * (n - 1) * 2);
  for (size_t iv = 0; iv < static_cast<size_t>(n_tot) * (n - 1); ++iv) {
    const auto c0 = split(coef[4 * iv]), c1 = split(coef[4 * iv + 1]), c2 = split(coef[4 * iv + 2]),
               c3 = split(coef[4 * iv + 3]);
    coef_df[2 * iv] = make_float4(c0.first, c0.second, c1.first, c1.second);
    coef_df[2 * iv + 1] = make_float4(c2.first, c2.second, c3.first, c3.second);
  }
  cudaFree(t->d_col_eps);
  cudaFree(t->d_col_coef);
  cudaFree(t->d_col_coef_df);
  t->d_col_eps = nullptr;
  t->d_col_coef = nullptr;
  t->d_col_coef_df = nullptr;
  if (q4c_status st = upload(&t->d_col_eps, e)) return st;
  if (q4c_status st = upload(&t->d_col_coef_df, coef_df)) return st;
  return upload(&t->d_col_coef, coef);
}

extern "C" q4c_status q4c_tables_export(const q4c_tables* t, int32_t radial, double* coef_host) {
  Q4C_CHECK_ARG(t && coef_host, "q4c_tables_export: NULL argument");
  Q4C_CHECK_ARG(radial >= 0 && radial < static_cast<int>(t->rad_l.size()), "q4c_tables_export: bad radial index");
  const size_t per = static_cast<size_t>(t->n_log - 1) * 4;
  for (size_t i = 0; i < per; ++i) coef_host[i] = t->h_coef[radial * per + i];
  return Q4C_OK;
}

extern "C" const char* q4c_last_error(void) { return q4c::last_error(); }
