// C ABI entry points for the compute calls: argument checks and dispatch to
// the FP64 or split-precision kernels.  No exception crosses this boundary.
#include "internal.h"

using namespace q4c;

namespace {

q4c_status check_pair(const q4c_tables* t, const q4c_grid* g, const char* who) {
  if (!t || !g) {
    set_error(std::string(who) + ": NULL handle");
    return Q4C_EINVAL;
  }
  if (g->tables != t) {
    set_error(std::string(who) + ": grid was partitioned with different tables");
    return Q4C_EINVAL;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device) {
    set_error(std::string(who) + ": current device differs from the grid's device");
    return Q4C_EINVAL;
  }
  return Q4C_OK;
}

}  // namespace

extern "C" q4c_status q4c_integrate(const q4c_tables* t, const q4c_grid* g, const double* v,
                                    q4c_precision prec, const q4c_matrices* out, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_integrate")) return st;
  Q4C_CHECK_ARG(v && out && out->V && out->W0 && out->SOx && out->SOy && out->SOz,
                "q4c_integrate: NULL input or output array");
  auto s = reinterpret_cast<cudaStream_t>(stream);
  try {
    if (prec == Q4C_FP64) return integrate_fp64(t, g, v, out, s);
    if (prec == Q4C_SPLIT) return integrate_split(t, g, v, out, s);
  } catch (const std::exception& e) {
    set_error(std::string("q4c_integrate: ") + e.what());
    return Q4C_ENOMEM;
  }
  set_error("q4c_integrate: unknown precision");
  return Q4C_EINVAL;
}

extern "C" q4c_status q4c_density(const q4c_tables* t, const q4c_grid* g, const double* P, q4c_precision prec,
                                  double* n, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_density")) return st;
  Q4C_CHECK_ARG(P && n, "q4c_density: NULL array");
  Q4C_CHECK_ARG(prec == Q4C_FP64 || prec == Q4C_SPLIT, "q4c_density: unknown precision");
  try {
    if (prec == Q4C_FP64) return density_fp64(t, g, P, n, reinterpret_cast<cudaStream_t>(stream));
    return density_split(t, g, P, n, reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::exception& e) {
    set_error(std::string("q4c_density: ") + e.what());
    return Q4C_ENOMEM;
  }
}

extern "C" q4c_status q4c_integrate_backward(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* G,
                                             q4c_precision prec, double* dLdv, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_integrate_backward")) return st;
  Q4C_CHECK_ARG(G && dLdv, "q4c_integrate_backward: NULL argument");
  Q4C_CHECK_ARG(prec == Q4C_FP64 || prec == Q4C_SPLIT, "q4c_integrate_backward: unknown precision");
  try {
    if (prec == Q4C_FP64) return backward_fp64(t, g, G, dLdv, reinterpret_cast<cudaStream_t>(stream));
    return backward_split(t, g, G, dLdv, reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::exception& e) {
    set_error(std::string("q4c_integrate_backward: ") + e.what());
    return Q4C_ENOMEM;
  }
}

extern "C" q4c_status q4c_density_full(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* P,
                                       q4c_precision prec, double* n, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_density_full")) return st;
  Q4C_CHECK_ARG(P && n, "q4c_density_full: NULL argument");
  Q4C_CHECK_ARG(prec == Q4C_FP64 || prec == Q4C_SPLIT, "q4c_density_full: unknown precision");
  auto s = reinterpret_cast<cudaStream_t>(stream);
  try {
    if (!P->V && !P->W0 && !P->SOx && !P->SOy && !P->SOz) {
      Q4C_CUDA(cudaMemsetAsync(n, 0, sizeof(double) * g->n_pts, s));
      return Q4C_OK;
    }
    if (prec == Q4C_FP64) return backward_fp64(t, g, P, n, s, false);
    return backward_split(t, g, P, n, s, false);
  } catch (const std::exception& e) {
    set_error(std::string("q4c_density_full: ") + e.what());
    return Q4C_ENOMEM;
  }
}

extern "C" q4c_status q4c_basis_eval(const q4c_tables* t, const q4c_grid* g, int64_t n_pts, const double* xyz,
                                     double* phi, double* grad, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_basis_eval")) return st;
  Q4C_CHECK_ARG(n_pts >= 0, "q4c_basis_eval: negative size");
  Q4C_CHECK_ARG(n_pts == 0 || (xyz && phi && grad), "q4c_basis_eval: NULL array");
  return basis_eval(t, g, n_pts, xyz, phi, grad, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" q4c_status q4c_integrate_columns(const q4c_tables* t, const q4c_grid* g, const double* v,
                                            q4c_precision prec, double* F, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_integrate_columns")) return st;
  Q4C_CHECK_ARG(v && F, "q4c_integrate_columns: NULL input or output array");
  Q4C_CHECK_ARG(prec == Q4C_FP64 || prec == Q4C_SPLIT, "q4c_integrate_columns: unknown precision");
  Q4C_CHECK_ARG(t->d_col_eps && t->d_col_coef,
                "q4c_integrate_columns: no column potentials (call q4c_tables_set_columns first)");
  try {
    if (prec == Q4C_SPLIT) return integrate_columns_split(t, g, v, F, reinterpret_cast<cudaStream_t>(stream));
    return integrate_columns_fp64(t, g, v, F, reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::exception& e) {
    set_error(std::string("q4c_integrate_columns: ") + e.what());
    return Q4C_ENOMEM;
  }
}

extern "C" q4c_status q4c_scf_pass(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* H,
                                   const q4c_matrices* P, double* n, const q4c_matrices* G, double* dLdv,
                                   q4c_precision prec, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_scf_pass")) return st;
  Q4C_CHECK_ARG(prec == Q4C_FP64 || prec == Q4C_SPLIT, "q4c_scf_pass: unknown precision");
  Q4C_CHECK_ARG(!H || (v && H->V && H->W0 && H->SOx && H->SOy && H->SOz),
                "q4c_scf_pass: H needs v and all five output arrays");
  Q4C_CHECK_ARG(!P || n, "q4c_scf_pass: P given without a density array");
  Q4C_CHECK_ARG(!G || dLdv, "q4c_scf_pass: G given without a gradient array");
  try {
    return scf_pass(t, g, v, H, P, n, G, dLdv, prec == Q4C_SPLIT, reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::exception& e) {
    set_error(std::string("q4c_scf_pass: ") + e.what());
    return Q4C_ENOMEM;
  }
}

extern "C" q4c_status q4c_autotune(const q4c_tables* t, q4c_grid* g, const double* v, q4c_stream stream) {
  if (q4c_status st = check_pair(t, g, "q4c_autotune")) return st;
  Q4C_CHECK_ARG(v, "q4c_autotune: NULL potential");
  try {
    return autotune_split(t, g, v, reinterpret_cast<cudaStream_t>(stream));
  } catch (const std::exception& e) {
    set_error(std::string("q4c_autotune: ") + e.what());
    return Q4C_ENOMEM;
  }
}

extern "C" q4c_status q4c_grid_tiling(const q4c_grid* g, int32_t bucket, int32_t* nb_max, int32_t* k_steps,
                                      int64_t* batches, double* ms_one, double* ms_two) {
  Q4C_CHECK_ARG(g, "q4c_grid_tiling: NULL grid");
  Q4C_CHECK_ARG(bucket >= 0 && bucket <= kTileBuckets, "q4c_grid_tiling: bucket out of range");
  if (bucket == kTileBuckets) {  // the density/adjoint kernel (one shape per grid)
    if (nb_max) *nb_max = 4096;
    if (k_steps) *k_steps = g->rd_ks;
    if (batches) *batches = g->n_batches;
    if (ms_one) *ms_one = g->rd_tune_ms[0];
    if (ms_two) *ms_two = g->rd_tune_ms[1];
    return Q4C_OK;
  }
  if (nb_max) *nb_max = kBucketNb[bucket];
  if (k_steps) *k_steps = g->split_ks[bucket];
  if (batches) {
    int64_t n = 0;
    for (int64_t b = 0; b < g->n_batches; ++b)
      if (tile_bucket(g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b]) == bucket) ++n;
    *batches = n;
  }
  if (ms_one) *ms_one = g->tune_ms[bucket][0];
  if (ms_two) *ms_two = g->tune_ms[bucket][1];
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_set_tiling(q4c_grid* g, int32_t bucket, int32_t k_steps) {
  Q4C_CHECK_ARG(g, "q4c_grid_set_tiling: NULL grid");
  Q4C_CHECK_ARG(bucket >= 0 && bucket <= kTileBuckets, "q4c_grid_set_tiling: bucket out of range");
  Q4C_CHECK_ARG(k_steps == 1 || k_steps == 2, "q4c_grid_set_tiling: k_steps must be 1 or 2");
  if (bucket == kTileBuckets)
    g->rd_ks = k_steps;
  else
    g->split_ks[bucket] = k_steps;
  return Q4C_OK;
}
