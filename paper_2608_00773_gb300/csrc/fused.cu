// One pass per SCF step: the integration of v into H, the density n of P
// (Eqs. 39-40, with the gradient terms of the kinetic-balance reading when P
// carries W0/SO slots) and the adjoint dL/dv of G, sharing the basis
// evaluation.  Per wave of batches the offset tables and the basis tiles
// (Phi and its gradient, with per-function exponents for the products and
// per-point exponents for the row-dot contractions) are built once, and the
// products, the density and the adjoint kernels read the same tiles.  Each
// result equals that of its separate call (q4c_integrate, q4c_density /
// q4c_density_full, q4c_integrate_backward) up to the order of the FP64
// atomic additions.
#include "internal.h"

namespace q4c {

namespace {
bool any(const q4c_matrices* m) { return m && (m->V || m->W0 || m->SOx || m->SOy || m->SOz); }
}  // namespace

q4c_status scf_pass(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* H,
                    const q4c_matrices* P, double* n, const q4c_matrices* Gm, double* dLdv, bool split,
                    cudaStream_t s) {
  const bool do_h = H != nullptr;
  const bool do_n = n != nullptr && any(P);
  const bool full_n = do_n && (P->W0 || P->SOx || P->SOy || P->SOz);  // gradient terms present
  const bool do_g = dLdv != nullptr && any(Gm);
  if (n && !do_n) Q4C_CUDA(cudaMemsetAsync(n, 0, sizeof(double) * g->n_pts, s));
  if (dLdv && !do_g) Q4C_CUDA(cudaMemsetAsync(dLdv, 0, sizeof(double) * g->n_pts, s));
  if (split) {
    if (do_h && g->max_np > 341) {
      set_error("q4c_scf_pass: the split path needs batches of at most 341 points");
      return Q4C_EUNSUPPORTED;
    }
    if ((do_n || do_g) && g->max_nb > 4096) {
      set_error("q4c_scf_pass: the split density/adjoint need at most 4096 active functions per batch");
      return Q4C_EUNSUPPORTED;
    }
  }
  if (do_h) {
    double* outs[5] = {H->V, H->W0, H->SOx, H->SOy, H->SOz};
    for (double* o : outs) Q4C_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * g->nnz, s));
  }
  if (!do_h && !do_n && !do_g) return Q4C_OK;
  const float2* mP[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const float2* mG[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  unsigned presentP = 0, presentG = 0;
  if (split && do_n) {
    const double* mats[5] = {P->V, P->W0, P->SOx, P->SOy, P->SOz};
    if (q4c_status st = rowdot_prepare(g, mats, 0, mP, &presentP, s)) return st;
  }
  if (split && do_g) {
    const double* mats[5] = {Gm->V, Gm->W0, Gm->SOx, Gm->SOy, Gm->SOz};
    if (q4c_status st = rowdot_prepare(g, mats, 5, mG, &presentG, s)) return st;
  }
  const int n_waves = static_cast<int>(g->wave_b0.size()) - 1;
  for (int wv = 0; wv < n_waves; ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (split) {
      if (q4c_status st = launch_fill_idx(t, g, b0, b1, s)) return st;
      const int nq = (do_h || do_g || full_n) ? 4 : 1;
      if (q4c_status st = launch_basis_df(t, g, b0, b1, do_h ? v : nullptr, do_h ? g->d_colexp : nullptr,
                                          (do_n || do_g) ? g->d_rowexp : nullptr, nq, s,
                                          do_h ? g->d_dpad : nullptr))
        return st;
      if (do_h)
        if (q4c_status st = products_wave(g, wv, H, s)) return st;
      if (do_n)
        if (q4c_status st = rowdot_wave(g, wv, full_n ? 1 : 0, mP, presentP, false, n, s)) return st;
      if (do_g)
        if (q4c_status st = rowdot_wave(g, wv, 1, mG, presentG, true, dLdv, s)) return st;
    } else {
      if (q4c_status st = launch_basis_tiles(t, g, b0, b1, nullptr, nullptr, s)) return st;
      if (do_h)
        if (q4c_status st = products_fp64_wave(g, wv, v, H, s)) return st;
      if (do_n) {
        if (full_n) {
          if (q4c_status st = backward_fp64_wave(g, wv, P, n, false, s)) return st;
        } else if (q4c_status st = density_fp64_wave(g, wv, P->V, n, s)) {
          return st;
        }
      }
      if (do_g)
        if (q4c_status st = backward_fp64_wave(g, wv, Gm, dLdv, true, s)) return st;
    }
  }
  if (do_h) return mirror_and_spinor(g, H, s);
  return Q4C_OK;
}

}  // namespace q4c
