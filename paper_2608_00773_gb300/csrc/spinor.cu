// Scalar -> spinor transformation of the Q4C method (Section II, Eqs. 9-14;
// Section III A, Eqs. 33-34 and 37-38; Appendix A; Algorithm 1).
//
// Spinor basis of an atom: per radial function (angular momentum l), in the
// species' order, j = l - 1/2 (kappa = l, only for l > 0) then j = l + 1/2
// (kappa = -l - 1), m_j = -j..j ascending; 2 (2l + 1) spinor functions per
// radial, so an atom has twice as many spinor as scalar functions.  Spinor
// function mu = sum_(t,s) G_(2t+s),mu phi_t eta_s with the coupling
// coefficients of Eq. 10,
//   C_alpha = a sqrt((l + a m_j + 1/2) / (2l + 1)),  C_beta = sqrt((l - a m_j + 1/2) / (2l + 1)),
// a = 2 (j - l), multiplying the complex harmonics Y~_l^(m_j -+ 1/2), which
// are written in the real harmonics of Appendix B with the Condon-Shortley
// phase: Y~^m = (Y_(l,m) + i Y_(l,-m)) / sqrt 2 for m > 0 and
// Y~^-m = (-1)^m (Y_(l,m) - i Y_(l,-m)) / sqrt 2.  Each spinor function
// touches at most four scalar-spin functions and each scalar-spin function
// at most four spinor functions, so both maps are stored as four entries.
//
// Forward (Eqs. 33-34), per pattern block (A, B, T), complex:
//   HL = G_A^dagger (V x 1) G_B,   HS = G_A^dagger (W0 1 + i SO.sigma) G_B
// (the large component, and the kinetic-balance small component whose
// scalar-spin blocks are those of q4c_integrate's spinor_SS output).
// Reverse (Eqs. 37-38): D'_ab = sum_mu,nu conj(G_a,mu) D_mu,nu G_b,nu and
//   P^V = P^W0 = Re tr_s D'_ij,  P^SOk = Re(i sum_ss' (sigma_k)_ss' D'_(is)(js')),
// the inputs of q4c_density_full.
//
// Kappa selection (q4c_tables_set_kappa): a radial function may carry the
// spinors of one kappa only, j = |kappa| - 1/2 with the coupling of the
// spin-angular function of that kappa.  Tables of the small-component radials
// Q (Eq. 12b) select kappa~ = -kappa of their large-component parent: the
// small component of spinor (kappa, m_j) is i Q/r Upsilon_(-kappa, m_j)
// (Eq. 11), so G of these tables is G^S of Eq. 14, its spinor functions line
// up one to one with those of the large-component tables when the radials
// come per parent in the order kappa = l, kappa = -l - 1, and
// G^S^dagger (F^S x 1) G^S is the SS block of Eq. 19.
#include <cmath>

#include "internal.h"

namespace q4c {
namespace spinor {

struct Ent {
  int idx;  // scalar-spin row 2t + s (column view) or spinor index (row view); -1 unused
  int pad;
  double re, im;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One CTA per pattern block; thread per spinor element (mu, nu).
// Spinor block q starts at spin_off[q] (complex elements), or at 4 blk_off[q]
// when spin_off is NULL (no kappa selection: twice the scalar counts).
__global__ void k_forward(const int* __restrict__ blk_row, const int* __restrict__ blk_col,
                          const int64_t* __restrict__ blk_off, const int64_t* __restrict__ spin_off,
                          const int* __restrict__ atom_sp, const int* __restrict__ sp_nfn,
                          const int* __restrict__ spn0, const Ent* __restrict__ col, const double* __restrict__ V,
                          const double* __restrict__ W0, const double* __restrict__ SOx,
                          const double* __restrict__ SOy, const double* __restrict__ SOz, double2* __restrict__ HL,
                          double2* __restrict__ HS) {
  const int q = blockIdx.x;
  const int A = blk_row[q], B = blk_col[q];
  const int sa = atom_sp[A], sb = atom_sp[B];
  const int nfB = sp_nfn[sb];
  const int nsA = spn0[sa + 1] - spn0[sa], nsB = spn0[sb + 1] - spn0[sb];
  const int64_t off = blk_off[q];
  const int64_t so = spin_off ? spin_off[q] : 4 * off;
  const Ent* cA = col + 4 * spn0[sa];
  const Ent* cB = col + 4 * spn0[sb];
  for (int e = threadIdx.x; e < nsA * nsB; e += blockDim.x) {
    const int mu = e / nsB, nu = e - mu * nsB;
    double2 hl = make_double2(0.0, 0.0), hs = make_double2(0.0, 0.0);
#pragma unroll
    for (int ea = 0; ea < 4; ++ea) {
      const Ent a = cA[4 * mu + ea];
      if (a.idx < 0) continue;
      const int ta = a.idx >> 1, s = a.idx & 1;
#pragma unroll
      for (int eb = 0; eb < 4; ++eb) {
        const Ent b = cB[4 * nu + eb];
        if (b.idx < 0) continue;
        const int tb = b.idx >> 1, s2 = b.idx & 1;
        const double2 g = cmul(make_double2(a.re, -a.im), make_double2(b.re, b.im));
        const int64_t k = off + static_cast<int64_t>(ta) * nfB + tb;
        if (V && s == s2) {
          const double v = V[k];
          hl.x += g.x * v;
          hl.y += g.y * v;
        }
        if (HS) {
          // (W0 1 + i SO.sigma)_(s, s2)
          const double w = W0 ? W0[k] : 0.0, x = SOx ? SOx[k] : 0.0, y = SOy ? SOy[k] : 0.0,
                       z = SOz ? SOz[k] : 0.0;
          double2 F;
          if (s == s2)
            F = make_double2(w, s == 0 ? z : -z);
          else
            F = make_double2(s == 0 ? y : -y, x);
          const double2 t = cmul(g, F);
          hs.x += t.x;
          hs.y += t.y;
        }
      }
    }
    const int64_t o = so + e;
    if (HL) HL[o] = hl;
    if (HS) HS[o] = hs;
  }
}

// One CTA per pattern block; thread per scalar element (t, u).
__global__ void k_reverse(const int* __restrict__ blk_row, const int* __restrict__ blk_col,
                          const int64_t* __restrict__ blk_off, const int64_t* __restrict__ spin_off,
                          const int* __restrict__ atom_sp, const int* __restrict__ sp_nfn,
                          const int* __restrict__ spn0, const int* __restrict__ ss0, const Ent* __restrict__ row,
                          const double2* __restrict__ D, double* __restrict__ PV, double* __restrict__ PW0,
                          double* __restrict__ PSOx, double* __restrict__ PSOy, double* __restrict__ PSOz) {
  const int q = blockIdx.x;
  const int A = blk_row[q], B = blk_col[q];
  const int sa = atom_sp[A], sb = atom_sp[B];
  const int nfA = sp_nfn[sa], nfB = sp_nfn[sb];
  const int nsB = spn0[sb + 1] - spn0[sb];
  const int64_t off = blk_off[q];
  const double2* Dq = D + (spin_off ? spin_off[q] : 4 * off);
  const Ent* rA = row + 4 * ss0[sa];
  const Ent* rB = row + 4 * ss0[sb];
  for (int e = threadIdx.x; e < nfA * nfB; e += blockDim.x) {
    const int t = e / nfB, u = e - t * nfB;
    double2 Dp[2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int ea = 0; ea < 4; ++ea) {
          const Ent a = rA[4 * (2 * t + s) + ea];
          if (a.idx < 0) continue;
#pragma unroll
          for (int eb = 0; eb < 4; ++eb) {
            const Ent b = rB[4 * (2 * u + s2) + eb];
            if (b.idx < 0) continue;
            const double2 g = cmul(make_double2(a.re, -a.im), make_double2(b.re, b.im));
            const double2 d = cmul(g, Dq[static_cast<int64_t>(a.idx) * nsB + b.idx]);
            acc.x += d.x;
            acc.y += d.y;
          }
        }
        Dp[s][s2] = acc;
      }
    const int64_t k = off + e;
    const double tr = Dp[0][0].x + Dp[1][1].x;
    if (PV) PV[k] = tr;
    if (PW0) PW0[k] = tr;
    if (PSOx) PSOx[k] = -(Dp[0][1].y + Dp[1][0].y);
    if (PSOy) PSOy[k] = Dp[0][1].x - Dp[1][0].x;
    if (PSOz) PSOz[k] = -(Dp[0][0].y - Dp[1][1].y);
  }
}

}  // namespace spinor

// Host tables of one set of species: column and row views of G, and the
// quantum numbers of every spinor function.
q4c_status build_spinor_tables(q4c_tables* t) {
  using spinor::Ent;
  const int ns = t->n_species;
  const bool sel = !t->h_kappa_sel.empty();
  auto kappa_sel = [&](int s, int k) { return sel ? t->h_kappa_sel[t->rad0[s] + k] : 0; };
  std::vector<int> spn0(ns + 1, 0), ss0(ns + 1, 0);
  for (int s = 0; s < ns; ++s) {
    ss0[s + 1] = ss0[s] + 2 * t->nfn[s];
    int n = 0;
    for (int k = 0; k < t->n_rad[s]; ++k) {
      const int l = t->rad_l[t->rad0[s] + k], kp = kappa_sel(s, k);
      n += kp ? 2 * std::abs(kp) : 2 * (2 * l + 1);
    }
    spn0[s + 1] = spn0[s] + n;
  }
  const int total = spn0[ns], total_ss = ss0[ns];
  std::vector<Ent> col(4 * static_cast<size_t>(total), Ent{-1, 0, 0.0, 0.0});
  std::vector<Ent> row(4 * static_cast<size_t>(total_ss), Ent{-1, 0, 0.0, 0.0});
  t->h_spn_radial.assign(total, 0);
  t->h_spn_kappa.assign(total, 0);
  t->h_spn_two_mj.assign(total, 0);
  const double r2 = std::sqrt(0.5);
  for (int s = 0; s < ns; ++s) {
    int t0 = 0, mu = 0;  // first scalar function of the shell, spinor index within the atom
    for (int k = 0; k < t->n_rad[s]; ++k) {
      const int l = t->rad_l[t->rad0[s] + k], kp = kappa_sel(s, k);
      for (int jx2 : {2 * l - 1, 2 * l + 1}) {
        if (jx2 < 0) continue;
        const int a = jx2 == 2 * l + 1 ? 1 : -1;
        if (kp && kp != (a > 0 ? -l - 1 : l)) continue;
        for (int mjx2 = -jx2; mjx2 <= jx2; mjx2 += 2, ++mu) {
          const int g = spn0[s] + mu;
          t->h_spn_radial[g] = k;
          t->h_spn_kappa[g] = a > 0 ? -l - 1 : l;
          t->h_spn_two_mj[g] = mjx2;
          const double den = 2.0 * (2 * l + 1);
          const double c[2] = {a * std::sqrt((2 * l + a * mjx2 + 1) / den), std::sqrt((2 * l - a * mjx2 + 1) / den)};
          int ne = 0;
          for (int sp = 0; sp < 2; ++sp) {  // spin up: m_l = m_j - 1/2; spin down: m_l = m_j + 1/2
            const int ml = (mjx2 + (sp == 0 ? -1 : 1)) / 2;
            if (ml < -l || ml > l) continue;
            // complex harmonic Y~_l^ml as (real index m, coefficient)
            struct Term {
              int m;
              double re, im;
            } terms[2];
            int nt = 0;
            if (ml == 0) {
              terms[nt++] = {0, 1.0, 0.0};
            } else if (ml > 0) {
              terms[nt++] = {ml, r2, 0.0};
              terms[nt++] = {-ml, 0.0, r2};
            } else {
              const double sg = ((-ml) & 1) ? -1.0 : 1.0;
              terms[nt++] = {-ml, sg * r2, 0.0};
              terms[nt++] = {ml, 0.0, -sg * r2};
            }
            for (int i = 0; i < nt; ++i) {
              const int rowi = 2 * (t0 + terms[i].m + l) + sp;
              const Ent e{rowi, 0, c[sp] * terms[i].re, c[sp] * terms[i].im};
              if (ne < 4) col[4 * static_cast<size_t>(g) + ne] = e;
              ++ne;
              // row view: the spinor functions of scalar-spin row rowi
              Ent* rv = &row[4 * static_cast<size_t>(ss0[s] + rowi)];
              int slot = 0;
              while (slot < 4 && rv[slot].idx >= 0) ++slot;
              if (slot == 4 || ne > 4) {  // at most two m_l x two j per row, two spins x two terms per column
                set_error("nao_tabulate: spinor relation table overflow");
                return Q4C_EINVAL;
              }
              rv[slot] = Ent{mu, 0, e.re, e.im};
            }
          }
        }
      }
      t0 += 2 * l + 1;
    }
  }
  t->h_spn0 = spn0;
  t->h_ss0 = ss0;
  // a rebuild (new kappa selection) replaces the device views
  cudaFree(t->d_spn0);
  cudaFree(t->d_ss0);
  cudaFree(t->d_spn_col);
  cudaFree(t->d_spn_row);
  t->d_spn0 = t->d_ss0 = nullptr;
  t->d_spn_col = t->d_spn_row = nullptr;
  Q4C_CUDA(cudaMalloc(&t->d_spn0, sizeof(int) * spn0.size()));
  Q4C_CUDA(cudaMemcpy(t->d_spn0, spn0.data(), sizeof(int) * spn0.size(), cudaMemcpyHostToDevice));
  Q4C_CUDA(cudaMalloc(&t->d_ss0, sizeof(int) * ss0.size()));
  Q4C_CUDA(cudaMemcpy(t->d_ss0, ss0.data(), sizeof(int) * ss0.size(), cudaMemcpyHostToDevice));
  Q4C_CUDA(cudaMalloc(&t->d_spn_col, sizeof(Ent) * col.size()));
  Q4C_CUDA(cudaMemcpy(t->d_spn_col, col.data(), sizeof(Ent) * col.size(), cudaMemcpyHostToDevice));
  Q4C_CUDA(cudaMalloc(&t->d_spn_row, sizeof(Ent) * row.size()));
  Q4C_CUDA(cudaMemcpy(t->d_spn_row, row.data(), sizeof(Ent) * row.size(), cudaMemcpyHostToDevice));
  return Q4C_OK;
}

// Offsets of the spinor blocks of a grid's pattern under tables with a kappa
// selection (prefix sums of n_spinor(A) n_spinor(B)); total in *n.
static std::vector<int64_t> spinor_block_offsets(const q4c_tables* t, const q4c_grid* g, int64_t* n) {
  std::vector<int64_t> off(static_cast<size_t>(g->n_blocks) + 1, 0);
  for (int A = 0; A < g->n_atoms; ++A) {
    const int sa = g->h_atom_sp[A];
    const int64_t nsA = t->h_spn0[sa + 1] - t->h_spn0[sa];
    for (int64_t q = g->h_blk_ptr[A]; q < g->h_blk_ptr[A + 1]; ++q) {
      const int sb = g->h_atom_sp[g->h_blk_col[q]];
      off[q + 1] = off[q] + nsA * (t->h_spn0[sb + 1] - t->h_spn0[sb]);
    }
  }
  *n = off.back();
  return off;
}

// Device copy of the spinor block offsets for one call (NULL without a
// kappa selection); the caller frees it on the stream.
static q4c_status upload_spinor_offsets(const q4c_tables* t, const q4c_grid* g, cudaStream_t s, int64_t** d) {
  *d = nullptr;
  if (t->h_kappa_sel.empty()) return Q4C_OK;
  int64_t n = 0;
  const std::vector<int64_t> off = spinor_block_offsets(t, g, &n);
  Q4C_CUDA(cudaMallocAsync(reinterpret_cast<void**>(d), sizeof(int64_t) * off.size(), s));
  // pageable source: the copy is staged before the call returns
  Q4C_CUDA(cudaMemcpyAsync(*d, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
  return Q4C_OK;
}

}  // namespace q4c

using namespace q4c;

extern "C" q4c_status q4c_tables_set_kappa(q4c_tables* t, const int32_t* kappa) {
  Q4C_CHECK_ARG(t, "q4c_tables_set_kappa: NULL tables");
  const int n = static_cast<int>(t->rad_l.size());
  std::vector<int> sel;
  if (kappa) {
    sel.assign(kappa, kappa + n);
    for (int k = 0; k < n; ++k) {
      const int kp = sel[k], l = t->rad_l[k];
      Q4C_CHECK_ARG(kp == 0 || kp == -l - 1 || (l > 0 && kp == l),
                    "q4c_tables_set_kappa: kappa must be 0, -l-1 or l (l > 0) of its radial function");
    }
    bool any = false;
    for (int kp : sel) any = any || kp != 0;
    if (!any) sel.clear();
  }
  t->h_kappa_sel = sel;
  return build_spinor_tables(t);
}

extern "C" q4c_status q4c_spinor_nnz(const q4c_tables* t, const q4c_grid* g, int64_t* n) {
  Q4C_CHECK_ARG(t && g && n, "q4c_spinor_nnz: NULL argument");
  Q4C_CHECK_ARG(g->tables == t, "q4c_spinor_nnz: grid was partitioned with different tables");
  spinor_block_offsets(t, g, n);
  return Q4C_OK;
}

extern "C" q4c_status q4c_spinor_basis(const q4c_tables* t, int32_t species, int32_t* n, int32_t* radial,
                                       int32_t* kappa, int32_t* two_mj) {
  Q4C_CHECK_ARG(t && n, "q4c_spinor_basis: NULL argument");
  Q4C_CHECK_ARG(species >= 0 && species < t->n_species, "q4c_spinor_basis: species out of range");
  const int a = t->h_spn0[species], b = t->h_spn0[species + 1];
  *n = b - a;
  for (int i = a; i < b; ++i) {
    if (radial) radial[i - a] = t->h_spn_radial[i];
    if (kappa) kappa[i - a] = t->h_spn_kappa[i];
    if (two_mj) two_mj[i - a] = t->h_spn_two_mj[i];
  }
  return Q4C_OK;
}

extern "C" q4c_status q4c_spinor_transform(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* F,
                                           double* HL, double* HS, q4c_stream stream) {
  Q4C_CHECK_ARG(t && g && F, "q4c_spinor_transform: NULL argument");
  Q4C_CHECK_ARG(g->tables == t, "q4c_spinor_transform: grid was partitioned with different tables");
  Q4C_CHECK_ARG(!HL || F->V, "q4c_spinor_transform: the large component needs F->V");
  Q4C_CHECK_ARG(!HS || F->W0 || F->SOx || F->SOy || F->SOz,
                "q4c_spinor_transform: the small component needs F->W0 or an SO slot");
  if ((!HL && !HS) || g->n_blocks == 0) return Q4C_OK;
  auto s = reinterpret_cast<cudaStream_t>(stream);
  int64_t* d_so = nullptr;
  q4c_status st = upload_spinor_offsets(t, g, s, &d_so);
  if (st) return st;
  {
    KernelScope ks("spinor_transform", s);
    spinor::k_forward<<<static_cast<unsigned>(g->n_blocks), 256, 0, s>>>(
        g->d_blk_row, g->d_blk_col, g->d_blk_off, d_so, g->d_atom_sp, t->d_sp_nfn, t->d_spn0,
        reinterpret_cast<const spinor::Ent*>(t->d_spn_col), HL ? F->V : nullptr, F->W0, F->SOx, F->SOy, F->SOz,
        reinterpret_cast<double2*>(HL), reinterpret_cast<double2*>(HS));
  }
  const cudaError_t e = cudaGetLastError();
  if (d_so) cudaFreeAsync(d_so, s);
  Q4C_CUDA(e);
  return Q4C_OK;
}

extern "C" q4c_status q4c_spinor_density_matrices(const q4c_tables* t, const q4c_grid* g, const double* D,
                                                  const q4c_matrices* P, q4c_stream stream) {
  Q4C_CHECK_ARG(t && g && D && P, "q4c_spinor_density_matrices: NULL argument");
  Q4C_CHECK_ARG(g->tables == t, "q4c_spinor_density_matrices: grid was partitioned with different tables");
  if (g->n_blocks == 0) return Q4C_OK;
  auto s = reinterpret_cast<cudaStream_t>(stream);
  int64_t* d_so = nullptr;
  q4c_status st = upload_spinor_offsets(t, g, s, &d_so);
  if (st) return st;
  {
    KernelScope ks("spinor_reverse", s);
    spinor::k_reverse<<<static_cast<unsigned>(g->n_blocks), 256, 0, s>>>(
        g->d_blk_row, g->d_blk_col, g->d_blk_off, d_so, g->d_atom_sp, t->d_sp_nfn, t->d_spn0, t->d_ss0,
        reinterpret_cast<const spinor::Ent*>(t->d_spn_row), reinterpret_cast<const double2*>(D), P->V, P->W0,
        P->SOx, P->SOy, P->SOz);
  }
  const cudaError_t e = cudaGetLastError();
  if (d_so) cudaFreeAsync(d_so, s);
  Q4C_CUDA(e);
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_batch_spinors(const q4c_grid* g, int64_t batch, int32_t* n, int32_t* centre,
                                             int32_t* spinor) {
  Q4C_CHECK_ARG(g && n, "q4c_grid_batch_spinors: NULL argument");
  Q4C_CHECK_ARG(batch >= 0 && batch < g->n_batches, "q4c_grid_batch_spinors: batch out of range");
  const q4c_tables* t = g->tables;
  // Algorithm 1 with the relation table "spinor function -> scalar functions
  // of its radial shell": the batch's local scalar functions are all the
  // functions of its active centres, so a global spinor function (centre c,
  // index mu within the atom) is present exactly when c is active.  The
  // centres are visited in ascending order, each spinor function once.
  int cnt = 0;
  for (int a = g->h_bat_atom_ptr[batch]; a < g->h_bat_atom_ptr[batch + 1]; ++a) {
    const int c = g->h_bat_atoms[a];
    const int sp = g->h_c_sp[c];
    const int m = t->h_spn0[sp + 1] - t->h_spn0[sp];
    for (int mu = 0; mu < m; ++mu, ++cnt) {
      if (centre) centre[cnt] = c;
      if (spinor) spinor[cnt] = mu;
    }
  }
  *n = cnt;
  return Q4C_OK;
}
