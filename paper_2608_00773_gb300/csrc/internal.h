// Internal declarations of the Q4C GB300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/q4c.h"
#include "df.cuh"

namespace q4c {

constexpr int kMaxL = 4;
constexpr int kMaxBatch = 1024;
constexpr int kDPitch = 352;  // points per batch row of the D = w v table (>= 32 * ceil(341 / 32))
// batch-size buckets of the split path's tile-shape choice: n_b <= 32, 64,
// 128 and above
constexpr int kTileBuckets = 4;
constexpr int kBucketNb[kTileBuckets] = {32, 64, 128, 1 << 30};
inline int tile_bucket(int64_t nb) {
  int k = 0;
  while (k + 1 < kTileBuckets && nb > kBucketNb[k]) ++k;
  return k;
}

// Distance of a point from a centre as every decision on it is taken (is the
// point inside the cutoff sphere r < r_c, is it below the first knot r <
// r_min): the squares summed as (dx dx + dy dy) + dz dz, each operation
// rounded on its own (no fused multiply-add), then a correctly rounded square
// root.  The radial functions' gradients jump at r_c and at r_min, so a point
// within rounding of either sphere must land on the same side in every path
// and in a plain FP64 evaluation of the same formula.
__host__ __device__ inline double centre_distance(double dx, double dy, double dz) {
#ifdef __CUDA_ARCH__
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
#else
  volatile double xx = dx * dx, yy = dy * dy, zz = dz * dz;  // stored: no contraction into an FMA
  volatile double s = xx + yy;
  return std::sqrt(s + zz);
#endif
}

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
#define Q4C_CHECK_ARG(cond, msg)          \
  do {                                    \
    if (!(cond)) {                        \
      ::q4c::set_error(msg);              \
      return Q4C_EINVAL;                  \
    }                                     \
  } while (0)
#define Q4C_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      ::q4c::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                 \
      return e_ == cudaErrorMemoryAllocation ? Q4C_ENOMEM : Q4C_ECUDA;                      \
    }                                                                                       \
  } while (0)

// ------------------------------------------------------- instrumentation
// Records CUDA events around one kernel launch on `s` while profiling is on.
class KernelScope {
 public:
  KernelScope(const char* name, cudaStream_t s);
  ~KernelScope();
 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t e0_ = nullptr;
};

// ----------------------------------------------------- device-side views
// Radial tables and species data as seen by kernels (passed by value).
struct DevBasis {
  const double* coef;    // [n_rad_tot][n_log-1][4] cubic in s on each interval
  const double* g0;      // [n_rad_tot] g = u/r^(l+1) below r_min
  const int* rad_l;      // [n_rad_tot]
  const int* sp_rad0;    // [n_species] first radial of each species
  const int* sp_nrad;    // [n_species]
  const int* sp_nfn;     // [n_species]
  double r_c, r_min, inv_rmin, inv_h;
  int n_log;
};

// Double-float views for the split path's basis evaluation.
struct DfTables {
  const float4* coef;     // [n_rad_tot][n_log-1][2]: (c0, c1), (c2, c3) as (hi, lo) pairs
  const df* g0;           // [n_rad_tot]
  const df* inv_knot;     // [n_log] 1 / r_k
  const df* pts;          // [n_points][3] kept points (batch order)
  const df* atoms;        // [n_centres][3] centre positions (atoms and periodic images)
  df inv_h_df;
  float inv_h, inv_rmin, rmin2, rc2;  // FP32 copies: 1/h, 1/r_min, r_min^2, r_c^2
};

// Grid, batches and pattern as seen by kernels.
struct DevGrid {
  const double *x, *y, *z, *w;  // kept points, batch order (SoA)
  const double* atom_xyz;       // [n_atoms][3] cell-0 atoms
  const int* atom_sp;           // [n_atoms]
  const double* c_xyz;          // [n_centres][3] centres: atoms and, in a periodic cell, images
  const int* c_sp;              // [n_centres] species of each centre
  const int64_t* pt_ptr;        // [n_batches+1]
  const int* bat_atom_ptr;      // [n_batches+1] into bat_atoms
  const int* bat_atoms;         // active centres, ascending
  const int* bat_atom_fn0;      // local index of each active centre's first function
  const int64_t* bat_fn_ptr;    // [n_batches+1] prefix of n_b
  const int* fn_info;           // [sum n_b] (local centre << 16) | index within its atom
  const int64_t* bat_pair_ptr;  // [n_batches+1] into pair_off (n_a^2 per batch)
  const int64_t* pair_off;      // value offset of the block of the centre pair (a, b) or -1
  const int64_t* bat_idx_ptr;   // [n_batches+1] into bat_idx (n_b^2 per batch)
  int* bat_idx;                 // value offset of element (i, j) of the batch, or -1 (one wave, filled per call)
  int n_atoms;
  unsigned long long wait_ns;   // limit of the tensor kernels' bounded work waits (q4c_set_wait_limit_ns)
};

// the work-wait limit that q4c_set_wait_limit_ns last set (1 s by default)
unsigned long long work_wait_limit_ns();

}  // namespace q4c

// ------------------------------------------------------------ handles
struct q4c_tables {
  int n_species = 0;
  std::vector<int> n_rad, rad0, nfn, rad_l;
  std::vector<double> alpha;
  double r_c = 0, r_on = 0, r_min = 0, h = 0;
  int n_log = 0;
  std::vector<double> h_coef;  // host copy [n_rad_tot][n_log-1][4]
  std::vector<double> h_g0;
  // per-column operator (q4c_tables_set_columns): eps and the spline
  // coefficients of V per radial function, [n_rad_tot] and [n_rad_tot][n_log-1][4]
  double* d_col_eps = nullptr;
  double* d_col_coef = nullptr;
  float4* d_col_coef_df = nullptr;  // the same coefficients as FP32 pairs (split path)
  // device
  double* d_coef = nullptr;
  double* d_g0 = nullptr;
  int *d_rad_l = nullptr, *d_sp_rad0 = nullptr, *d_sp_nrad = nullptr, *d_sp_nfn = nullptr;
  int device = 0;
  // double-float copies for the split path
  float4* d_coef_df = nullptr;
  q4c::df* d_g0_df = nullptr;
  q4c::df* d_inv_knot_df = nullptr;
  // scalar -> spinor relation tables (spinor.cu): per species the first
  // spinor index (twice the first scalar function), and per spinor function
  // its radial index, kappa and 2 m_j; device column and row views of G
  std::vector<int> h_spn0, h_spn_radial, h_spn_kappa, h_spn_two_mj;
  // per radial function the one kappa whose spinors it carries, 0 for both
  // (q4c_tables_set_kappa; empty: both for every radial); with a selection
  // the spinor counts differ from twice the scalar counts, so the row view
  // is indexed by the scalar-spin offsets h_ss0 and spinor blocks are laid
  // out by their own offsets
  std::vector<int> h_kappa_sel, h_ss0;
  int* d_ss0 = nullptr;
  int* d_spn0 = nullptr;
  void* d_spn_col = nullptr;
  void* d_spn_row = nullptr;
  q4c::DevBasis view() const;
  q4c::DfTables df_view() const;
};

struct q4c_grid {
  const q4c_tables* tables = nullptr;
  int device = 0;
  int n_atoms = 0, n_basis = 0, max_nb = 0, max_np = 0, max_na = 0;
  int64_t n_pts = 0, n_batches = 0, n_blocks = 0, nnz = 0;
  double flops_alg = 0, sum_np_nb = 0;
  // host copies
  std::vector<double> h_xyz, h_w;
  std::vector<int64_t> h_pid, h_pt_ptr, h_blk_ptr, h_blk_off, h_bat_fn_ptr;
  std::vector<int> h_blk_col, h_bat_atom_ptr, h_bat_atoms, h_atom_sp, h_atom_fn0, h_nf_atom;
  std::vector<double> h_atom_xyz;
  // centres: c = cell * n_atoms + atom, cells in lexicographic order of
  // T in [-n_shell, n_shell]^3 (one cell, T = 0, for a molecule)
  int n_centres = 0, n_shell = 0, cell_side = 1;
  std::vector<double> h_c_xyz;
  std::vector<int> h_c_sp, h_blk_shift;  // h_blk_shift [n_blocks][3]
  // k-pattern: atom pairs with some block; each covers the pattern blocks [q0, q1)
  std::vector<int64_t> h_kblk_ptr, h_kblk_off, h_kblk_q0, h_kblk_q1;
  std::vector<int> h_kblk_col;
  int64_t nnz_k = 0;
  int* d_blk_shift = nullptr;
  int64_t *d_kblk_q0 = nullptr, *d_kblk_q1 = nullptr, *d_kblk_off = nullptr;
  double* d_c_xyz = nullptr;
  int* d_c_sp = nullptr;
  // device: points
  double *d_xyz = nullptr, *d_x = nullptr, *d_y = nullptr, *d_z = nullptr, *d_w = nullptr;
  q4c::df* d_pts_df = nullptr;    // [n_pts][3]
  q4c::df* d_atoms_df = nullptr;  // [n_centres][3]
  // device: atoms and batches
  double* d_atom_xyz = nullptr;
  int *d_atom_sp = nullptr, *d_atom_fn0 = nullptr;
  int64_t* d_pt_ptr = nullptr;
  int *d_bat_atom_ptr = nullptr, *d_bat_atoms = nullptr, *d_bat_atom_fn0 = nullptr;
  int64_t* d_bat_fn_ptr = nullptr;
  int* d_fn_info = nullptr;
  int64_t *d_bat_pair_ptr = nullptr, *d_pair_off = nullptr;
  // device: pattern
  int64_t* d_blk_off = nullptr;
  int *d_blk_row = nullptr, *d_blk_col = nullptr, *d_blk_T = nullptr;
  int* d_blk_role = nullptr;  // mirror role: 1 canonical (copied to its partner), 2 own partner, 0 target
  // FP64 path: waves of batches whose basis tiles fit the scratch buffer
  std::vector<int64_t> wave_b0;            // [n_waves+1] batch ranges
  std::vector<int64_t> h_scr_off;          // [n_batches] offset (doubles) within its wave
  int64_t* d_scr_off = nullptr;
  std::vector<int64_t> wave_t0;            // [n_waves+1] ranges into the tile list
  int4* d_tiles = nullptr;                 // (batch, ti, tj, 0), ti <= tj, 32x32 tiles
  std::vector<int64_t> colt_w0;            // [n_waves+1] ranges into d_col_tiles
  int4* d_col_tiles = nullptr;             // per-column operator, FP64 path: every 32x32 tile pair (batch, ti, tj, 0)
  double* d_scratch = nullptr;
  int64_t scratch_doubles = 0;
  // split path: work items (batch, output, ti, tj) per wave, sorted by cost,
  // per-batch column exponents, persistent-kernel counters, status word
  int* d_sched = nullptr;
  int* d_counter = nullptr;                // [n_waves]
  std::vector<int64_t> split_w0;           // [n_waves+1] ranges into d_split_items
  // [n_waves][kTileBuckets+1] item ranges of each batch-size bucket (the
  // items of a wave are grouped by bucket), and the same for d_col_items
  std::vector<int64_t> split_bw0, col_bw0;
  int split_ks[4] = {1, 1, 1, 1};          // K-steps of 16 points per pipeline stage, per bucket (tuner)
  double tune_ms[4][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};  // tuner timings per bucket and shape
  int rd_ks = 1;                           // K-steps per stage of the density/adjoint kernel (tuner)
  double rd_tune_ms[2] = {-1, -1};         // tuner timings of the adjoint with one and two K-steps
  int4* d_split_items = nullptr;
  std::vector<int64_t> col_w0;             // [n_waves+1] ranges into d_col_items
  int4* d_col_items = nullptr;             // per-column operator: (batch, 5, ti, tj), every tile pair
  float* d_split_mag = nullptr;            // [items of the largest wave][128] rounding constants
  void* d_tmaps = nullptr;                 // [2][n_batches] 3-D TMA maps (points, functions, quantity) of the
                                           // tiles: boxes 16 x 64 (products), 64 x 16 (density, adjoint)
  float2* d_dpad = nullptr;                // [n_batches][kDPitch] D = w v as (hi, lo), zero past n_p
  int* d_colexp = nullptr;                 // [8 * sum n_b]
  std::vector<int64_t> rd_w0;              // [n_waves+1] ranges into d_rd_items
  int2* d_rd_items = nullptr;              // (batch, 64-point tile) for density/adjoint
  int* d_rowexp = nullptr;                 // [n_points][4] per-point exponents
  unsigned char* d_gsl = nullptr;          // G' digit blocks of one wave (density/adjoint)
  unsigned char* d_gzero = nullptr;        // one zero G' digit block (12 KB)
  int64_t* d_gsl_off = nullptr;            // [n_batches] byte offsets into d_gsl (per wave)
  int64_t gsl_bytes = 0;
  int64_t idx_entries = 0;                 // size of the per-wave dense offset tables
  int64_t* d_bat_idx_ptr = nullptr;
  int* d_bat_idx = nullptr;                // per batch n_b x n_b value offsets (-1 outside)
  unsigned* d_status = nullptr;            // bit 0: a bounded wait expired
  float2* d_gdf = nullptr;                 // [10][nnz] FP32-pair copies of the density (0-4) and adjoint (5-9) matrices
  // per pattern block q, at cm_off[q]: the largest |value| of each of its
  // nf_B columns, then of each of its nf_A rows (FP32, rounded up), for each
  // of the ten matrices of d_gdf ([10][cm_total]); the G' pre-pass bounds a
  // batch column's largest element from them
  int64_t* d_cm_off = nullptr;             // [n_blocks + 1]
  int64_t cm_total = 0;
  float* d_cm = nullptr;
  int* d_pair_blk = nullptr;               // per batch, n_a^2: pattern block of centre pair (a, b) or -1
  int64_t split_ws_bytes = 0;
  void* d_split_ws = nullptr;
  q4c::DevGrid view() const;
};

namespace q4c {
// fp64.cu
q4c_status integrate_fp64(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* out,
                          cudaStream_t s);
q4c_status density_fp64(const q4c_tables* t, const q4c_grid* g, const double* P, double* n, cudaStream_t s);
q4c_status backward_fp64(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* G, double* dLdv,
                         cudaStream_t s, bool weighted = true);
q4c_status basis_eval(const q4c_tables* t, const q4c_grid* g, int64_t n_pts, const double* xyz, double* phi,
                      double* grad, cudaStream_t s);
q4c_status mirror_and_spinor(const q4c_grid* g, const q4c_matrices* out, cudaStream_t s);
q4c_status launch_basis_tiles(const q4c_tables* t, const q4c_grid* g, int64_t b0, int64_t b1, const double* v,
                              int* colexp, cudaStream_t s);
// fp64.cu: the per-column operator of Eq. 19 in FP64
q4c_status integrate_columns_fp64(const q4c_tables* t, const q4c_grid* g, const double* v, double* F,
                                  cudaStream_t s);
// grid.cu: dense per-batch offset tables of the batches [b0, b1) (one wave)
q4c_status launch_fill_idx(const q4c_tables* t, const q4c_grid* g, int64_t b0, int64_t b1, cudaStream_t s);

// basis_df.cu
// spinor.cu: scalar -> spinor relation tables of a set of species
q4c_status build_spinor_tables(q4c_tables* t);
// nq = 4: Phi, X, Y, Z tiles; nq = 1: Phi alone; nq = 2: Phi and the
// per-column operator's Psi = (v + eps_j - V_j) phi_j with D = w
q4c_status launch_basis_df(const q4c_tables* t, const q4c_grid* g, int64_t b0, int64_t b1, const double* v,
                           int* colexp, int* rowexp, int nq, cudaStream_t s, float2* dpad = nullptr);
// rowdot.cu
q4c_status density_split(const q4c_tables* t, const q4c_grid* g, const double* P, double* n, cudaStream_t s);
q4c_status backward_split(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* G, double* dLdv,
                          cudaStream_t s, bool weighted = true);
// split.cu
q4c_status integrate_split(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* out,
                           cudaStream_t s);
q4c_status integrate_columns_split(const q4c_tables* t, const q4c_grid* g, const double* v, double* F,
                                   cudaStream_t s);
// per-wave pieces of the split path, for the fused pass (fused.cu)
q4c_status products_wave(const q4c_grid* g, int wv, const q4c_matrices* out, cudaStream_t s);
q4c_status rowdot_prepare(const q4c_grid* g, const double* const mats[5], int slot0, const float2* mdf[5],
                          unsigned* present, cudaStream_t s);
q4c_status rowdot_wave(const q4c_grid* g, int wv, int mode, const float2* const mdf[5], unsigned present,
                       bool weighted, double* out, cudaStream_t s);
// per-wave pieces of the FP64 path
q4c_status products_fp64_wave(const q4c_grid* g, int wv, const double* v, const q4c_matrices* out,
                              cudaStream_t s);
q4c_status density_fp64_wave(const q4c_grid* g, int wv, const double* P, double* n, cudaStream_t s);
q4c_status backward_fp64_wave(const q4c_grid* g, int wv, const q4c_matrices* G, double* dLdv, bool weighted,
                              cudaStream_t s);
// split.cu: the tile-shape tuner (stores its choice in the grid); rowdot.cu: its row-dot part
q4c_status autotune_split(const q4c_tables* t, q4c_grid* g, const double* v, cudaStream_t s);
q4c_status autotune_rowdot(q4c_grid* g, double* out, cudaStream_t s);
// the fused pass (fused.cu)
q4c_status scf_pass(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* H,
                    const q4c_matrices* P, double* n, const q4c_matrices* Gm, double* dLdv, bool split,
                    cudaStream_t s);
// grid.cu
q4c_status becke_weights(const double* d_raw_xyz, const double* d_base_w, int64_t n_raw, int pts_per_atom,
                         const double* d_atom_xyz, const double* d_inv_rab, int n_atoms, double r_c, double r_nb,
                         double* d_w, unsigned char* d_near);
}  // namespace q4c
