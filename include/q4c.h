/*
 * q4c.h -- C ABI of the GB300 Q4C real-space integration library.
 *
 * The library evaluates, on one GPU, the order-N real-space integration of
 * the Q4C Hamiltonian-type matrix elements over compact batches of an
 * atom-centred grid (arxiv 2608.00773, Section III A, Eqs. 29-32), the grid
 * density of Eqs. 39-40 and the adjoint of the integration.
 *
 * Conventions for every entry point:
 *   - returns q4c_status (0 = Q4C_OK); on failure q4c_last_error() returns a
 *     message for the calling thread; no C++ exception crosses the ABI;
 *   - opaque handles (q4c_tables, q4c_grid) are library-owned and released
 *     with their *_destroy call;
 *   - arrays marked "host" are read during the call only; arrays marked
 *     "device" are caller-owned CUDA device memory on the current device;
 *   - q4c_stream is a cudaStream_t (NULL = legacy default stream).  Compute
 *     calls enqueue work on it and return without synchronising unless
 *     stated otherwise;
 *   - units are Bohr and Hartree; matrices are FP64.
 *
 * Matrix layout ("block pattern"): rows and columns are atoms; block (A, B)
 * exists iff |R_A - R_B| < 2 r_cut, stored in CSR order over A
 * (blk_ptr[n_atoms+1], blk_col[n_blocks], sorted by B) with the values of
 * block q a dense row-major nf_A x nf_B array starting at blk_off[q]
 * (blk_off[n_blocks] = nnz).  Basis functions of an atom are ordered by
 * radial function of its species, then m = -l..l.
 */
#ifndef Q4C_H
#define Q4C_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define Q4C_API __attribute__((visibility("default")))
#else
#define Q4C_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum q4c_status {
  Q4C_OK = 0,
  Q4C_EINVAL = 1,        /* invalid argument (NULL, size, range, mismatch) */
  Q4C_ENOMEM = 2,        /* host or device allocation failed */
  Q4C_ECUDA = 3,         /* a CUDA runtime call failed */
  Q4C_ETIMEOUT = 4,      /* a bounded device wait expired */
  Q4C_EUNSUPPORTED = 5   /* valid request outside what is implemented */
} q4c_status;

typedef enum q4c_precision {
  Q4C_FP64 = 0,   /* every product and sum in FP64 */
  Q4C_SPLIT = 1   /* batch products as exact BF16 slice products with FP32
                     accumulation on tcgen05 tensor cores, recombined and
                     summed across batches in FP64 (Ozaki-type splitting) */
} q4c_precision;

typedef struct CUstream_st* q4c_stream; /* = cudaStream_t */
typedef struct q4c_tables q4c_tables;
typedef struct q4c_grid q4c_grid;

/* ---------------------------------------------------------------------- */
/* Radial tables (Eq. 12: phi = u_l(r)/r Y_lm, u_l tabulated numerically on a
 * one-dimensional logarithmic grid).
 *
 * Radial function k of a species: u(r) = r^(l+1) exp(-alpha r^2) c(r), with
 * c(r) = 1 for r <= r_on, 0 for r >= r_cut, 1 - (10s^3 - 15s^4 + 6s^5),
 * s = (r - r_on)/(r_cut - r_on), in between; tabulated at
 * r_k = r_min (r_cut/r_min)^(k/(n_log-1)) and interpolated by a natural cubic
 * spline in the grid index; below r_min u = u(r_min) (r/r_min)^(l+1).
 * ---------------------------------------------------------------------- */
typedef struct q4c_basis_desc {
  int32_t n_species;
  const int32_t* n_rad;  /* host [n_species]: radial functions per species (>= 1) */
  const int32_t* l;      /* host [sum n_rad]: species-major angular momenta, 0 <= l <= 4 */
  const double* alpha;   /* host [sum n_rad]: Gaussian exponents (> 0) */
  double r_cut;          /* support radius of every function (> r_on) */
  double r_on;           /* start of the cutoff ramp (> r_min) */
  double r_min;          /* first logarithmic knot (> 0) */
  int32_t n_log;         /* knots (>= 4) */
} q4c_basis_desc;

/* Builds the spline tables on the host in FP64 and uploads them to the
 * current device.  *out receives a new handle.  EINVAL on a bad descriptor,
 * EUNSUPPORTED for l > 4, ENOMEM/ECUDA on allocation/copy failure. */
Q4C_API q4c_status nao_tabulate(const q4c_basis_desc* desc, q4c_tables** out);

/* The same tables from radial functions given by their values at the knots
 * instead of (l, alpha): knots host [sum n_rad][n_log], u(r_k) with
 * r_k = r_min (r_cut/r_min)^(k/(n_log-1)) (phi = u(r)/r Y_lm, so u ~ r^(l+1)
 * at small r; below r_min u = u(r_min) (r/r_min)^(l+1)); desc->alpha may be
 * NULL.  This is how the small-component functions phi^S = Q(r)/r Y_(l~m~)
 * (Eq. 12b) enter: a tables handle of the Q radials with l~ = l +- 1.
 * Errors as nao_tabulate. */
Q4C_API q4c_status nao_tabulate_knots(const q4c_basis_desc* desc, const double* knots, q4c_tables** out);
Q4C_API void q4c_tables_destroy(q4c_tables* tables);

/* Host copy of the cubic coefficients of radial function k (species-major
 * index): coef[n_log-1][4] with u(s) = c0 + c1 s + c2 s^2 + c3 s^3 on the
 * interval [k, k+1] of the index variable, s = t - k. */
Q4C_API q4c_status q4c_tables_export(const q4c_tables* tables, int32_t radial, double* coef_host);

/* ---------------------------------------------------------------------- */
/* Integration grid, partition and batches (Section III A, Figs. 1-2,
 * Eqs. 31-32 and the reduced index set nnz(B_v)).
 *
 * Per atom: n_rad_shells Gauss-Chebyshev (second kind) radial shells mapped
 * by r = R (1+x)/(1-x), times Gauss-Legendre(n_theta) in cos(theta) times
 * n_phi uniform azimuths phi_b = (b + 1/2) 2 pi / n_phi.  Point weights
 * w = w_rad w_ang p_A(r), p_A the Becke (or, by the descriptor's partition
 * field, Stratmann) partition, no size adjustment, over the atoms within
 * r_nb of the point.  Points farther than
 * r_cut from every atom, or with w = 0, are dropped.  The kept points are
 * split into batches by recursive median bisection along the longest
 * bounding-box axis until a batch holds <= batch_max points; the raw point
 * id ((atom*n_rad + shell)*n_theta + theta)*n_phi + phi is kept.
 *
 * Periodic cells (Eqs. 24-25, the real-space H(T) before any k-phase): with
 * a lattice, the centres are the atoms and their images R_A + T.L, T an
 * integer triple in [-n_shell, n_shell]^3 (n_shell must cover r_nb + r_cut
 * around the cell).  Grid points come from the cell-0 atoms only; the
 * partition, the pruning and the active-function sets run over all centres.
 * The block pattern becomes (A, B, T) for cell-0 atoms A, B with
 * |R_A - R_B - T.L| < 2 r_cut, T in [-2 n_shell, 2 n_shell]^3, sorted by
 * (A, B, T); a pair of centres (A, Ta), (B, Tb) active at a point adds into
 * block (A, B, Tb - Ta).  Without a lattice everything reduces to the
 * molecule (T = 0).
 *
 * Batched molecules (many independent molecules in one grid and one call):
 * with mol_atom_ptr the atoms form n_molecules consecutive ranges.  Each
 * molecule is partitioned, pruned, batched and screened on its own atoms
 * only (its Becke neighbour sets, active sets and pattern blocks never
 * include another molecule's atoms, wherever the molecules sit), so every
 * batch holds one molecule's points and the molecule's blocks (its atom
 * rows of the pattern) are what integrating it alone would give.  Not
 * combined with a lattice.
 * ---------------------------------------------------------------------- */
typedef struct q4c_grid_desc {
  int32_t n_atoms;
  const double* xyz;       /* host [n_atoms][3] Bohr */
  const int32_t* species;  /* host [n_atoms], indices into the tables' species */
  int32_t n_rad_shells;    /* radial shells per atom (>= 1) */
  double R;                /* radial map scale, Bohr (> 0) */
  int32_t n_theta, n_phi;  /* angular product grid (>= 1 each) */
  double r_nb;             /* Becke neighbour radius, Bohr (> 0) */
  int32_t batch_max;       /* maximum points per batch (1..1024) */
  const double* lattice;   /* host [3][3] lattice vectors as rows (Bohr), or NULL for a molecule */
  int32_t n_shell;         /* image shell of a periodic cell (0..8); ignored without a lattice */
  int32_t n_molecules;     /* independent molecules (0 or 1: one system) */
  const int32_t* mol_atom_ptr; /* host [n_molecules+1]: atom ranges, 0 = p[0] < p[1] < ... = n_atoms;
                                  NULL when n_molecules <= 1 */
  int32_t partition;       /* cell function of the partition of unity: 0 Becke (1988, three
                              iterations; a zeroed descriptor), 1 Stratmann, Scuseria and Frisch
                              (1996: odd degree-7 polynomial, a = 0.64, exactly 1 and 0 beyond);
                              no size adjustment in either */
} q4c_grid_desc;

/* Builds the grid (raw points and base weights on the host, Becke weights in
 * an FP64 kernel, pruning, bisection, active-function lists and the block
 * pattern) and keeps everything resident on the current device.
 * Synchronous.  EINVAL on a bad descriptor or an empty grid. */
Q4C_API q4c_status grid_partition(const q4c_grid_desc* desc, const q4c_tables* tables, q4c_grid** out);
Q4C_API void q4c_grid_destroy(q4c_grid* grid);

typedef struct q4c_grid_info {
  int64_t n_points;    /* kept points */
  int64_t n_batches;
  int64_t n_blocks;    /* pattern blocks */
  int64_t nnz;         /* values per matrix on the pattern */
  int32_t n_atoms;
  int32_t n_basis;
  int32_t max_nb;      /* largest |nnz(B_v)| over batches */
  int32_t max_np;      /* largest batch */
  double flops_alg;    /* sum over batches of 14 n_p n_b^2 (the integration's
                          seven n_b x n_p x n_b products) */
  double sum_np_nb;    /* sum over batches of n_p n_b */
  int64_t scratch_bytes; /* device workspace held by the grid */
} q4c_grid_info;
Q4C_API q4c_status q4c_grid_get_info(const q4c_grid* grid, q4c_grid_info* info);

/* Host copies of the grid (points in batch order).  Any pointer may be NULL.
 * xyz[n_points][3], w[n_points], point_id[n_points], batch_ptr[n_batches+1],
 * batch_atom_ptr[n_batches+1], batch_atoms[batch_atom_ptr[n_batches]]
 * (active atoms per batch, ascending), blk_ptr[n_atoms+1],
 * blk_col[n_blocks], blk_off[n_blocks+1].  Synchronous. */
Q4C_API q4c_status q4c_grid_export(const q4c_grid* grid, double* xyz, double* w, int64_t* point_id,
                           int64_t* batch_ptr, int64_t* batch_atom_ptr, int32_t* batch_atoms,
                           int64_t* blk_ptr, int32_t* blk_col, int64_t* blk_off);

/* Host copy of the lattice shift T of every pattern block, shifts[n_blocks][3]
 * (all zero for a molecule).  In a periodic grid the batch_atoms of
 * q4c_grid_export are centre indices, cell * n_atoms + atom with the cells in
 * lexicographic order of T in [-n_shell, n_shell]^3.  Synchronous. */
Q4C_API q4c_status q4c_grid_export_shifts(const q4c_grid* grid, int32_t* shifts);

/* k-pattern of a grid: the atom pairs (A, B) that have at least one pattern
 * block (A, B, T), CSR by atom rows (kblk_ptr[n_atoms+1], kblk_col[],
 * kblk_off[n+1] value offsets of dense nf_A x nf_B blocks); *nnz_k = values
 * per k-point.  Any pointer may be NULL.  Synchronous.  For a molecule it is
 * the pattern itself. */
Q4C_API q4c_status q4c_grid_kpattern(const q4c_grid* grid, int64_t* nnz_k, int64_t* kblk_ptr, int32_t* kblk_col,
                             int64_t* kblk_off);

/* k-phase fold of a real-space matrix on the pattern (Eqs. 24-26, 36):
 *   H(k)_AB = sum_T exp(2 pi i k.T) H(T)_AB
 * for n_k k-points in reduced coordinates (k_host[n_k][3], fractions of the
 * reciprocal lattice vectors; T the integer shifts of q4c_grid_export_shifts).
 * H_dev device [nnz]; Hk_dev device complex128 [n_k][nnz_k] (interleaved re,
 * im) on the k-pattern, overwritten.  FP64.  Stream-ordered. */
Q4C_API q4c_status q4c_kfold(const q4c_grid* grid, const double* H_dev, int32_t n_k, const double* k_host,
                     double* Hk_dev, q4c_stream stream);

/* Device pointers (grid-owned, read-only) to the kept points in batch order:
 * xyz[n_points][3] and w[n_points], so callers can build v on the device. */
Q4C_API q4c_status q4c_grid_points(const q4c_grid* grid, const double** xyz_dev, const double** w_dev,
                           int64_t* n_points);

/* ---------------------------------------------------------------------- */
/* Matrices on the block pattern. */
typedef struct q4c_matrices {
  double* V;    /* device [nnz] */
  double* W0;   /* device [nnz] */
  double* SOx;  /* device [nnz] */
  double* SOy;  /* device [nnz] */
  double* SOz;  /* device [nnz] */
  double* spinor_SS; /* device [8*nnz] or NULL: complex128 (re, im) SS blocks,
                        block q a row-major (2 nf_A) x (2 nf_B) matrix at
                        4*blk_off[q], row 2i+s, column 2j+s' */
} q4c_matrices;

/* Integration (Eqs. 29-32 with F = v; the SS block of Eq. 16 read with the
 * kinetic-balance small component, (s.a)(s.b) = a.b + i s.(a x b)):
 *   V_ij   = sum_p w_p v_p phi_i phi_j
 *   W0_ij  = sum_p w_p v_p grad phi_i . grad phi_j
 *   SOk_ij = sum_p w_p v_p (grad phi_i x grad phi_j)_k
 * and, if out->spinor_SS != NULL, the 2x2 complex blocks
 *   [[W0 + i SOz, SOy + i SOx], [-SOy + i SOx, W0 - i SOz]].
 * v_dev: device [n_points] in batch order.  Outputs are overwritten (not
 * accumulated).  V and W0 come out exactly symmetric, SO exactly
 * antisymmetric.  EINVAL on NULL arguments or handles of different setups. */
Q4C_API q4c_status q4c_integrate(const q4c_tables* tables, const q4c_grid* grid, const double* v_dev,
                         q4c_precision prec, const q4c_matrices* out, q4c_stream stream);

/* Density (Eqs. 39-40): n_p = sum_ij P_ij phi_i(p) phi_j(p), P_dev device
 * [nnz] on the block pattern (any P; only its symmetric part contributes),
 * n_dev device [n_points] in batch order, overwritten.  Q4C_SPLIT takes
 * batches of up to 4096 active functions (above 512 the sum over i runs in
 * exact segments of 512 combined in FP64), Q4C_FP64 up to 7264;
 * Q4C_EUNSUPPORTED beyond.  The split limit holds for q4c_density_full and
 * q4c_integrate_backward too; their FP64 path takes up to 5811. */
Q4C_API q4c_status q4c_density(const q4c_tables* tables, const q4c_grid* grid, const double* P_dev,
                       q4c_precision prec, double* n_dev, q4c_stream stream);

/* Density with the gradient (small-component) terms (the density counterpart
 * of the W0 and W_SO integrands, Eqs. 4, 21, 39-40 with the kinetic-balance
 * small component of R1):
 *   n_p = sum_ij [ P^V_ij phi_i phi_j + P^W0_ij grad phi_i . grad phi_j
 *                  + sum_k P^SOk_ij (grad phi_i x grad phi_j)_k ](p)
 * P->V..P->SOz device [nnz] on the block pattern, NULL slots count as zero
 * (only the symmetric part of P^V, P^W0 and the antisymmetric part of P^SOk
 * contribute); spinor_SS is ignored.  n_dev device [n_points], overwritten.
 * With only the V slot it equals q4c_density. */
Q4C_API q4c_status q4c_density_full(const q4c_tables* tables, const q4c_grid* grid, const q4c_matrices* P,
                            q4c_precision prec, double* n_dev, q4c_stream stream);

/* ------------------------------------------------- per-column operator
 * The large-component matrix of Eq. 19 in the scalar form, where every
 * element carries the eigenvalue and defining potential of the radial
 * function of its column function j:
 *   F_ij = sum_p w_p phi_i(p) [eps_j - V_j(|p - R_j|) + v_p] phi_j(p)
 * (R_j the centre of j, an atom or a periodic image).  F is not symmetric. */

/* Stores eps (host [sum n_rad], species-major, Hartree) and V (host
 * [sum n_rad][n_log]: values at the radial knots r_k = r_min (r_cut/r_min)^(k/(n_log-1)),
 * interpolated by a natural cubic spline in the knot index; below r_min the
 * first knot's value, from r_cut on the last one's) with the tables,
 * replacing earlier ones.  Synchronous.  EINVAL on NULL arguments. */
Q4C_API q4c_status q4c_tables_set_columns(q4c_tables* tables, const double* eps, const double* knots);

/* F on the grid's block pattern (device [nnz], overwritten; every element
 * of every block, no symmetry used), v_dev device [n_points] in batch order.
 * prec Q4C_FP64: FP64 tiles and products.  Q4C_SPLIT: the tensor-core path
 * of q4c_integrate, F = (w Phi)^T Psi per batch with
 * Psi_pj = (v_p + eps_j - V_j(r_pj)) phi_j(p) formed in double-float and
 * sliced into six BF16 digits (~1e-12 relative; EUNSUPPORTED above 341
 * points per batch).  EINVAL without q4c_tables_set_columns.
 * Stream-ordered, with one host synchronisation per wave of batches. */
Q4C_API q4c_status q4c_integrate_columns(const q4c_tables* tables, const q4c_grid* grid, const double* v_dev,
                                 q4c_precision prec, double* F_dev, q4c_stream stream);

/* ---------------------------------------------------------------- spinors
 * Scalar -> spinor transformation (Section II, Eqs. 9-14; Section III A,
 * Eqs. 33-34, 37-38; Appendix A).  Spinor basis of an atom: per radial
 * function (angular momentum l) in the species' order, j = l - 1/2
 * (kappa = l, only for l > 0) then j = l + 1/2 (kappa = -l - 1), m_j = -j..j
 * ascending; 2 (2l + 1) spinor functions per radial function, twice the
 * atom's scalar functions.  Spinor function mu = sum G_(2t+s),mu phi_t eta_s
 * with the Clebsch-Gordan coefficients of Eq. 10 and the complex harmonics
 * Y~_l^m (Condon-Shortley phase) written in the real harmonics of
 * Appendix B.  Spinor blocks are complex128 (re, im), block q of the pattern
 * a row-major (2 nf_A) x (2 nf_B) matrix at 4*blk_off[q] (the layout of
 * q4c_matrices.spinor_SS, rows spinor functions of atom A).
 *
 * With a kappa selection (q4c_tables_set_kappa) a radial function carries the
 * spinor functions of one kappa only (2|kappa| of them); the spinor blocks are
 * then n_spinor(A) x n_spinor(B) matrices laid out consecutively in pattern
 * order (q4c_spinor_nnz gives the total), and the row view of G keeps the
 * scalar-spin index 2t + s of these tables.  Small-component tables (radials
 * Q, Eq. 12b; nao_tabulate_knots) with kappa~ = -kappa of each parent,
 * ordered per parent as kappa = l then kappa = -l - 1, have exactly the
 * spinor functions of the large-component tables in the same order (the
 * small component of spinor (kappa, m_j) is i Q/r Upsilon_(-kappa, m_j),
 * Eq. 11), so their blocks share the large component's layout. */

/* Per radial function (host [sum n_rad], species-major) the kappa whose
 * spinors it carries: 0 for both (the default), -l-1 (j = l + 1/2) or, for
 * l > 0, l (j = l - 1/2); kappa = NULL (or all zeros) restores the default.
 * Rebuilds the tables' spinor relation tables; synchronous.  Grids keep
 * working with the new selection.  EINVAL on a kappa that does not belong to
 * its radial function's l. */
Q4C_API q4c_status q4c_tables_set_kappa(q4c_tables* tables, const int32_t* kappa);

/* Number of complex spinor elements of the grid's pattern under the tables'
 * spinor basis (4 nnz without a kappa selection).  Synchronous. */
Q4C_API q4c_status q4c_spinor_nnz(const q4c_tables* tables, const q4c_grid* grid, int64_t* n);

/* Quantum numbers of the spinor functions of one species: *n = 2 x its
 * scalar function count (without a kappa selection); radial[i] (index of the radial function within the
 * species), kappa[i], two_mj[i] = 2 m_j, host arrays of *n entries, any may
 * be NULL.  Synchronous, no device work. */
Q4C_API q4c_status q4c_spinor_basis(const q4c_tables* tables, int32_t species, int32_t* n, int32_t* radial,
                            int32_t* kappa, int32_t* two_mj);

/* Eqs. 33-34, per pattern block (A, B, T):
 *   HL = G_A^dagger (V x 1) G_B               (large component, from F->V)
 *   HS = G_A^dagger (W0 1 + i SO.sigma) G_B   (kinetic-balance small component,
 *                                              from F->W0, F->SOx..SOz; NULL
 *                                              slots count as zero)
 * F: real device arrays [nnz] on the grid's pattern (q4c_integrate's output,
 * or any real matrix on the pattern, symmetric or not: F->V may be
 * q4c_integrate_columns' F); HL_dev, HS_dev: device double [2 x spinor nnz]
 * (complex128 [4*nnz] without a kappa selection) or NULL to skip,
 * overwritten.  For small-component tables (kappa selection above) HL with
 * F->V = their scalar matrix is the SS spinor block of Eq. 19, e.g.
 * G^S^dagger (F^S x 1) G^S; adding it to the large component's HL gives H+
 * (and with overlap matrices S+).  EINVAL if HL is asked without F->V or HS without any of the
 * small-component slots.  Stream-ordered. */
Q4C_API q4c_status q4c_spinor_transform(const q4c_tables* tables, const q4c_grid* grid, const q4c_matrices* F,
                                double* HL_dev, double* HS_dev, q4c_stream stream);

/* Eqs. 37-38, the reverse map of a spinor density matrix D (device double
 * [2 x spinor nnz], complex128 blocks as above, normally Hermitian: block (B, A, -T)
 * = block (A, B, T)^dagger) to the scalar density matrices of the large and
 * small components:
 *   D'_ab = sum_mu,nu conj(G_a,mu) D_mu,nu G_b,nu,
 *   P->V = P->W0 = Re tr_s D'_ij,  P->SOk = Re(i sum_ss' (sigma_k)_ss' D'_(is)(js'))
 * so that q4c_density(P->V) gives the large-component density and
 * q4c_density_full with (NULL, P->W0, P->SOx, P->SOy, P->SOz) the small one
 * (kinetic-balance reading).  With small-component tables (kappa selection)
 * P->V is the scalar density matrix of the Q functions, and q4c_density on
 * those tables gives the small-component density of Eq. 21.
 * P slots: device [nnz], overwritten; NULL slots are skipped.  Stream-ordered. */
Q4C_API q4c_status q4c_spinor_density_matrices(const q4c_tables* tables, const q4c_grid* grid, const double* D_dev,
                                       const q4c_matrices* P, q4c_stream stream);

/* Algorithm 1 for one batch: the spinor functions present on the batch's
 * local scalar functions (those of its active centres), in ascending global
 * order (centre, then spinor index within the centre's atom).  *n gets the
 * count (twice the batch's n_b without a kappa selection); centre[] and spinor[] (host, *n entries,
 * either may be NULL) the pairs.  Synchronous, no device work. */
Q4C_API q4c_status q4c_grid_batch_spinors(const q4c_grid* grid, int64_t batch, int32_t* n, int32_t* centre,
                                  int32_t* spinor);


/* Adjoint of q4c_integrate for L = <G^V,V> + <G^W0,W0> + sum_k <G^SOk,SOk>:
 *   dLdv_p = w_p sum_M sum_ij G^M_ij f^M_ij(p)
 * with f^V = phi_i phi_j, f^W0 = grad phi_i . grad phi_j,
 * f^SOk = (grad phi_i x grad phi_j)_k; the basis is recomputed, never stored.
 * G->V..G->SOz device [nnz] each, NULL slots count as zero; spinor_SS is
 * ignored.  dLdv_dev device [n_points], overwritten. */
Q4C_API q4c_status q4c_integrate_backward(const q4c_tables* tables, const q4c_grid* grid,
                                  const q4c_matrices* G, q4c_precision prec, double* dLdv_dev,
                                  q4c_stream stream);

/* One pass per SCF step over the grid (the gradient-density row of the
 * method's density update batched with the integration; Eqs. 4, 21, 29-30,
 * 39-40): per wave of batches the basis (Phi and its gradient, Eq. 12 with
 * Appendix B) is evaluated once and feeds, from the same tiles, each part
 * whose arguments are given:
 *   H != NULL:  the integration of v_dev into H (exactly as q4c_integrate:
 *               V, W0, SOx, SOy, SOz [nnz] overwritten, spinor_SS if set);
 *   P != NULL:  the density n_dev[n_points] = sum_M sum_ij P^M_ij f^M_ij(p)
 *               (q4c_density_full; with only P->V it is q4c_density, Eq. 39);
 *   G != NULL:  the adjoint dLdv_dev[n_points] of q4c_integrate_backward.
 * All arrays are device arrays on the grid's pattern or points (batch order),
 * caller-owned; NULL slots inside P or G count as zero.  Each result equals
 * that of its separate call up to the order of the FP64 additions; the saving
 * is the basis evaluation and offset tables the separate calls would repeat.
 * Q4C_EINVAL for a missing array (H without v or an output, P without n_dev,
 * G without dLdv_dev), Q4C_EUNSUPPORTED where the split path's batch limits
 * are exceeded (as for the separate calls). */
Q4C_API q4c_status q4c_scf_pass(const q4c_tables* tables, const q4c_grid* grid, const double* v_dev,
                                const q4c_matrices* H, const q4c_matrices* P, double* n_dev,
                                const q4c_matrices* G, double* dLdv_dev, q4c_precision prec, q4c_stream stream);

/* Tile shapes of the split path's batch products, chosen per batch-size
 * bucket (the active functions n_b of a batch: <= 32, <= 64, <= 128, more;
 * Q4C_TILE_BUCKETS buckets).  A shape is the number of 16-point K-steps one
 * pipeline stage of the tensor-core kernel carries: 1 (four stages in
 * flight) or 2 (two stages of twice the points, half the handshakes per
 * point); the 64-function tiles and their N width (the functions of the B
 * tile rounded up to 16) follow from the batch.  A new grid uses 1 for every
 * bucket.  Not in the paper: a library control of the kernels.
 *
 * q4c_autotune times both shapes on the grid's first wave of batches with
 * potential v_dev (each bucket's products launched once untimed and three
 * times between CUDA events on `stream`, into scratch outputs it allocates
 * and frees), keeps the faster one per bucket in the grid, and synchronises
 * the stream.  The choice applies to every later split-path integration
 * (q4c_integrate, q4c_integrate_columns, q4c_scf_pass) on the grid; results
 * do not depend on it beyond the order of FP64 additions.
 * The density/adjoint kernel (row-dot products over 16-function K-steps)
 * has one such shape per grid, tuned on the same wave with its adjoint; it is
 * addressed as bucket Q4C_TILE_BUCKETS below.
 * q4c_grid_tiling reports a bucket: its largest n_b (4096 for the row-dot
 * kernel), the shape in use, the grid's batches in it (all for the row-dot
 * kernel), and the tuner's mean time per launch for one and two K-steps
 * (-1 if not timed); NULL outputs are skipped.
 * q4c_grid_set_tiling sets a bucket's shape by hand (1 or 2).  Q4C_EINVAL
 * for a bucket outside 0..Q4C_TILE_BUCKETS or another shape. */
#define Q4C_TILE_BUCKETS 4
Q4C_API q4c_status q4c_autotune(const q4c_tables* tables, q4c_grid* grid, const double* v_dev, q4c_stream stream);
Q4C_API q4c_status q4c_grid_tiling(const q4c_grid* grid, int32_t bucket, int32_t* nb_max, int32_t* k_steps,
                                   int64_t* batches, double* ms_one, double* ms_two);
Q4C_API q4c_status q4c_grid_set_tiling(q4c_grid* grid, int32_t bucket, int32_t k_steps);

/* q4c_integrate with prec = Q4C_FP64 for callers that cannot allocate device
 * memory when they integrate (an application whose own pool owns the device
 * memory, or a loop that must not pay for cudaMalloc/cudaFree, which can
 * synchronise the device).  The paper has no counterpart; this is a library
 * convenience.  It allocates nothing: the per-batch basis-tile workspace is a
 * statically reserved 64 MiB device array that every GPU loading the library
 * holds until exit, used in waves of batches.  Same arguments, outputs and
 * results as q4c_integrate(..., Q4C_FP64, ...).  Q4C_EUNSUPPORTED if one
 * batch's tiles (4 n_b ceil8(n_p) doubles) exceed 64 MiB.  All calls share
 * the array: calls that overlap on the GPU race and must be serialised by
 * the caller.  The first call on each device looks up the array's device
 * address and keeps it for the rest of the process; make that first call
 * before any stream capture, and do not call this entry point again on a
 * device whose primary context the process has destroyed (cudaDeviceReset). */
Q4C_API q4c_status q4c_integrate_noalloc(const q4c_tables* tables, const q4c_grid* grid, const double* v_dev,
                                         const q4c_matrices* out, q4c_stream stream);

/* Basis values at arbitrary points with the kernels' own evaluation (for
 * parity checks): phi_dev[n_basis][n_pts], grad_dev[n_basis][n_pts][3]
 * (device, overwritten); xyz_dev device [n_pts][3]. */
Q4C_API q4c_status q4c_basis_eval(const q4c_tables* tables, const q4c_grid* grid, int64_t n_pts,
                          const double* xyz_dev, double* phi_dev, double* grad_dev,
                          q4c_stream stream);

/* Synchronises `stream` and reports whether any kernel that ran on this
 * grid's data hit the iteration limit of one of its bounded waits (tensor-core
 * completion barriers): Q4C_ETIMEOUT if so (the flag is then cleared), else
 * Q4C_OK.  Such a kernel stops early instead of hanging, so its outputs are
 * incomplete. */
Q4C_API q4c_status q4c_grid_status(const q4c_grid* grid, q4c_stream stream);

/* Limit, in nanoseconds of wall clock, of each bounded wait of the working
 * roles of the tensor-core kernels (the split path), for kernels launched
 * after the call, from any thread, on any device; 0 restores the default of
 * one second.  A wait that runs out sets the grid's status flag (reported by
 * q4c_grid_status) and stops the kernel early, so its outputs are
 * incomplete; the waits with which a stopping kernel drains its own copies
 * and tensor-core operations keep the fixed one-second limit.  Meant for
 * tests of the failure path (a tiny limit makes the first wait that is not
 * already satisfied give up) and for callers that want a stall reported
 * sooner.  Always Q4C_OK.  Not in the paper: a library control. */
Q4C_API q4c_status q4c_set_wait_limit_ns(uint64_t ns);

/* Kernel instrumentation.  q4c_profile(1) makes every later compute call
 * record a pair of CUDA events on its stream around each kernel it launches
 * (and count the launches); q4c_profile(0) stops recording.
 * q4c_profile_read synchronises on the recorded events, adds up the elapsed
 * time of the kernels whose name starts with `prefix` (NULL or "" = all),
 * returns the total in *ms and the number of launches in *launches, and
 * forgets the records it read.  Kernel names: "basis", "products_fp64",
 * "mirror", "spinor", "density_fp64", "backward_fp64", "split_*". */
Q4C_API q4c_status q4c_profile(int32_t enable);
Q4C_API q4c_status q4c_profile_read(const char* prefix, double* ms, int64_t* launches);

/* Message of the last failure on the calling thread ("" if none). */
Q4C_API const char* q4c_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* Q4C_H */
