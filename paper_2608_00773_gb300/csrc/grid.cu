// grid_partition: atom-centred integration grid, Becke partition weights,
// pruning, cut-plane batches, reduced index sets nnz(B_v) and the block
// pattern (Section III A, Figs. 1-2, Eqs. 31-32).
//
// Host work is bookkeeping (raw points, bisection, index lists); the FP64
// partition weights, the only arithmetic-heavy setup step (O(|N(r)|^2) per
// point), run in one kernel.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <thread>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"

namespace q4c {

constexpr int kMaxNeighbours = 512;

// Centres binned into cubes of side `size` from the corner `lo` (n[3] bins a
// side), CSR over bins in (z, y, x) order, centres ascending within a bin:
// every centre within `size` of a point lies in the 27 bins around the
// point's bin.  ptr == NULL: no bins (each point scans its candidate range).
struct CellList {
  const int* ptr;
  const int* idx;
  double lo[3];
  double size;
  int n[3];
};

struct HostCellList {
  std::vector<int> ptr, idx;
  double lo[3] = {0, 0, 0};
  double size = 1;
  int n[3] = {1, 1, 1};
  HostCellList(const double* xyz, int count, double side) : size(side) {
    double hi[3] = {-1e300, -1e300, -1e300};
    for (int d = 0; d < 3; ++d) lo[d] = 1e300;
    for (int c = 0; c < count; ++c)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xyz[3 * c + d]);
        hi[d] = std::max(hi[d], xyz[3 * c + d]);
      }
    for (int d = 0; d < 3; ++d) n[d] = std::max(1, static_cast<int>(std::floor((hi[d] - lo[d]) / size)) + 1);
    std::vector<int> bin(count);
    ptr.assign(static_cast<size_t>(n[0]) * n[1] * n[2] + 1, 0);
    for (int c = 0; c < count; ++c) {
      int k[3];
      for (int d = 0; d < 3; ++d) k[d] = std::min(n[d] - 1, static_cast<int>(std::floor((xyz[3 * c + d] - lo[d]) / size)));
      bin[c] = (k[2] * n[1] + k[1]) * n[0] + k[0];
      ++ptr[bin[c] + 1];
    }
    for (size_t b = 0; b + 1 < ptr.size(); ++b) ptr[b + 1] += ptr[b];
    idx.resize(count);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int c = 0; c < count; ++c) idx[fill[bin[c]]++] = c;  // ascending within a bin
  }
  // centres within distance `reach` of the box [a, b] (a superset: whole bins), ascending
  void near_box(const double a[3], const double b[3], double reach, std::vector<int>& out) const {
    out.clear();
    int k0[3], k1[3];
    for (int d = 0; d < 3; ++d) {
      k0[d] = static_cast<int>(std::max(-1.0, std::floor((a[d] - reach - lo[d]) / size)));
      k1[d] = static_cast<int>(std::min(static_cast<double>(n[d]), std::floor((b[d] + reach - lo[d]) / size)));
      k0[d] = std::max(k0[d], 0);
      k1[d] = std::min(k1[d], n[d] - 1);
    }
    for (int z = k0[2]; z <= k1[2]; ++z)
      for (int y = k0[1]; y <= k1[1]; ++y)
        for (int x = k0[0]; x <= k1[0]; ++x) {
          const int bb = (z * n[1] + y) * n[0] + x;
          out.insert(out.end(), idx.begin() + ptr[bb], idx.begin() + ptr[bb + 1]);
        }
    std::sort(out.begin(), out.end());
  }
};

// Gauss-Legendre nodes (ascending) and weights by Newton's method on P_n,
// with P_n' from (1 - x^2) P_n' = n (P_{n-1} - x P_n).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double z = std::cos(M_PI * (4.0 * k + 3.0) / (4.0 * n + 2.0));
    double p = 1.0, q = 0.0, dp = 1.0;
    for (int it = 0; it < 64; ++it) {
      p = z;
      q = 1.0;
      for (int j = 2; j <= n; ++j) {
        const double nxt = ((2 * j - 1) * z * p - (j - 1) * q) / j;
        q = p;
        p = nxt;
      }
      if (n == 1) { p = z; q = 1.0; }
      dp = n * (q - z * p) / (1.0 - z * z);
      const double step = p / dp;
      z -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    p = z;
    q = 1.0;
    for (int j = 2; j <= n; ++j) {
      const double nxt = ((2 * j - 1) * z * p - (j - 1) * q) / j;
      q = p;
      p = nxt;
    }
    dp = n * (q - z * p) / (1.0 - z * z);
    x[n - 1 - k] = z;
    w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Becke cell function s(mu) = (1 - f(f(f(mu))))/2, f(mu) = 1.5 mu - 0.5 mu^3
__device__ __forceinline__ double becke_s(double mu) {
  double f = mu;
#pragma unroll
  for (int k = 0; k < 3; ++k) f = 1.5 * f - 0.5 * f * f * f;
  return 0.5 * (1.0 - f);
}

// Stratmann, Scuseria and Frisch (1996) cell function without size
// adjustment: s(mu) = (1 - g(mu))/2, g(x) = (35 x - 35 x^3 + 21 x^5 - 5 x^7)/16
// of x = mu/a on |mu| <= a = 0.64, g = -1 below and +1 above
__device__ __forceinline__ double stratmann_s(double mu) {
  constexpr double a = 0.64;
  if (mu <= -a) return 1.0;
  if (mu >= a) return 0.0;
  const double x = mu / a, x2 = x * x;
  return 0.5 - x * (35.0 + x2 * (-35.0 + x2 * (21.0 - 5.0 * x2))) * (1.0 / 32.0);
}

// One thread per raw point: neighbour set N(r) = atoms within r_nb, then
// p_owner = P_owner / sum_{C in N} P_C with P_A = prod_{B in N, B != A} s(mu_AB),
// mu_AB = (|r - R_A| - |r - R_B|)/|R_A - R_B|.  near = some atom within r_c.
__global__ void k_becke(const double* __restrict__ raw, const double* __restrict__ base_w, int64_t n_raw,
                        int pts_per_atom, int owner_base, const double* __restrict__ atom_xyz,
                        const int2* __restrict__ cand, CellList bins, double r_c, double r_nb, int scheme,
                        double* __restrict__ w_out, unsigned char* __restrict__ near_out,
                        int* __restrict__ overflow) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= n_raw) return;
  const int gen = static_cast<int>(p / pts_per_atom);  // generating (cell-0) atom
  const int owner = owner_base + gen;
  // centres that can take part: the generating atom's molecule, or all
  const int2 range = cand[gen];
  const double px = raw[3 * p], py = raw[3 * p + 1], pz = raw[3 * p + 2];
  int nb_idx[kMaxNeighbours];
  double nb_d[kMaxNeighbours];
  int nn = 0, own_slot = -1;
  bool near = false;
  bool full = false;  // more than kMaxNeighbours centres within r_nb
  auto consider = [&](int B) {
    const double dx = px - atom_xyz[3 * B], dy = py - atom_xyz[3 * B + 1], dz = pz - atom_xyz[3 * B + 2];
    const double d = centre_distance(dx, dy, dz);
    if (d < r_c) near = true;
    if (d < r_nb) {
      if (nn == kMaxNeighbours) {
        full = true;
        return;
      }
      if (B == owner) own_slot = nn;
      nb_idx[nn] = B;
      nb_d[nn] = d;
      ++nn;
    }
  };
  if (bins.ptr) {  // the 27 bins around the point (bins are at least max(r_c, r_nb) wide)
    const double pc[3] = {px, py, pz};
    int k0[3], k1[3];
    for (int d = 0; d < 3; ++d) {
      const double k = fmin(fmax(floor((pc[d] - bins.lo[d]) / bins.size), -2.0), bins.n[d] + 1.0);
      k0[d] = max(static_cast<int>(k) - 1, 0);
      k1[d] = min(static_cast<int>(k) + 1, bins.n[d] - 1);
    }
    for (int z = k0[2]; z <= k1[2] && !full; ++z)
      for (int y = k0[1]; y <= k1[1] && !full; ++y)
        for (int x = k0[0]; x <= k1[0] && !full; ++x) {
          const int bb = (z * bins.n[1] + y) * bins.n[0] + x;
          for (int q = bins.ptr[bb]; q < bins.ptr[bb + 1] && !full; ++q) consider(bins.idx[q]);
        }
  } else {
    for (int B = range.x; B < range.y && !full; ++B) consider(B);
  }
  if (full) {
    atomicExch(overflow, 1);
    w_out[p] = 0.0;
    near_out[p] = 0;
    return;
  }
  near_out[p] = near ? 1 : 0;
  if (!near || own_slot < 0) {
    w_out[p] = 0.0;
    return;
  }
  auto cell = [&](int a) {
    const int A = nb_idx[a];
    const double ax = atom_xyz[3 * A], ay = atom_xyz[3 * A + 1], az = atom_xyz[3 * A + 2];
    double P = 1.0;
    for (int b = 0; b < nn && P != 0.0; ++b) {
      if (b == a) continue;
      const int B = nb_idx[b];
      const double dx = ax - atom_xyz[3 * B], dy = ay - atom_xyz[3 * B + 1], dz = az - atom_xyz[3 * B + 2];
      const double rab = sqrt(dx * dx + dy * dy + dz * dz);
      const double mu = (nb_d[a] - nb_d[b]) / rab;
      P *= scheme == 1 ? stratmann_s(mu) : becke_s(mu);
    }
    return P;
  };
  const double Pown = cell(own_slot);
  if (Pown == 0.0) {
    w_out[p] = 0.0;
    return;
  }
  double sum = 0.0;
  for (int a = 0; a < nn; ++a) sum += (a == own_slot) ? Pown : cell(a);
  w_out[p] = base_w[p] * (Pown / sum);
}

}  // namespace q4c

using namespace q4c;

DevGrid q4c_grid::view() const {
  DevGrid v;
  v.x = d_x;
  v.y = d_y;
  v.z = d_z;
  v.w = d_w;
  v.atom_xyz = d_atom_xyz;
  v.atom_sp = d_atom_sp;
  v.c_xyz = d_c_xyz;
  v.c_sp = d_c_sp;
  v.pt_ptr = d_pt_ptr;
  v.bat_atom_ptr = d_bat_atom_ptr;
  v.bat_atoms = d_bat_atoms;
  v.bat_atom_fn0 = d_bat_atom_fn0;
  v.bat_fn_ptr = d_bat_fn_ptr;
  v.fn_info = d_fn_info;
  v.bat_pair_ptr = d_bat_pair_ptr;
  v.pair_off = d_pair_off;
  v.bat_idx_ptr = d_bat_idx_ptr;
  v.bat_idx = d_bat_idx;
  v.n_atoms = n_atoms;
  v.wait_ns = q4c::work_wait_limit_ns();
  return v;
}

template <typename T>
static q4c_status up(T** dst, const std::vector<T>& src) {
  Q4C_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * std::max<size_t>(src.size(), 1)));
  if (!src.empty()) Q4C_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return Q4C_OK;
}

template <typename F>
static void parallel_for(int64_t n, F&& f) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < 64) nt = 1;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int64_t i = t; i < n; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

namespace q4c {

// Dense offset tables of one wave's batches (one CTA per batch) from the
// centre-pair offsets: element (i, j) -> pair_off[a_i, a_j] + k_i nf(a_j) + k_j.
__global__ void k_fill_idx(DevBasis B, DevGrid G, int64_t b0) {
  const int64_t b = b0 + blockIdx.x;
  const int64_t f0 = G.bat_fn_ptr[b];
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - f0);
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const int64_t pp = G.bat_pair_ptr[b];
  int* idx = G.bat_idx + G.bat_idx_ptr[b];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    const int ii = G.fn_info[f0 + i], jj = G.fn_info[f0 + j];
    const int64_t off = G.pair_off[pp + static_cast<int64_t>(ii >> 16) * na + (jj >> 16)];
    const int nfj = __ldg(B.sp_nfn + G.c_sp[G.bat_atoms[a0 + (jj >> 16)]]);
    idx[e] = off < 0 ? -1 : static_cast<int>(off + static_cast<int64_t>(ii & 0xffff) * nfj + (jj & 0xffff));
  }
}

q4c_status launch_fill_idx(const q4c_tables* t, const q4c_grid* g, int64_t b0, int64_t b1, cudaStream_t s) {
  if (b1 <= b0) return Q4C_OK;
  KernelScope ks("fill_idx", s);
  k_fill_idx<<<static_cast<unsigned>(b1 - b0), 256, 0, s>>>(t->view(), g->view(), b0);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

}  // namespace q4c

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// One TMA map per batch over its basis tiles in the scratch buffer: a 3-D
// tensor (point, function, quantity) of 8-byte (hi, lo) pairs with extents
// (n_p, n_b, 4) and row pitch ceil8(n_p), read in boxes of 16 points x 64
// functions with the 128-byte swizzle.  Points past n_p and functions past
// n_b read as zeros.
// A second set with boxes of 64 points x 16 functions (no swizzle) serves the
// density and the adjoint, whose A operand runs over points.
static q4c_status encode_tile_maps(q4c_grid* g) {
  const int64_t nB = g->n_batches;
  const size_t n_maps = static_cast<size_t>(std::max<int64_t>(nB, 1));
  std::vector<CUtensorMap> maps(2 * n_maps);
  std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  auto enc = tensor_map_encoder();
  if (!enc) {
    set_error("grid_partition: cuTensorMapEncodeTiled is not available from the driver");
    return Q4C_ECUDA;
  }
  for (int64_t b = 0; b < nB; ++b) {
    const int64_t np = g->h_pt_ptr[b + 1] - g->h_pt_ptr[b];
    const int64_t nb = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
    if (np <= 0 || nb <= 0) continue;  // no items read this batch
    const int64_t ldp = (np + 7) / 8 * 8;
    void* base = g->d_scratch + g->h_scr_off[b];
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(np), static_cast<cuuint64_t>(nb), 4};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(ldp * 8), static_cast<cuuint64_t>(nb * ldp * 8)};
    const cuuint32_t box[3] = {16, 64, 1}, box_rd[3] = {64, 16, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&maps[b], CU_TENSOR_MAP_DATA_TYPE_INT64, 3, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = enc(&maps[n_maps + b], CU_TENSOR_MAP_DATA_TYPE_INT64, 3, base, dims, strides, box_rd, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("grid_partition: cuTensorMapEncodeTiled failed for batch " + std::to_string(b) + " (CUresult " +
                std::to_string(static_cast<int>(r)) + ")");
      return Q4C_ECUDA;
    }
  }
  Q4C_CUDA(cudaMemcpy(g->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
  return Q4C_OK;
}

static int64_t scratch_cap_doubles() {
  int64_t mb = 4096;
  if (const char* e = std::getenv("Q4C_SCRATCH_MB")) mb = std::max<int64_t>(16, std::atoll(e));
  return mb * (1 << 20) / 8;
}

extern "C" q4c_status grid_partition(const q4c_grid_desc* d, const q4c_tables* t, q4c_grid** out) {
  Q4C_CHECK_ARG(d && t && out, "grid_partition: NULL argument");
  *out = nullptr;
  Q4C_CHECK_ARG(d->n_atoms >= 1 && d->xyz && d->species, "grid_partition: no atoms");
  Q4C_CHECK_ARG(d->n_rad_shells >= 1 && d->n_theta >= 1 && d->n_phi >= 1 && d->R > 0 && d->r_nb > 0,
                "grid_partition: bad grid parameters");
  Q4C_CHECK_ARG(d->batch_max >= 1 && d->batch_max <= kMaxBatch, "grid_partition: batch_max must be in 1..1024");
  Q4C_CHECK_ARG(d->partition == 0 || d->partition == 1, "grid_partition: partition must be 0 (Becke) or 1 (Stratmann)");
  for (int a = 0; a < d->n_atoms; ++a)
    Q4C_CHECK_ARG(d->species[a] >= 0 && d->species[a] < t->n_species, "grid_partition: species out of range");
  const int nA = d->n_atoms;
  const double r_c = t->r_c;

  auto* g = new q4c_grid();
  g->tables = t;
  cudaGetDevice(&g->device);
  g->n_atoms = nA;
  g->h_atom_xyz.assign(d->xyz, d->xyz + 3 * nA);
  g->h_atom_sp.assign(d->species, d->species + nA);
  g->h_nf_atom.resize(nA);
  g->h_atom_fn0.resize(nA);
  int nb_tot = 0;
  for (int a = 0; a < nA; ++a) {
    g->h_atom_fn0[a] = nb_tot;
    g->h_nf_atom[a] = t->nfn[d->species[a]];
    nb_tot += g->h_nf_atom[a];
  }
  g->n_basis = nb_tot;

  // ---- centres: the atoms and, in a periodic cell, their images R_A + T.L
  // (c = cell * n_atoms + A, cells in lexicographic order of T)
  const bool periodic = d->lattice != nullptr;
  if (periodic) {
    const double* L = d->lattice;
    const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                       L[2] * (L[3] * L[7] - L[4] * L[6]);
    if (!(d->n_shell >= 0 && d->n_shell <= 8) || !std::isfinite(det) || std::fabs(det) < 1e-6) {
      set_error("grid_partition: a lattice needs n_shell in 0..8 and three independent vectors");
      delete g;
      return Q4C_EINVAL;
    }
  }
  g->n_shell = periodic ? d->n_shell : 0;
  g->cell_side = 2 * g->n_shell + 1;
  const int n_cells = g->cell_side * g->cell_side * g->cell_side;
  const int cell0 = (n_cells - 1) / 2;  // T = (0, 0, 0)
  g->n_centres = n_cells * nA;
  const int nC = g->n_centres;
  auto cell_T = [&](int cell, int T[3]) {
    const int sd = g->cell_side, sh = g->n_shell;
    T[0] = cell / (sd * sd) - sh;
    T[1] = (cell / sd) % sd - sh;
    T[2] = cell % sd - sh;
  };
  // ---- molecules: atom ranges; every atom's candidate centres
  const int n_mol = d->n_molecules > 1 ? d->n_molecules : 1;
  std::vector<int> mol_ptr{0, nA};
  if (n_mol > 1) {
    bool ok = d->mol_atom_ptr != nullptr && !periodic && d->mol_atom_ptr[0] == 0 && d->mol_atom_ptr[n_mol] == nA;
    for (int m = 0; ok && m < n_mol; ++m) ok = d->mol_atom_ptr[m] < d->mol_atom_ptr[m + 1];
    if (!ok) {
      set_error("grid_partition: mol_atom_ptr must rise strictly from 0 to n_atoms (and no lattice)");
      delete g;
      return Q4C_EINVAL;
    }
    mol_ptr.assign(d->mol_atom_ptr, d->mol_atom_ptr + n_mol + 1);
  }
  std::vector<int2> cand(nA);  // candidate centre range of each cell-0 atom
  std::vector<int> atom_mol(nA);
  for (int m = 0; m < n_mol; ++m)
    for (int A = mol_ptr[m]; A < mol_ptr[m + 1]; ++A) {
      atom_mol[A] = m;
      cand[A] = n_mol > 1 ? make_int2(mol_ptr[m], mol_ptr[m + 1]) : make_int2(0, nC);
    }
  g->h_c_xyz.resize(3 * static_cast<size_t>(nC));
  g->h_c_sp.resize(nC);
  for (int cell = 0; cell < n_cells; ++cell) {
    int T[3];
    cell_T(cell, T);
    double sh[3] = {0, 0, 0};
    if (periodic)
      for (int k = 0; k < 3; ++k)
        for (int dd = 0; dd < 3; ++dd) sh[dd] += T[k] * d->lattice[3 * k + dd];
    for (int A = 0; A < nA; ++A) {
      const int c = cell * nA + A;
      for (int dd = 0; dd < 3; ++dd) g->h_c_xyz[3 * c + dd] = d->xyz[3 * A + dd] + sh[dd];
      g->h_c_sp[c] = d->species[A];
    }
  }

  // ---- raw points and base weights (w_rad * w_GL * 2 pi / n_phi)
  std::vector<double> rr(d->n_rad_shells), wr(d->n_rad_shells), ct, wt;
  for (int i = 1; i <= d->n_rad_shells; ++i) {
    const double th = i * M_PI / (d->n_rad_shells + 1);
    const double x = std::cos(th);
    rr[i - 1] = d->R * (1.0 + x) / (1.0 - x);
    wr[i - 1] = M_PI / (d->n_rad_shells + 1) * std::sin(th) * rr[i - 1] * rr[i - 1] * 2.0 * d->R /
                ((1.0 - x) * (1.0 - x));
  }
  gauss_legendre(d->n_theta, ct, wt);
  const int ppa = d->n_rad_shells * d->n_theta * d->n_phi;
  const int64_t n_raw = static_cast<int64_t>(ppa) * nA;
  std::vector<double> raw(3 * n_raw), base(n_raw);
  parallel_for(nA, [&](int64_t A) {
    int64_t p = A * ppa;
    for (int i = 0; i < d->n_rad_shells; ++i)
      for (int a = 0; a < d->n_theta; ++a) {
        const double st = std::sqrt(1.0 - ct[a] * ct[a]);
        for (int b = 0; b < d->n_phi; ++b, ++p) {
          const double ph = (b + 0.5) * 2.0 * M_PI / d->n_phi;
          raw[3 * p] = d->xyz[3 * A] + rr[i] * st * std::cos(ph);
          raw[3 * p + 1] = d->xyz[3 * A + 1] + rr[i] * st * std::sin(ph);
          raw[3 * p + 2] = d->xyz[3 * A + 2] + rr[i] * ct[a];
          base[p] = wr[i] * wt[a] * (2.0 * M_PI / d->n_phi);
        }
      }
  });

  // ---- centre bins of a single system (one molecule or a periodic cell):
  // cubes at least max(r_c, r_nb) wide, so that a point finds its neighbours
  // in the 27 bins around it; batched molecules scan their own atoms instead
  std::unique_ptr<HostCellList> bins;
  if (n_mol == 1) bins.reset(new HostCellList(g->h_c_xyz.data(), nC, std::max(r_c, d->r_nb)));

  // ---- Becke weights on the device
  std::vector<double> wfull(n_raw);
  std::vector<unsigned char> nearv(n_raw);
  {
    double *d_raw = nullptr, *d_base = nullptr, *d_w = nullptr, *d_axyz = nullptr;
    unsigned char* d_near = nullptr;
    int* d_ovf = nullptr;
    int2* d_cand = nullptr;
    int *d_bptr = nullptr, *d_bidx = nullptr;
    auto cleanup = [&] {
      cudaFree(d_raw); cudaFree(d_base); cudaFree(d_w); cudaFree(d_axyz); cudaFree(d_near); cudaFree(d_ovf);
      cudaFree(d_cand); cudaFree(d_bptr); cudaFree(d_bidx);
    };
    CellList cl{};
    cudaError_t e = cudaSuccess;
    int ovf = 0;
    do {
      if ((e = cudaMalloc(&d_raw, sizeof(double) * 3 * n_raw))) break;
      if ((e = cudaMalloc(&d_base, sizeof(double) * n_raw))) break;
      if ((e = cudaMalloc(&d_w, sizeof(double) * n_raw))) break;
      if ((e = cudaMalloc(&d_axyz, sizeof(double) * 3 * nC))) break;
      if ((e = cudaMalloc(&d_near, n_raw))) break;
      if ((e = cudaMalloc(&d_ovf, sizeof(int)))) break;
      if ((e = cudaMalloc(&d_cand, sizeof(int2) * nA))) break;
      if ((e = cudaMemcpy(d_cand, cand.data(), sizeof(int2) * nA, cudaMemcpyHostToDevice))) break;
      if ((e = cudaMemset(d_ovf, 0, sizeof(int)))) break;
      if ((e = cudaMemcpy(d_raw, raw.data(), sizeof(double) * 3 * n_raw, cudaMemcpyHostToDevice))) break;
      if ((e = cudaMemcpy(d_base, base.data(), sizeof(double) * n_raw, cudaMemcpyHostToDevice))) break;
      if ((e = cudaMemcpy(d_axyz, g->h_c_xyz.data(), sizeof(double) * 3 * nC, cudaMemcpyHostToDevice))) break;
      if (bins) {
        if ((e = cudaMalloc(&d_bptr, sizeof(int) * bins->ptr.size()))) break;
        if ((e = cudaMalloc(&d_bidx, sizeof(int) * bins->idx.size()))) break;
        if ((e = cudaMemcpy(d_bptr, bins->ptr.data(), sizeof(int) * bins->ptr.size(), cudaMemcpyHostToDevice))) break;
        if ((e = cudaMemcpy(d_bidx, bins->idx.data(), sizeof(int) * bins->idx.size(), cudaMemcpyHostToDevice))) break;
        cl.ptr = d_bptr;
        cl.idx = d_bidx;
        cl.size = bins->size;
        for (int k = 0; k < 3; ++k) {
          cl.lo[k] = bins->lo[k];
          cl.n[k] = bins->n[k];
        }
      }
      const int threads = 128;
      const int64_t blocks = (n_raw + threads - 1) / threads;
      k_becke<<<static_cast<unsigned>(blocks), threads>>>(d_raw, d_base, n_raw, ppa, cell0 * nA, d_axyz, d_cand, cl,
                                                          r_c, d->r_nb, d->partition, d_w, d_near, d_ovf);
      if ((e = cudaGetLastError())) break;
      if ((e = cudaMemcpy(wfull.data(), d_w, sizeof(double) * n_raw, cudaMemcpyDeviceToHost))) break;
      if ((e = cudaMemcpy(nearv.data(), d_near, n_raw, cudaMemcpyDeviceToHost))) break;
      if ((e = cudaMemcpy(&ovf, d_ovf, sizeof(int), cudaMemcpyDeviceToHost))) break;
    } while (0);
    cleanup();
    if (e != cudaSuccess) {
      set_error(std::string("grid_partition: Becke pass: ") + cudaGetErrorString(e));
      delete g;
      return e == cudaErrorMemoryAllocation ? Q4C_ENOMEM : Q4C_ECUDA;
    }
    if (ovf) {
      set_error("grid_partition: more than 512 centres within r_nb of a grid point");
      delete g;
      return Q4C_EUNSUPPORTED;
    }
  }

  // ---- prune: keep points within r_c of some atom with w != 0
  std::vector<int64_t> kept;
  kept.reserve(n_raw / 2);
  for (int64_t p = 0; p < n_raw; ++p)
    if (nearv[p] && wfull[p] != 0.0) kept.push_back(p);
  if (kept.empty()) {
    set_error("grid_partition: no grid point survives pruning");
    delete g;
    return Q4C_EINVAL;
  }

  // ---- cut-plane batches: recursive median bisection along the longest
  // bounding-box axis; order by (coordinate, raw id)
  std::vector<int64_t> order = kept;
  std::vector<int64_t> bptr{0};
  {
    struct Range { int64_t lo, hi; };
    // split r at the median of its longest bounding-box axis (in place)
    auto split = [&](const Range& r) -> int64_t {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t i = r.lo; i < r.hi; ++i)
        for (int k = 0; k < 3; ++k) {
          const double c = raw[3 * order[i] + k];
          lo[k] = std::min(lo[k], c);
          hi[k] = std::max(hi[k], c);
        }
      int ax = 0;
      for (int k = 1; k < 3; ++k)
        if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
      const int64_t mid = r.lo + (r.hi - r.lo) / 2;
      std::nth_element(order.begin() + r.lo, order.begin() + mid, order.begin() + r.hi,
                       [&](int64_t a, int64_t b) {
                         const double ca = raw[3 * a + ax], cb = raw[3 * b + ax];
                         return ca < cb || (ca == cb && a < b);
                       });
      return mid;
    };
    // one root range per molecule (kept points are atom-major, so each
    // molecule's points are contiguous), then a few breadth-first levels so
    // that there are enough independent subtrees for the host threads; the
    // leaves of every subtree come out depth-first, left half first, and the
    // subtrees are concatenated left to right: the same batches as one
    // depth-first pass
    std::vector<Range> front;
    {
      int64_t i = 0;
      for (int m = 0; m < n_mol; ++m) {
        const int64_t lo = i;
        while (i < static_cast<int64_t>(order.size()) && atom_mol[order[i] / ppa] == m) ++i;
        if (i > lo) front.push_back({lo, i});
      }
    }
    for (int level = 0; level < 12 && front.size() < 64; ++level) {
      std::vector<Range> next;
      bool any = false;
      for (const Range& r : front) {
        if (r.hi - r.lo <= d->batch_max) {
          next.push_back(r);
          continue;
        }
        const int64_t mid = split(r);
        next.push_back({r.lo, mid});
        next.push_back({mid, r.hi});
        any = true;
      }
      front.swap(next);
      if (!any) break;
    }
    std::vector<std::vector<Range>> leaves(front.size());
    std::atomic<int64_t> next_sub{0};
    auto worker = [&] {
      for (int64_t f; (f = next_sub.fetch_add(1)) < static_cast<int64_t>(front.size());) {
        std::vector<Range> stack{front[f]};
        while (!stack.empty()) {
          Range r = stack.back();
          stack.pop_back();
          if (r.hi - r.lo <= d->batch_max) {
            leaves[f].push_back(r);
            continue;
          }
          const int64_t mid = split(r);
          stack.push_back({mid, r.hi});  // right half pushed first: left half emitted first
          stack.push_back({r.lo, mid});
        }
      }
    };
    {
      const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
      std::vector<std::thread> th;
      for (unsigned t = 0; t < nt; ++t) th.emplace_back(worker);
      for (auto& x : th) x.join();
    }
    for (const auto& lv : leaves)
      for (const Range& r : lv) bptr.push_back(r.hi);
  }
  const int64_t nB = static_cast<int64_t>(bptr.size()) - 1;
  const int64_t nP = static_cast<int64_t>(order.size());
  g->n_pts = nP;
  g->n_batches = nB;
  g->h_pt_ptr = bptr;
  g->h_xyz.resize(3 * nP);
  g->h_w.resize(nP);
  g->h_pid = order;
  for (int64_t i = 0; i < nP; ++i) {
    const int64_t p = order[i];
    g->h_xyz[3 * i] = raw[3 * p];
    g->h_xyz[3 * i + 1] = raw[3 * p + 1];
    g->h_xyz[3 * i + 2] = raw[3 * p + 2];
    g->h_w[i] = wfull[p];
  }
  raw.clear(); raw.shrink_to_fit();

  // ---- active centres per batch: some point strictly within r_c
  std::vector<std::vector<int>> act(nB);
  parallel_for(nB, [&](int64_t b) {
    const int64_t p0 = bptr[b], p1 = bptr[b + 1];
    double c[3] = {0, 0, 0};
    for (int64_t i = p0; i < p1; ++i)
      for (int k = 0; k < 3; ++k) c[k] += g->h_xyz[3 * i + k];
    for (int k = 0; k < 3; ++k) c[k] /= static_cast<double>(p1 - p0);
    double rad = 0;
    for (int64_t i = p0; i < p1; ++i) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += (g->h_xyz[3 * i + k] - c[k]) * (g->h_xyz[3 * i + k] - c[k]);
      rad = std::max(rad, std::sqrt(s));
    }
    const double* cx = g->h_c_xyz.data();
    // candidates: the batch's molecule, or the binned centres near the batch's box
    std::vector<int> near;
    if (bins) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t i = p0; i < p1; ++i)
        for (int k = 0; k < 3; ++k) {
          lo[k] = std::min(lo[k], g->h_xyz[3 * i + k]);
          hi[k] = std::max(hi[k], g->h_xyz[3 * i + k]);
        }
      bins->near_box(lo, hi, r_c, near);
    } else {
      const int2 range = cand[g->h_pid[p0] / ppa];  // the batch's molecule
      for (int A = range.x; A < range.y; ++A) near.push_back(A);
    }
    for (int A : near) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += (cx[3 * A + k] - c[k]) * (cx[3 * A + k] - c[k]);
      if (std::sqrt(s) >= rad + r_c + 1e-9) continue;
      for (int64_t i = p0; i < p1; ++i) {
        const double dx = g->h_xyz[3 * i] - cx[3 * A], dy = g->h_xyz[3 * i + 1] - cx[3 * A + 1],
                     dz = g->h_xyz[3 * i + 2] - cx[3 * A + 2];
        if (centre_distance(dx, dy, dz) < r_c) {
          act[b].push_back(A);
          break;
        }
      }
    }
  });

  // ---- block pattern: (A, B, T) iff |R_A - R_B - T.L| < 2 r_c, T in
  // [-2 n_shell, 2 n_shell]^3 (T = 0 for a molecule); CSR over A, sorted by (B, T)
  g->h_blk_ptr.assign(nA + 1, 0);
  std::vector<int> blk_row;
  int64_t off = 0;
  const int s2 = 2 * g->n_shell, side2 = 2 * s2 + 1;
  {
    // each row on its own (rows in parallel), then concatenated in row order
    std::vector<std::vector<int>> rowB(nA), rowT(nA);
    parallel_for(nA, [&](int64_t A) {
      for (int B = mol_ptr[atom_mol[A]]; B < mol_ptr[atom_mol[A] + 1]; ++B) {
        for (int cell = 0; cell < side2 * side2 * side2; ++cell) {
          const int T[3] = {cell / (side2 * side2) - s2, (cell / side2) % side2 - s2, cell % side2 - s2};
          double sh[3] = {0, 0, 0};
          if (periodic)
            for (int k = 0; k < 3; ++k)
              for (int dd = 0; dd < 3; ++dd) sh[dd] += T[k] * d->lattice[3 * k + dd];
          const double dx = d->xyz[3 * A] - d->xyz[3 * B] - sh[0], dy = d->xyz[3 * A + 1] - d->xyz[3 * B + 1] - sh[1],
                       dz = d->xyz[3 * A + 2] - d->xyz[3 * B + 2] - sh[2];
          if (std::sqrt(dx * dx + dy * dy + dz * dz) < 2.0 * r_c) {
            rowB[A].push_back(B);
            rowT[A].insert(rowT[A].end(), {T[0], T[1], T[2]});
          }
        }
      }
    });
    for (int A = 0; A < nA; ++A) {
      for (size_t k = 0; k < rowB[A].size(); ++k) {
        const int B = rowB[A][k];
        g->h_blk_col.push_back(B);
        g->h_blk_shift.insert(g->h_blk_shift.end(), rowT[A].begin() + 3 * k, rowT[A].begin() + 3 * k + 3);
        blk_row.push_back(A);
        g->h_blk_off.push_back(off);
        off += static_cast<int64_t>(g->h_nf_atom[A]) * g->h_nf_atom[B];
      }
      g->h_blk_ptr[A + 1] = static_cast<int64_t>(g->h_blk_col.size());
      std::vector<int>().swap(rowB[A]);
      std::vector<int>().swap(rowT[A]);
    }
  }
  g->h_blk_off.push_back(off);
  g->n_blocks = static_cast<int64_t>(g->h_blk_col.size());
  g->nnz = off;
  // block (A, B, T) or -1; rows are sorted by (B, T) lexicographically
  auto find_block = [&](int A, int B, const int T[3]) -> int64_t {
    int64_t lo = g->h_blk_ptr[A], hi = g->h_blk_ptr[A + 1];
    auto key_less = [&](int64_t q) {  // block q before (B, T)?
      const int* t = g->h_blk_shift.data() + 3 * q;
      if (g->h_blk_col[q] != B) return g->h_blk_col[q] < B;
      if (t[0] != T[0]) return t[0] < T[0];
      if (t[1] != T[1]) return t[1] < T[1];
      return t[2] < T[2];
    };
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (key_less(mid)) lo = mid + 1;
      else hi = mid;
    }
    if (lo < g->h_blk_ptr[A + 1] && g->h_blk_col[lo] == B) {
      const int* t = g->h_blk_shift.data() + 3 * lo;
      if (t[0] == T[0] && t[1] == T[1] && t[2] == T[2]) return lo;
    }
    return -1;
  };
  // transpose partner (B, A, -T) of every block, and its role in the mirror:
  // the canonical half is T > 0 (lexicographic) or T = 0 and A <= B
  std::vector<int> blk_T(g->n_blocks), blk_role(g->n_blocks);
  for (int64_t q = 0; q < g->n_blocks; ++q) {
    const int* t = g->h_blk_shift.data() + 3 * q;
    const int mT[3] = {-t[0], -t[1], -t[2]};
    blk_T[q] = static_cast<int>(find_block(g->h_blk_col[q], blk_row[q], mT));
    const bool zero = t[0] == 0 && t[1] == 0 && t[2] == 0;
    const bool pos = t[0] > 0 || (t[0] == 0 && (t[1] > 0 || (t[1] == 0 && t[2] > 0)));
    const int A = blk_row[q], B = g->h_blk_col[q];
    blk_role[q] = (zero && A == B) ? 2 : ((pos || (zero && A < B)) ? 1 : 0);
  }

  // ---- k-pattern: atom pairs (A, B) with some block (A, B, T); the blocks of
  // one pair are a contiguous run of the pattern (rows sorted by (B, T))
  g->h_kblk_ptr.assign(nA + 1, 0);
  {
    int64_t koff = 0;
    for (int A = 0; A < nA; ++A) {
      for (int64_t q = g->h_blk_ptr[A]; q < g->h_blk_ptr[A + 1];) {
        int64_t q1 = q + 1;
        while (q1 < g->h_blk_ptr[A + 1] && g->h_blk_col[q1] == g->h_blk_col[q]) ++q1;
        g->h_kblk_col.push_back(g->h_blk_col[q]);
        g->h_kblk_off.push_back(koff);
        g->h_kblk_q0.push_back(q);
        g->h_kblk_q1.push_back(q1);
        koff += static_cast<int64_t>(g->h_nf_atom[A]) * g->h_nf_atom[g->h_blk_col[q]];
        q = q1;
      }
      g->h_kblk_ptr[A + 1] = static_cast<int64_t>(g->h_kblk_col.size());
    }
    g->h_kblk_off.push_back(koff);
    g->nnz_k = koff;
  }

  // ---- per-batch tables (over the batch's active centres)
  auto c_atom = [&](int c) { return c % nA; };
  auto c_cell = [&](int c) { return c / nA; };
  g->h_bat_atom_ptr.assign(nB + 1, 0);
  g->h_bat_fn_ptr.assign(nB + 1, 0);
  std::vector<int64_t> pair_ptr(nB + 1, 0);
  for (int64_t b = 0; b < nB; ++b) {
    const int na = static_cast<int>(act[b].size());
    int nb = 0;
    for (int A : act[b]) nb += g->h_nf_atom[c_atom(A)];
    g->h_bat_atom_ptr[b + 1] = g->h_bat_atom_ptr[b] + na;
    g->h_bat_fn_ptr[b + 1] = g->h_bat_fn_ptr[b] + nb;
    pair_ptr[b + 1] = pair_ptr[b] + static_cast<int64_t>(na) * na;
    const int np = static_cast<int>(bptr[b + 1] - bptr[b]);
    g->max_nb = std::max(g->max_nb, nb);
    g->max_np = std::max(g->max_np, np);
    g->max_na = std::max(g->max_na, na);
    g->flops_alg += 14.0 * np * static_cast<double>(nb) * nb;
    g->sum_np_nb += static_cast<double>(np) * nb;
  }
  std::vector<int> bat_atom_fn0(g->h_bat_atom_ptr[nB]);
  g->h_bat_atoms.resize(g->h_bat_atom_ptr[nB]);
  std::vector<int> fn_info(g->h_bat_fn_ptr[nB]);
  std::vector<int64_t> pair_off(pair_ptr[nB]);
  std::vector<int> pair_blk(pair_ptr[nB]);
  parallel_for(nB, [&](int64_t b) {
    const int na = static_cast<int>(act[b].size());
    int f = 0;
    for (int a = 0; a < na; ++a) {
      const int A = act[b][a];
      g->h_bat_atoms[g->h_bat_atom_ptr[b] + a] = A;
      bat_atom_fn0[g->h_bat_atom_ptr[b] + a] = f;
      for (int k = 0; k < g->h_nf_atom[c_atom(A)]; ++k) fn_info[g->h_bat_fn_ptr[b] + f++] = (a << 16) | k;
      int Ta[3];
      cell_T(c_cell(A), Ta);
      for (int c = 0; c < na; ++c) {
        const int Cc = act[b][c];
        int Tb[3];
        cell_T(c_cell(Cc), Tb);
        const int T[3] = {Tb[0] - Ta[0], Tb[1] - Ta[1], Tb[2] - Ta[2]};
        // no block: the two centres are never within r_c of one point of
        // the batch (active at opposite ends of it), so the pair adds nothing
        const int64_t q = find_block(c_atom(A), c_atom(Cc), T);
        pair_off[pair_ptr[b] + static_cast<int64_t>(a) * na + c] = q < 0 ? -1 : g->h_blk_off[q];
        pair_blk[pair_ptr[b] + static_cast<int64_t>(a) * na + c] = static_cast<int>(q);
      }
    }
  });
  if (g->nnz > INT32_MAX) {
    set_error("grid_partition: more than 2^31 matrix values on the block pattern");
    delete g;
    return Q4C_EUNSUPPORTED;
  }

  // ---- FP64 path: waves whose basis tiles fit the scratch cap; 32x32 tiles
  const int64_t cap = scratch_cap_doubles();
  g->h_scr_off.assign(nB, 0);
  std::vector<int4> tiles;
  g->wave_b0.push_back(0);
  g->wave_t0.push_back(0);
  int64_t used = 0, peak = 0;
  for (int64_t b = 0; b < nB; ++b) {
    const int64_t np = bptr[b + 1] - bptr[b];
    const int64_t nb = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
    const int64_t need = 4 * nb * ((np + 7) / 8 * 8);
    if (used > 0 && used + need > cap) {
      g->wave_b0.push_back(b);
      g->wave_t0.push_back(static_cast<int64_t>(tiles.size()));
      used = 0;
    }
    g->h_scr_off[b] = used;
    used += need;
    peak = std::max(peak, used);
    const int nt = static_cast<int>((nb + 31) / 32);
    for (int i = 0; i < nt; ++i)
      for (int j = i; j < nt; ++j) tiles.push_back(make_int4(static_cast<int>(b), i, j, 0));
  }
  g->wave_b0.push_back(nB);
  g->wave_t0.push_back(static_cast<int64_t>(tiles.size()));
  g->scratch_doubles = std::max<int64_t>(peak, 1);
  // per-column operator on the FP64 path (not symmetric): every tile pair
  std::vector<int4> col_tiles;
  g->colt_w0.push_back(0);
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    for (int64_t b = g->wave_b0[wv]; b < g->wave_b0[wv + 1]; ++b) {
      const int nt = static_cast<int>((g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b] + 31) / 32);
      for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j) col_tiles.push_back(make_int4(static_cast<int>(b), i, j, 0));
    }
    g->colt_w0.push_back(static_cast<int64_t>(col_tiles.size()));
  }

  // per-batch dense tables of pattern offsets, idx[i * n_b + j] = value
  // offset of element (i, j) (local functions) or -1 outside the pattern;
  // filled on the device for one wave at a time (sum n_b^2 of a whole grid
  // can be far larger than a wave's)
  std::vector<int64_t> idx_ptr(nB + 1, 0);
  g->idx_entries = 1;
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    int64_t used = 0;
    for (int64_t b = g->wave_b0[wv]; b < g->wave_b0[wv + 1]; ++b) {
      const int64_t nb = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
      idx_ptr[b] = used;
      used += nb * nb;
    }
    g->idx_entries = std::max(g->idx_entries, used);
  }

  // ---- split path: (batch, output, ti, tj) items per wave, tiles of 64
  // functions, tile pairs ti <= tj only (SO: the antisymmetric part of A_k on
  // diagonal pairs, two K-concatenated products on off-diagonal ones).  The
  // batches of a wave are grouped by batch-size bucket (each bucket is one
  // launch with its own stage shape), the costliest first within a bucket;
  // the items of one batch stay adjacent (W0, three products, leading) so
  // that concurrent CTAs share its tiles in L2.
  std::vector<int4> sitems;
  int64_t max_wave_items = 1;
  g->split_w0.push_back(0);
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    struct Key {
      int bucket;
      double cost;
      int64_t b;
    };
    std::vector<Key> bl;
    for (int64_t b = g->wave_b0[wv]; b < g->wave_b0[wv + 1]; ++b) {
      const double np = static_cast<double>(bptr[b + 1] - bptr[b]);
      const int64_t nbi = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
      const double nb = static_cast<double>(nbi);
      bl.push_back({tile_bucket(nbi), np * nb * nb, b});
    }
    std::stable_sort(bl.begin(), bl.end(), [](const Key& x, const Key& y) {
      return x.bucket != y.bucket ? x.bucket < y.bucket : x.cost > y.cost;
    });
    std::vector<int64_t> bw(kTileBuckets + 1, -1);
    for (const Key& x : bl) {
      for (int k = 0; k <= x.bucket; ++k)
        if (bw[k] < 0) bw[k] = static_cast<int64_t>(sitems.size());
      const int64_t b = x.b;
      const int nb = static_cast<int>(g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b]);
      const int nt = (nb + 63) / 64;
      for (int o : {1, 0, 2, 3, 4})
        for (int i = 0; i < nt; ++i)
          for (int j = i; j < nt; ++j) sitems.push_back(make_int4(static_cast<int>(b), o, i, j));
    }
    for (int k = 0; k <= kTileBuckets; ++k)
      if (bw[k] < 0) bw[k] = static_cast<int64_t>(sitems.size());
    g->split_bw0.insert(g->split_bw0.end(), bw.begin(), bw.end());
    max_wave_items = std::max(max_wave_items, static_cast<int64_t>(sitems.size()) - g->split_w0.back());
    g->split_w0.push_back(static_cast<int64_t>(sitems.size()));
  }
  // per-column operator (output 5): one product on every tile pair (it is
  // not symmetric), in the same batch order and buckets
  std::vector<int4> citems;
  g->col_w0.push_back(0);
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    std::vector<int64_t> bw(kTileBuckets + 1, -1);
    for (int64_t n = g->split_w0[wv]; n < g->split_w0[wv + 1]; ++n) {
      const int4 it = sitems[n];
      if (it.y != 1 || it.z != 0 || it.w != 0) continue;  // once per batch (its first item)
      const int64_t b = it.x;
      const int64_t nbi = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
      for (int k = 0; k <= tile_bucket(nbi); ++k)
        if (bw[k] < 0) bw[k] = static_cast<int64_t>(citems.size());
      const int nt = static_cast<int>((nbi + 63) / 64);
      for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nt; ++j) citems.push_back(make_int4(static_cast<int>(b), 5, i, j));
    }
    for (int k = 0; k <= kTileBuckets; ++k)
      if (bw[k] < 0) bw[k] = static_cast<int64_t>(citems.size());
    g->col_bw0.insert(g->col_bw0.end(), bw.begin(), bw.end());
    max_wave_items = std::max(max_wave_items, static_cast<int64_t>(citems.size()) - g->col_w0.back());
    g->col_w0.push_back(static_cast<int64_t>(citems.size()));
  }
  // density/adjoint: (batch, 64-point tile) items per wave, costliest first
  std::vector<int2> rditems;
  g->rd_w0.push_back(0);
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    std::vector<std::pair<double, int64_t>> bl;
    for (int64_t b = g->wave_b0[wv]; b < g->wave_b0[wv + 1]; ++b) {
      const double nb = static_cast<double>(g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b]);
      bl.push_back({nb * nb, b});
    }
    std::stable_sort(bl.begin(), bl.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (const auto& x : bl) {  // the point tiles of one batch stay adjacent
      const int64_t b = x.second, np = bptr[b + 1] - bptr[b];
      for (int pt = 0; pt * 64 < np; ++pt) rditems.push_back(make_int2(static_cast<int>(b), pt));
    }
    g->rd_w0.push_back(static_cast<int64_t>(rditems.size()));
  }
  // G' digit blocks of the density/adjoint, per wave: per batch five matrices
  // x ceil(nb/64) j-tiles x ceil(nb/16) i-chunks x 12 KB
  std::vector<int64_t> gsl_off(nB, 0);
  g->gsl_bytes = 0;
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    int64_t used = 0;
    for (int64_t b = g->wave_b0[wv]; b < g->wave_b0[wv + 1]; ++b) {
      const int64_t nb = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
      gsl_off[b] = used;
      used += 5 * ((nb + 63) / 64) * ((nb + 15) / 16) * 12288;
    }
    g->gsl_bytes = std::max(g->gsl_bytes, used);
  }

  // ---- schedule for persistent kernels: descending n_p n_b^2
  std::vector<int> sched(nB);
  std::iota(sched.begin(), sched.end(), 0);
  std::stable_sort(sched.begin(), sched.end(), [&](int a, int b) {
    auto cost = [&](int x) {
      const double np = static_cast<double>(bptr[x + 1] - bptr[x]);
      const double nb = static_cast<double>(g->h_bat_fn_ptr[x + 1] - g->h_bat_fn_ptr[x]);
      return np * nb * nb;
    };
    return cost(a) > cost(b);
  });

  // ---- per-block column and row maxima segments: [nf_B columns][nf_A rows]
  std::vector<int64_t> cm_off(g->n_blocks + 1, 0);
  for (int64_t q = 0; q < g->n_blocks; ++q)
    cm_off[q + 1] = cm_off[q] + g->h_nf_atom[blk_row[q]] + g->h_nf_atom[g->h_blk_col[q]];
  g->cm_total = std::max<int64_t>(cm_off[g->n_blocks], 1);

  // ---- upload
  std::vector<double> sx(nP), sy(nP), sz(nP);
  for (int64_t i = 0; i < nP; ++i) {
    sx[i] = g->h_xyz[3 * i];
    sy[i] = g->h_xyz[3 * i + 1];
    sz[i] = g->h_xyz[3 * i + 2];
  }
  auto dsplit = [](double x) { const float h = static_cast<float>(x); return df{h, static_cast<float>(x - h)}; };
  std::vector<df> pts_df(3 * nP), atoms_df(3 * static_cast<size_t>(nC));
  for (int64_t i = 0; i < 3 * nP; ++i) pts_df[i] = dsplit(g->h_xyz[i]);
  for (int i = 0; i < 3 * nC; ++i) atoms_df[i] = dsplit(g->h_c_xyz[i]);
  q4c_status st;
  if ((st = up(&g->d_pts_df, pts_df)) || (st = up(&g->d_atoms_df, atoms_df)) ||
      (st = up(&g->d_c_xyz, g->h_c_xyz)) || (st = up(&g->d_c_sp, g->h_c_sp)) || (st = up(&g->d_xyz, g->h_xyz)) || (st = up(&g->d_x, sx)) || (st = up(&g->d_y, sy)) ||
      (st = up(&g->d_z, sz)) || (st = up(&g->d_w, g->h_w)) || (st = up(&g->d_atom_xyz, g->h_atom_xyz)) ||
      (st = up(&g->d_atom_sp, g->h_atom_sp)) || (st = up(&g->d_atom_fn0, g->h_atom_fn0)) ||
      (st = up(&g->d_pt_ptr, g->h_pt_ptr)) || (st = up(&g->d_bat_atom_ptr, g->h_bat_atom_ptr)) ||
      (st = up(&g->d_bat_atoms, g->h_bat_atoms)) || (st = up(&g->d_bat_atom_fn0, bat_atom_fn0)) ||
      (st = up(&g->d_bat_fn_ptr, g->h_bat_fn_ptr)) || (st = up(&g->d_fn_info, fn_info)) ||
      (st = up(&g->d_bat_pair_ptr, pair_ptr)) || (st = up(&g->d_pair_off, pair_off)) ||
      (st = up(&g->d_pair_blk, pair_blk)) || (st = up(&g->d_cm_off, cm_off)) ||
      (st = up(&g->d_blk_off, g->h_blk_off)) || (st = up(&g->d_blk_row, blk_row)) ||
      (st = up(&g->d_blk_col, g->h_blk_col)) || (st = up(&g->d_blk_T, blk_T)) || (st = up(&g->d_blk_role, blk_role)) ||
      (st = up(&g->d_blk_shift, g->h_blk_shift)) || (st = up(&g->d_kblk_q0, g->h_kblk_q0)) ||
      (st = up(&g->d_kblk_q1, g->h_kblk_q1)) || (st = up(&g->d_kblk_off, g->h_kblk_off)) ||
      (st = up(&g->d_scr_off, g->h_scr_off)) || (st = up(&g->d_tiles, tiles)) || (st = up(&g->d_col_tiles, col_tiles)) || (st = up(&g->d_sched, sched)) ||
      (st = up(&g->d_split_items, sitems)) || (st = up(&g->d_col_items, citems)) ||
      (st = up(&g->d_rd_items, rditems)) ||
      (st = up(&g->d_bat_idx_ptr, idx_ptr)) ||
      (st = up(&g->d_gsl_off, gsl_off))) {
    q4c_grid_destroy(g);
    return st;
  }
  {
    const size_t n_waves = g->wave_b0.size() - 1;
    cudaError_t e = cudaMalloc(&g->d_scratch, sizeof(double) * g->scratch_doubles);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_counter, sizeof(int) * std::max<size_t>(n_waves, 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_colexp, sizeof(int) * 8 * std::max<int64_t>(g->h_bat_fn_ptr[nB], 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_rowexp, sizeof(int) * 4 * nP);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_gsl, static_cast<size_t>(std::max<int64_t>(g->gsl_bytes, 16)));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_gdf, sizeof(float2) * 10 * std::max<int64_t>(g->nnz, 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_cm, sizeof(float) * 10 * g->cm_total);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_gzero, 12288);
    if (e == cudaSuccess) e = cudaMemset(g->d_gzero, 0, 12288);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_bat_idx, sizeof(int) * g->idx_entries);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_split_mag, sizeof(float) * 128 * max_wave_items);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_dpad, sizeof(float2) * kDPitch * std::max<int64_t>(nB, 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_tmaps, 2 * sizeof(CUtensorMap) * std::max<int64_t>(nB, 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(unsigned));
    g->split_ws_bytes = static_cast<int64_t>(sizeof(int)) * (8 * g->h_bat_fn_ptr[nB] + 4 * nP) +
                        static_cast<int64_t>(sizeof(float2)) * 5 * g->nnz + g->gsl_bytes +
                        static_cast<int64_t>(sizeof(float)) * 10 * g->cm_total;
    if (e != cudaSuccess) {
      set_error(std::string("grid_partition: workspace: ") + cudaGetErrorString(e));
      q4c_grid_destroy(g);
      return e == cudaErrorMemoryAllocation ? Q4C_ENOMEM : Q4C_ECUDA;
    }
  }
  if (q4c_status st2 = encode_tile_maps(g)) {
    q4c_grid_destroy(g);
    return st2;
  }
  *out = g;
  return Q4C_OK;
}

extern "C" void q4c_grid_destroy(q4c_grid* g) {
  if (!g) return;
  void* ptrs[] = {g->d_xyz, g->d_x, g->d_y, g->d_z, g->d_w, g->d_atom_xyz, g->d_atom_sp, g->d_atom_fn0,
                  g->d_pt_ptr, g->d_bat_atom_ptr, g->d_bat_atoms, g->d_bat_atom_fn0, g->d_bat_fn_ptr,
                  g->d_fn_info, g->d_bat_pair_ptr, g->d_pair_off, g->d_blk_off, g->d_blk_row, g->d_blk_col,
                  g->d_blk_T, g->d_scr_off, g->d_tiles, g->d_col_tiles, g->d_scratch, g->d_sched, g->d_counter, g->d_split_ws,
                  g->d_split_items, g->d_col_items, g->d_split_mag, g->d_dpad, g->d_tmaps, g->d_colexp, g->d_status, g->d_rd_items, g->d_rowexp, g->d_gsl, g->d_gsl_off,
                  g->d_bat_idx_ptr, g->d_bat_idx, g->d_pts_df, g->d_atoms_df, g->d_gdf, g->d_gzero,
                  g->d_c_xyz, g->d_c_sp, g->d_blk_role, g->d_blk_shift, g->d_kblk_q0, g->d_kblk_q1,
                  g->d_kblk_off, g->d_cm_off, g->d_cm, g->d_pair_blk};
  for (void* p : ptrs) cudaFree(p);
  delete g;
}

extern "C" q4c_status q4c_grid_get_info(const q4c_grid* g, q4c_grid_info* info) {
  Q4C_CHECK_ARG(g && info, "q4c_grid_get_info: NULL argument");
  info->n_points = g->n_pts;
  info->n_batches = g->n_batches;
  info->n_blocks = g->n_blocks;
  info->nnz = g->nnz;
  info->n_atoms = g->n_atoms;
  info->n_basis = g->n_basis;
  info->max_nb = g->max_nb;
  info->max_np = g->max_np;
  info->flops_alg = g->flops_alg;
  info->sum_np_nb = g->sum_np_nb;
  info->scratch_bytes = 8 * g->scratch_doubles + g->split_ws_bytes + 4 * g->idx_entries;
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_export(const q4c_grid* g, double* xyz, double* w, int64_t* point_id,
                                      int64_t* batch_ptr, int64_t* batch_atom_ptr, int32_t* batch_atoms,
                                      int64_t* blk_ptr, int32_t* blk_col, int64_t* blk_off) {
  Q4C_CHECK_ARG(g, "q4c_grid_export: NULL grid");
  if (xyz) std::copy(g->h_xyz.begin(), g->h_xyz.end(), xyz);
  if (w) std::copy(g->h_w.begin(), g->h_w.end(), w);
  if (point_id) std::copy(g->h_pid.begin(), g->h_pid.end(), point_id);
  if (batch_ptr) std::copy(g->h_pt_ptr.begin(), g->h_pt_ptr.end(), batch_ptr);
  if (batch_atom_ptr)
    for (size_t i = 0; i < g->h_bat_atom_ptr.size(); ++i) batch_atom_ptr[i] = g->h_bat_atom_ptr[i];
  if (batch_atoms) std::copy(g->h_bat_atoms.begin(), g->h_bat_atoms.end(), batch_atoms);
  if (blk_ptr) std::copy(g->h_blk_ptr.begin(), g->h_blk_ptr.end(), blk_ptr);
  if (blk_col) std::copy(g->h_blk_col.begin(), g->h_blk_col.end(), blk_col);
  if (blk_off) std::copy(g->h_blk_off.begin(), g->h_blk_off.end(), blk_off);
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_export_shifts(const q4c_grid* g, int32_t* shifts) {
  Q4C_CHECK_ARG(g && shifts, "q4c_grid_export_shifts: NULL argument");
  std::copy(g->h_blk_shift.begin(), g->h_blk_shift.end(), shifts);
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_kpattern(const q4c_grid* g, int64_t* nnz_k, int64_t* kblk_ptr, int32_t* kblk_col,
                                        int64_t* kblk_off) {
  Q4C_CHECK_ARG(g, "q4c_grid_kpattern: NULL grid");
  if (nnz_k) *nnz_k = g->nnz_k;
  if (kblk_ptr) std::copy(g->h_kblk_ptr.begin(), g->h_kblk_ptr.end(), kblk_ptr);
  if (kblk_col) std::copy(g->h_kblk_col.begin(), g->h_kblk_col.end(), kblk_col);
  if (kblk_off) std::copy(g->h_kblk_off.begin(), g->h_kblk_off.end(), kblk_off);
  return Q4C_OK;
}

namespace q4c {
// One CTA per k-pattern block (A, B): the sum over its run of pattern blocks
// (A, B, T) with the phase exp(2 pi i k.T) (FP64 sincospi of the reduced phase).
__global__ void k_kfold(const int64_t* __restrict__ q0, const int64_t* __restrict__ q1,
                        const int64_t* __restrict__ koff, const int64_t* __restrict__ blk_off,
                        const int* __restrict__ shift, const double* __restrict__ H, double k1, double k2, double k3,
                        double2* __restrict__ out) {
  const int kb = blockIdx.x;
  const int64_t a = q0[kb], z = q1[kb];
  const int64_t n_el = blk_off[a + 1] - blk_off[a];
  for (int64_t e = threadIdx.x; e < n_el; e += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int64_t q = a; q < z; ++q) {
      const double t = k1 * shift[3 * q] + k2 * shift[3 * q + 1] + k3 * shift[3 * q + 2];
      double sn, cs;
      sincospi(2.0 * t, &sn, &cs);
      const double h = H[blk_off[q] + e];
      re = fma(h, cs, re);
      im = fma(h, sn, im);
    }
    out[koff[kb] + e] = make_double2(re, im);
  }
}
}  // namespace q4c

extern "C" q4c_status q4c_kfold(const q4c_grid* g, const double* H, int32_t n_k, const double* k,
                                double* Hk, q4c_stream stream) {
  Q4C_CHECK_ARG(g && (n_k == 0 || (H && k && Hk)), "q4c_kfold: NULL argument");
  Q4C_CHECK_ARG(n_k >= 0, "q4c_kfold: negative number of k-points");
  auto s = reinterpret_cast<cudaStream_t>(stream);
  const auto nkb = static_cast<unsigned>(g->h_kblk_col.size());
  if (nkb == 0) return Q4C_OK;
  for (int ik = 0; ik < n_k; ++ik) {
    KernelScope ks("kfold", s);
    k_kfold<<<nkb, 128, 0, s>>>(g->d_kblk_q0, g->d_kblk_q1, g->d_kblk_off, g->d_blk_off, g->d_blk_shift, H,
                                k[3 * ik], k[3 * ik + 1], k[3 * ik + 2],
                                reinterpret_cast<double2*>(Hk) + static_cast<int64_t>(ik) * g->nnz_k);
    Q4C_CUDA(cudaGetLastError());
  }
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_points(const q4c_grid* g, const double** xyz_dev, const double** w_dev,
                                      int64_t* n_points) {
  Q4C_CHECK_ARG(g, "q4c_grid_points: NULL grid");
  if (xyz_dev) *xyz_dev = g->d_xyz;
  if (w_dev) *w_dev = g->d_w;
  if (n_points) *n_points = g->n_pts;
  return Q4C_OK;
}

namespace {
std::atomic<unsigned long long> g_work_wait_ns{1000000000ull};
}  // namespace

unsigned long long q4c::work_wait_limit_ns() { return g_work_wait_ns.load(std::memory_order_relaxed); }

extern "C" q4c_status q4c_set_wait_limit_ns(uint64_t ns) {
  g_work_wait_ns.store(ns ? static_cast<unsigned long long>(ns) : 1000000000ull, std::memory_order_relaxed);
  return Q4C_OK;
}

extern "C" q4c_status q4c_grid_status(const q4c_grid* g, q4c_stream stream) {
  Q4C_CHECK_ARG(g, "q4c_grid_status: NULL grid");
  Q4C_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  unsigned st = 0;
  Q4C_CUDA(cudaMemcpy(&st, g->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (st) {
    Q4C_CUDA(cudaMemset(g->d_status, 0, sizeof(unsigned)));
    set_error("a bounded device wait expired in a kernel of this grid");
    return Q4C_ETIMEOUT;
  }
  return Q4C_OK;
}
