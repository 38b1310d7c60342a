// Plain FP64 path: basis tiles per batch, batch products on the FP64 ALUs,
// FP64 atomic scatter into the block pattern, mirror, spinor assembly,
// density (Eqs. 39-40) and the adjoint.  This is the reference-precision GPU
// path the split-precision tensor-core path is measured against.
#include "basis.cuh"
#include "internal.h"

namespace q4c {

// ------------------------------------------------------------------ basis
// Tiles of batch b in the scratch wave: Phi, X, Y, Z each [n_b][ldp],
// ldp = n_p rounded up to 8; one thread per (point, active atom).
// With colexp != NULL (split path) it also records, per batch and local
// function, binary exponents e with |value| < 2^e for the unscaled sets
// (Phi, X, Y, Z: slots 4..7) and upper bounds for the D-scaled sets
// (D = w v; slots 0..3, from e(D_p) + e(value)), colexp[8 n_b] per batch.
__device__ __forceinline__ int binexp(double x) {  // |x| < 2^binexp(x), x != 0
  const int E = static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF);
  return E - 1022;
}
constexpr int kNoExp = -30000;
// scr_base: subtracted from the batch offsets (the first offset of a sub-wave
// whose tiles start at `scratch`; 0 for the grid's own workspace)
__global__ void k_basis_tiles(DevBasis B, DevGrid G, int64_t b0, const int64_t* __restrict__ scr_off,
                              int64_t scr_base, double* __restrict__ scratch, const double* __restrict__ v,
                              int* __restrict__ colexp) {
  extern __shared__ int s_exp[];  // [8][nb] when colexp != NULL
  const int64_t b = b0 + blockIdx.x;
  const int64_t p0 = G.pt_ptr[b];
  const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
  const int ldp = (np + 7) & ~7;
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  double* base = scratch + (scr_off[b] - scr_base);
  const int64_t plane = static_cast<int64_t>(nb) * ldp;
  if (colexp) {
    for (int i = threadIdx.x; i < 8 * nb; i += blockDim.x) s_exp[i] = kNoExp;
    __syncthreads();
  }
  for (int item = threadIdx.x; item < np * na; item += blockDim.x) {
    const int a = item / np, p = item - a * np;
    const int A = G.bat_atoms[a0 + a];
    const int f0 = G.bat_atom_fn0[a0 + a];
    const double dx = G.x[p0 + p] - G.c_xyz[3 * A], dy = G.y[p0 + p] - G.c_xyz[3 * A + 1],
                 dz = G.z[p0 + p] - G.c_xyz[3 * A + 2];
    int eD = kNoExp;
    if (colexp) {
      const double D = G.w[p0 + p] * v[p0 + p];
      if (D != 0.0) eD = binexp(D);
    }
    atom_functions(B, G.c_sp[A], dx, dy, dz, [&](int k, double phi, double gx, double gy, double gz) {
      double* q = base + static_cast<int64_t>(f0 + k) * ldp + p;
      q[0] = phi;
      q[plane] = gx;
      q[2 * plane] = gy;
      q[3 * plane] = gz;
      if (colexp) {
        const double vals[4] = {phi, gx, gy, gz};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (vals[s] == 0.0) continue;
          const int e = binexp(vals[s]);
          atomicMax(&s_exp[(4 + s) * nb + f0 + k], e);
          if (eD != kNoExp) atomicMax(&s_exp[s * nb + f0 + k], e + eD);
        }
      }
    });
  }
  if (colexp) {
    __syncthreads();
    int* out = colexp + 8 * G.bat_fn_ptr[b];
    for (int i = threadIdx.x; i < 8 * nb; i += blockDim.x) out[i] = s_exp[i];
  }
}

q4c_status launch_basis_tiles(const q4c_tables* t, const q4c_grid* g, int64_t b0, int64_t b1, const double* v,
                              int* colexp, cudaStream_t s) {
  const size_t smem = colexp ? sizeof(int) * 8 * std::max(g->max_nb, 1) : 0;
  if (smem > 48 * 1024)
    Q4C_CUDA(cudaFuncSetAttribute(k_basis_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  KernelScope ks("basis", s);
  k_basis_tiles<<<static_cast<unsigned>(b1 - b0), 256, smem, s>>>(t->view(), g->view(), b0, g->d_scr_off, 0,
                                                                   g->d_scratch, v, colexp);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

// nf of the atom behind local atom a of a batch
__device__ __forceinline__ int local_nf(const DevBasis& B, const DevGrid& G, int a0, int a) {
  return __ldg(B.sp_nfn + G.c_sp[G.bat_atoms[a0 + a]]);
}

// ------------------------------------------------------------ products
// One CTA per 32x32 tile (ti <= tj) of one batch, 16x16 threads, 2x2
// elements each; accumulates V, W0 and SO directly on the upper triangle
// (i <= j) and scatters with FP64 atomics into the upper blocks.
constexpr int kT = 32, kK = 16;
__global__ void __launch_bounds__(256) k_products_fp64(DevBasis B, DevGrid G, const int4* __restrict__ tiles,
                                                       int64_t t0, const int64_t* __restrict__ scr_off,
                                                       int64_t scr_base, const double* __restrict__ scratch,
                                                       const double* __restrict__ v, double* V, double* W0,
                                                       double* SOx, double* SOy, double* SOz) {
  __shared__ double sa[4][kK][kT];  // D-scaled i side
  __shared__ double sb[4][kK][kT];  // j side
  __shared__ double sd[kK];
  const int4 tile = tiles[t0 + blockIdx.x];
  const int64_t b = tile.x;
  const int ti = tile.y, tj = tile.z;
  const int64_t p0 = G.pt_ptr[b];
  const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
  const int ldp = (np + 7) & ~7;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  const int64_t plane = static_cast<int64_t>(nb) * ldp;
  const double* base = scratch + (scr_off[b] - scr_base);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2][5];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int q = 0; q < 5; ++q) acc[u][w][q] = 0.0;

  for (int k0 = 0; k0 < np; k0 += kK) {
    if (threadIdx.x < kK) {
      const int p = k0 + threadIdx.x;
      sd[threadIdx.x] = p < np ? G.w[p0 + p] * v[p0 + p] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * kK * kT; e += blockDim.x) {
      const int q = e / (kK * kT), rem = e - q * kK * kT, f = rem / kK, kk = rem - f * kK;
      const int p = k0 + kk;
      const int fi = ti * kT + f, fj = tj * kT + f;
      const double ai = (p < np && fi < nb) ? base[q * plane + static_cast<int64_t>(fi) * ldp + p] : 0.0;
      const double bj = (p < np && fj < nb) ? base[q * plane + static_cast<int64_t>(fj) * ldp + p] : 0.0;
      sa[q][kk][f] = ai * sd[kk];
      sb[q][kk][f] = bj;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kK; ++kk) {
      double a[2][4], c[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[u][q] = sa[q][kk][2 * ty + u];
          c[u][q] = sb[q][kk][2 * tx + u];
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          acc[u][w][0] = fma(a[u][0], c[w][0], acc[u][w][0]);
          acc[u][w][1] = fma(a[u][1], c[w][1], fma(a[u][2], c[w][2], fma(a[u][3], c[w][3], acc[u][w][1])));
          acc[u][w][2] = fma(a[u][2], c[w][3], fma(-a[u][3], c[w][2], acc[u][w][2]));
          acc[u][w][3] = fma(a[u][3], c[w][1], fma(-a[u][1], c[w][3], acc[u][w][3]));
          acc[u][w][4] = fma(a[u][1], c[w][2], fma(-a[u][2], c[w][1], acc[u][w][4]));
        }
    }
    __syncthreads();
  }
  // scatter the upper triangle
  const int64_t f0 = G.bat_fn_ptr[b];
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const int64_t pp = G.bat_pair_ptr[b];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int i = ti * kT + 2 * ty + u, j = tj * kT + 2 * tx + w;
      if (i >= nb || j >= nb || i > j) continue;
      const int ii = G.fn_info[f0 + i], jj = G.fn_info[f0 + j];
      const int ai = ii >> 16, ki = ii & 0xffff, aj = jj >> 16, kj = jj & 0xffff;
      const int64_t off = G.pair_off[pp + static_cast<int64_t>(ai) * na + aj];
      if (off < 0) continue;
      const int64_t e = off + static_cast<int64_t>(ki) * local_nf(B, G, a0, aj) + kj;
      atomicAdd(V + e, acc[u][w][0]);
      atomicAdd(W0 + e, acc[u][w][1]);
      if (i != j) {
        atomicAdd(SOx + e, acc[u][w][2]);
        atomicAdd(SOy + e, acc[u][w][3]);
        atomicAdd(SOz + e, acc[u][w][4]);
      }
    }
}

// ------------------------------------------------- mirror + spinor blocks
// One CTA per block.  The batch kernels accumulate only the canonical half
// of the pattern: local functions are ordered by centre (cell, atom) with the
// cells lexicographic in T, so a pair i <= j always lands in a block (A, B, T)
// with T > 0, or T = 0 and A <= B.  Canonical blocks (role 1) are copied
// transposed into their partner (B, A, -T) (negated for SO); a block that is
// its own partner (A = B, T = 0; role 2) fills i > j from (j, i); role 0
// blocks are the copy targets.
__global__ void k_mirror(const int* __restrict__ blk_row, const int* __restrict__ blk_col,
                         const int* __restrict__ blk_T, const int* __restrict__ blk_role,
                         const int64_t* __restrict__ blk_off, const int* atom_sp, const int* sp_nfn, double* V,
                         double* W0, double* SOx, double* SOy, double* SOz) {
  const int q = blockIdx.x;
  const int role = blk_role[q];
  if (role == 0) return;
  const int A = blk_row[q], Bc = blk_col[q];
  const int nfA = sp_nfn[atom_sp[A]], nfB = sp_nfn[atom_sp[Bc]];
  const bool self = role == 2;
  const int64_t o = blk_off[q], oT = blk_off[blk_T[q]];
  for (int e = threadIdx.x; e < nfA * nfB; e += blockDim.x) {
    const int i = e / nfB, j = e - i * nfB;
    if (self && i <= j) continue;
    const int64_t src = self ? o + static_cast<int64_t>(j) * nfB + i : o + e;
    const int64_t dst = self ? o + e : oT + static_cast<int64_t>(j) * nfA + i;
    V[dst] = V[src];
    W0[dst] = W0[src];
    SOx[dst] = -SOx[src];
    SOy[dst] = -SOy[src];
    SOz[dst] = -SOz[src];
  }
}

// [[W0 + i SOz, SOy + i SOx], [-SOy + i SOx, W0 - i SOz]] per element
__global__ void k_spinor(const int* __restrict__ blk_row, const int* __restrict__ blk_col,
                         const int64_t* __restrict__ blk_off, const int* atom_sp, const int* sp_nfn,
                         const double* __restrict__ W0, const double* __restrict__ SOx,
                         const double* __restrict__ SOy, const double* __restrict__ SOz, double2* __restrict__ SS) {
  const int q = blockIdx.x;
  const int nfB = sp_nfn[atom_sp[blk_col[q]]];
  const int nfA = sp_nfn[atom_sp[blk_row[q]]];
  const int64_t o = blk_off[q];
  for (int e = threadIdx.x; e < nfA * nfB; e += blockDim.x) {
    const int i = e / nfB, j = e - i * nfB;
    const double w = W0[o + e], x = SOx[o + e], y = SOy[o + e], z = SOz[o + e];
    double2* r0 = SS + 4 * o + static_cast<int64_t>(2 * i) * (2 * nfB) + 2 * j;
    double2* r1 = r0 + 2 * nfB;
    r0[0] = make_double2(w, z);
    r0[1] = make_double2(y, x);
    r1[0] = make_double2(-y, x);
    r1[1] = make_double2(w, -z);
  }
}

q4c_status mirror_and_spinor(const q4c_grid* g, const q4c_matrices* out, cudaStream_t s) {
  const q4c_tables* t = g->tables;
  if (g->n_blocks == 0) return Q4C_OK;
  {
  KernelScope ks("mirror", s);
  k_mirror<<<static_cast<unsigned>(g->n_blocks), 128, 0, s>>>(g->d_blk_row, g->d_blk_col, g->d_blk_T,
                                                             g->d_blk_role, g->d_blk_off, g->d_atom_sp,
                                                             t->d_sp_nfn, out->V,
                                                             out->W0, out->SOx, out->SOy, out->SOz);
  }
  Q4C_CUDA(cudaGetLastError());
  if (out->spinor_SS) {
    KernelScope ks("spinor", s);
    k_spinor<<<static_cast<unsigned>(g->n_blocks), 128, 0, s>>>(
        g->d_blk_row, g->d_blk_col, g->d_blk_off, g->d_atom_sp, t->d_sp_nfn, out->W0, out->SOx, out->SOy,
        out->SOz, reinterpret_cast<double2*>(out->spinor_SS));
    Q4C_CUDA(cudaGetLastError());
  }
  return Q4C_OK;
}

// the products of one wave (its basis tiles in place)
q4c_status products_fp64_wave(const q4c_grid* g, int wv, const double* v, const q4c_matrices* out,
                              cudaStream_t s) {
  const int64_t t0 = g->wave_t0[wv], t1 = g->wave_t0[wv + 1];
  if (t1 <= t0) return Q4C_OK;
  KernelScope ks("products_fp64", s);
  k_products_fp64<<<static_cast<unsigned>(t1 - t0), 256, 0, s>>>(g->tables->view(), g->view(), g->d_tiles, t0,
                                                                   g->d_scr_off, 0, g->d_scratch, v, out->V,
                                                                   out->W0, out->SOx, out->SOy, out->SOz);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

q4c_status integrate_fp64(const q4c_tables* t, const q4c_grid* g, const double* v, const q4c_matrices* out,
                          cudaStream_t s) {
  double* outs[5] = {out->V, out->W0, out->SOx, out->SOy, out->SOz};
  for (double* o : outs) Q4C_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * g->nnz, s));
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 > b0) {
      if (q4c_status st = launch_basis_tiles(t, g, b0, b1, nullptr, nullptr, s)) return st;
    }
    if (q4c_status st = products_fp64_wave(g, static_cast<int>(wv), v, out, s)) return st;
  }
  return mirror_and_spinor(g, out, s);
}

// ------------------------------------------------------ per-column operator
// Eq. 19 in the scalar form of the large component: every element carries
// the eigenvalue and defining potential of its COLUMN's radial function,
//   F_ij = sum_p phi_i(p) theta_pj,  theta_pj = w_p (v_p + eps_j - V_j(|p - R_j|)) phi_j(p),
// so F is not symmetric: one CTA per 32x32 tile over all tile pairs of a
// batch, the column factors built while loading the j side, every element
// scattered (no mirror).  V_j: cubic in the knot index on each interval,
// the first knot's value below r_min and the last one's from r_c on.
__device__ __forceinline__ double column_potential(const DevBasis& B, const double* __restrict__ vcoef, int rad,
                                                   double r) {
  const double* c = vcoef + static_cast<int64_t>(rad) * (B.n_log - 1) * 4;
  if (r < B.r_min) return c[0];
  if (r >= B.r_c) {
    const double* e = c + (B.n_log - 2) * 4;
    return e[0] + e[1] + e[2] + e[3];
  }
  const double t = log(r * B.inv_rmin) * B.inv_h;
  const int k = min(max(static_cast<int>(t), 0), B.n_log - 2);
  const double s = t - k;
  const double* e = c + k * 4;
  return e[0] + s * (e[1] + s * (e[2] + s * e[3]));
}

__global__ void __launch_bounds__(256) k_columns_fp64(DevBasis B, DevGrid G, const int4* __restrict__ tiles,
                                                      const int64_t* __restrict__ scr_off,
                                                      const double* __restrict__ scratch,
                                                      const double* __restrict__ v, const double* __restrict__ eps,
                                                      const double* __restrict__ vcoef, double* F) {
  __shared__ double sa[kK][kT], sb[kK][kT];
  __shared__ double s_c[3][kT], s_eps[kT];
  __shared__ int s_rad[kT];
  const int4 tile = tiles[blockIdx.x];
  const int64_t b = tile.x;
  const int ti = tile.y, tj = tile.z;
  const int64_t p0 = G.pt_ptr[b];
  const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
  const int ldp = (np + 7) & ~7;
  const int64_t f0 = G.bat_fn_ptr[b];
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - f0);
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const double* base = scratch + scr_off[b];
  if (threadIdx.x < kT) {  // centre, radial and eigenvalue of each column function of the tile
    const int fj = tj * kT + threadIdx.x;
    int rad = -1;
    if (fj < nb) {
      const int info = G.fn_info[f0 + fj];
      const int c = G.bat_atoms[a0 + (info >> 16)], k = info & 0xffff;
      const int sp = G.c_sp[c], r0 = __ldg(B.sp_rad0 + sp), nr = __ldg(B.sp_nrad + sp);
      for (int q = 0, first = 0; q < nr; ++q) {
        const int n = 2 * __ldg(B.rad_l + r0 + q) + 1;
        if (k < first + n) {
          rad = r0 + q;
          break;
        }
        first += n;
      }
      s_c[0][threadIdx.x] = G.c_xyz[3 * c];
      s_c[1][threadIdx.x] = G.c_xyz[3 * c + 1];
      s_c[2][threadIdx.x] = G.c_xyz[3 * c + 2];
      s_eps[threadIdx.x] = rad >= 0 ? eps[rad] : 0.0;
    }
    s_rad[threadIdx.x] = rad;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < np; k0 += kK) {
    for (int e = threadIdx.x; e < kK * kT; e += blockDim.x) {
      const int f = e / kK, kk = e - f * kK, p = k0 + kk;
      const int fi = ti * kT + f, fj = tj * kT + f;
      sa[kk][f] = (p < np && fi < nb) ? base[static_cast<int64_t>(fi) * ldp + p] : 0.0;
      double th = 0.0;
      if (p < np && fj < nb && s_rad[f] >= 0) {
        const int64_t gp = p0 + p;
        const double dx = G.x[gp] - s_c[0][f], dy = G.y[gp] - s_c[1][f], dz = G.z[gp] - s_c[2][f];
        const double Vr = column_potential(B, vcoef, s_rad[f], centre_distance(dx, dy, dz));
        th = base[static_cast<int64_t>(fj) * ldp + p] * G.w[gp] * (v[gp] + s_eps[f] - Vr);
      }
      sb[kk][f] = th;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kK; ++kk) {
      const double a0v = sa[kk][2 * ty], a1v = sa[kk][2 * ty + 1];
      const double c0v = sb[kk][2 * tx], c1v = sb[kk][2 * tx + 1];
      acc[0][0] = fma(a0v, c0v, acc[0][0]);
      acc[0][1] = fma(a0v, c1v, acc[0][1]);
      acc[1][0] = fma(a1v, c0v, acc[1][0]);
      acc[1][1] = fma(a1v, c1v, acc[1][1]);
    }
    __syncthreads();
  }
  const int64_t pp = G.bat_pair_ptr[b];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int i = ti * kT + 2 * ty + u, j = tj * kT + 2 * tx + w;
      if (i >= nb || j >= nb) continue;
      const int ii = G.fn_info[f0 + i], jj = G.fn_info[f0 + j];
      const int64_t off = G.pair_off[pp + static_cast<int64_t>(ii >> 16) * na + (jj >> 16)];
      if (off < 0) continue;
      atomicAdd(F + off + static_cast<int64_t>(ii & 0xffff) * local_nf(B, G, a0, jj >> 16) + (jj & 0xffff),
                acc[u][w]);
    }
}

q4c_status integrate_columns_fp64(const q4c_tables* t, const q4c_grid* g, const double* v, double* F,
                                  cudaStream_t s) {
  Q4C_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * g->nnz, s));
  const DevBasis B = t->view();
  const DevGrid G = g->view();
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    const int64_t t0 = g->colt_w0[wv], t1 = g->colt_w0[wv + 1];  // every tile pair of the wave's batches
    if (b1 <= b0 || t1 <= t0) continue;
    if (q4c_status st = launch_basis_tiles(t, g, b0, b1, nullptr, nullptr, s)) return st;
    KernelScope ks("columns_fp64", s);
    k_columns_fp64<<<static_cast<unsigned>(t1 - t0), 256, 0, s>>>(B, G, g->d_col_tiles + t0, g->d_scr_off,
                                                                    g->d_scratch, v, t->d_col_eps, t->d_col_coef, F);
    Q4C_CUDA(cudaGetLastError());
  }
  return Q4C_OK;
}

// ------------------------------------------------------------- density
// One CTA per batch, one thread per point; P rows gathered into shared
// memory kRows at a time: n_p = sum_i Phi_pi sum_j P_ij Phi_pj.  kRows is 16,
// or fewer where 16 rows of a large batch would not fit in shared memory.
template <int kRows>
__global__ void k_density_fp64(DevBasis B, DevGrid G, int64_t b0, const int64_t* __restrict__ scr_off,
                               const double* __restrict__ scratch, const double* __restrict__ P,
                               double* __restrict__ n_out) {
  extern __shared__ double sP[];  // [kRows][nb]
  const int64_t b = b0 + blockIdx.x;
  const int64_t p0 = G.pt_ptr[b];
  const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
  const int ldp = (np + 7) & ~7;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  const int64_t f0 = G.bat_fn_ptr[b];
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const int64_t pp = G.bat_pair_ptr[b];
  const double* Phi = scratch + scr_off[b];
  for (int pbase = 0; pbase < np; pbase += blockDim.x) {
    const int p = pbase + threadIdx.x;
    double acc = 0.0;
    for (int i0 = 0; i0 < nb; i0 += kRows) {
      const int rows = min(kRows, nb - i0);
      __syncthreads();
      for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
        const int r = e / nb, j = e - r * nb;
        const int ii = G.fn_info[f0 + i0 + r], jj = G.fn_info[f0 + j];
        const int64_t off = G.pair_off[pp + static_cast<int64_t>(ii >> 16) * na + (jj >> 16)];
        sP[e] = off < 0 ? 0.0 : P[off + static_cast<int64_t>(ii & 0xffff) * local_nf(B, G, a0, jj >> 16) +
                                  (jj & 0xffff)];
      }
      __syncthreads();
      if (p < np) {
        double t[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) t[r] = 0.0;
        for (int j = 0; j < nb; ++j) {
          const double pj = Phi[static_cast<int64_t>(j) * ldp + p];
#pragma unroll
          for (int r = 0; r < kRows; ++r)
            if (r < rows) t[r] = fma(sP[r * nb + j], pj, t[r]);
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r)
          if (r < rows) acc = fma(Phi[static_cast<int64_t>(i0 + r) * ldp + p], t[r], acc);
      }
    }
    if (p < np) n_out[p0 + p] = acc;
  }
}

// the density of one wave (its basis tiles in place)
q4c_status density_fp64_wave(const q4c_grid* g, int wv, const double* P, double* n, cudaStream_t s) {
  const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
  if (b1 <= b0) return Q4C_OK;
  constexpr size_t kSmemMax = 232448;
  const size_t row = sizeof(double) * std::max(g->max_nb, 1);  // one P row of a batch
  const int rows = 16 * row <= kSmemMax ? 16 : 8 * row <= kSmemMax ? 8 : 4;
  if (rows * row > kSmemMax) {
    set_error("the FP64 density needs at most 7264 active functions per batch");
    return Q4C_EUNSUPPORTED;
  }
  const size_t smem = rows * row;
  auto k_density = rows == 16 ? k_density_fp64<16> : rows == 8 ? k_density_fp64<8> : k_density_fp64<4>;
  Q4C_CUDA(cudaFuncSetAttribute(k_density, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  KernelScope ks("density_fp64", s);
  k_density<<<static_cast<unsigned>(b1 - b0), 128, smem, s>>>(g->tables->view(), g->view(), b0, g->d_scr_off,
                                                                   g->d_scratch, P, n);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

q4c_status density_fp64(const q4c_tables* t, const q4c_grid* g, const double* P, double* n, cudaStream_t s) {
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_basis_tiles(t, g, b0, b1, nullptr, nullptr, s)) return st;
    if (q4c_status st = density_fp64_wave(g, static_cast<int>(wv), P, n, s)) return st;
  }
  return Q4C_OK;
}

// ------------------------------------------------------------- adjoint
// dL/dv_p = w_p sum_ij [G^V phi_i phi_j + G^W grad_i.grad_j
//                        + G^x (Y_i Z_j - Z_i Y_j) + G^y (Z_i X_j - X_i Z_j)
//                        + G^z (X_i Y_j - Y_i X_j)]
// kRowsB rows of G per pass: 8, or 4, 2 or 1 where five 8-row blocks of a
// large batch would not fit in shared memory
template <int kRowsB>
__global__ void k_backward_fp64(DevBasis B, DevGrid G, int64_t b0, const int64_t* __restrict__ scr_off,
                                const double* __restrict__ scratch, const double* GV, const double* GW,
                                const double* Gx, const double* Gy, const double* Gz, double* __restrict__ dLdv,
                                int weighted) {
  extern __shared__ double sG[];  // [5][kRowsB][nb]
  const int64_t b = b0 + blockIdx.x;
  const int64_t p0 = G.pt_ptr[b];
  const int np = static_cast<int>(G.pt_ptr[b + 1] - p0);
  const int ldp = (np + 7) & ~7;
  const int nb = static_cast<int>(G.bat_fn_ptr[b + 1] - G.bat_fn_ptr[b]);
  const int64_t plane = static_cast<int64_t>(nb) * ldp;
  const int64_t f0 = G.bat_fn_ptr[b];
  const int a0 = G.bat_atom_ptr[b], na = G.bat_atom_ptr[b + 1] - a0;
  const int64_t pp = G.bat_pair_ptr[b];
  const double* T = scratch + scr_off[b];
  const double* Gm[5] = {GV, GW, Gx, Gy, Gz};
  for (int pbase = 0; pbase < np; pbase += blockDim.x) {
    const int p = pbase + threadIdx.x;
    double acc = 0.0;
    for (int i0 = 0; i0 < nb; i0 += kRowsB) {
      const int rows = min(kRowsB, nb - i0);
      __syncthreads();
      for (int e = threadIdx.x; e < rows * nb; e += blockDim.x) {
        const int r = e / nb, j = e - r * nb;
        const int ii = G.fn_info[f0 + i0 + r], jj = G.fn_info[f0 + j];
        const int64_t off = G.pair_off[pp + static_cast<int64_t>(ii >> 16) * na + (jj >> 16)];
        const int64_t el = off < 0 ? -1 : off + static_cast<int64_t>(ii & 0xffff) * local_nf(B, G, a0, jj >> 16) +
                                              (jj & 0xffff);
#pragma unroll
        for (int m = 0; m < 5; ++m)
          sG[(m * kRowsB + r) * nb + j] = (el < 0 || Gm[m] == nullptr) ? 0.0 : Gm[m][el];
      }
      __syncthreads();
      if (p < np) {
        double fi[kRowsB][4];
#pragma unroll
        for (int r = 0; r < kRowsB; ++r)
#pragma unroll
          for (int q = 0; q < 4; ++q) fi[r][q] = r < rows ? T[q * plane + static_cast<int64_t>(i0 + r) * ldp + p] : 0.0;
        for (int j = 0; j < nb; ++j) {
          const double pj = T[static_cast<int64_t>(j) * ldp + p], xj = T[plane + static_cast<int64_t>(j) * ldp + p],
                       yj = T[2 * plane + static_cast<int64_t>(j) * ldp + p],
                       zj = T[3 * plane + static_cast<int64_t>(j) * ldp + p];
#pragma unroll
          for (int r = 0; r < kRowsB; ++r) {
            if (r >= rows) continue;
            const double* gr = sG + r * nb + j;
            double s = gr[0] * fi[r][0] * pj;
            s = fma(gr[kRowsB * nb], fi[r][1] * xj + fi[r][2] * yj + fi[r][3] * zj, s);
            s = fma(gr[2 * kRowsB * nb], fi[r][2] * zj - fi[r][3] * yj, s);
            s = fma(gr[3 * kRowsB * nb], fi[r][3] * xj - fi[r][1] * zj, s);
            s = fma(gr[4 * kRowsB * nb], fi[r][1] * yj - fi[r][2] * xj, s);
            acc += s;
          }
        }
      }
    }
    if (p < np) dLdv[p0 + p] = weighted ? G.w[p0 + p] * acc : acc;
  }
}

// the adjoint (weighted) or gradient density (unweighted) of one wave (its
// basis tiles in place)
q4c_status backward_fp64_wave(const q4c_grid* g, int wv, const q4c_matrices* Gm, double* dLdv, bool weighted,
                              cudaStream_t s) {
  const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
  if (b1 <= b0) return Q4C_OK;
  constexpr size_t kSmemMax = 232448;
  const size_t row = sizeof(double) * 5 * std::max(g->max_nb, 1);  // five G rows of a batch
  if (row > kSmemMax) {
    set_error("the FP64 adjoint needs at most 5811 active functions per batch");
    return Q4C_EUNSUPPORTED;
  }
  const int rows = 8 * row <= kSmemMax ? 8 : 4 * row <= kSmemMax ? 4 : 2 * row <= kSmemMax ? 2 : 1;
  const size_t smem = rows * row;
  auto kern = rows == 8 ? k_backward_fp64<8> : rows == 4 ? k_backward_fp64<4> : rows == 2 ? k_backward_fp64<2>
                                                                                        : k_backward_fp64<1>;
  Q4C_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  KernelScope ks("backward_fp64", s);
  kern<<<static_cast<unsigned>(b1 - b0), 128, smem, s>>>(g->tables->view(), g->view(), b0, g->d_scr_off,
                                                         g->d_scratch, Gm->V, Gm->W0, Gm->SOx, Gm->SOy, Gm->SOz,
                                                         dLdv, weighted ? 1 : 0);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

q4c_status backward_fp64(const q4c_tables* t, const q4c_grid* g, const q4c_matrices* Gm, double* dLdv,
                         cudaStream_t s, bool weighted) {
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    const int64_t b0 = g->wave_b0[wv], b1 = g->wave_b0[wv + 1];
    if (b1 <= b0) continue;
    if (q4c_status st = launch_basis_tiles(t, g, b0, b1, nullptr, nullptr, s)) return st;
    if (q4c_status st = backward_fp64_wave(g, static_cast<int>(wv), Gm, dLdv, weighted, s)) return st;
  }
  return Q4C_OK;
}

// ---------------------------------------------------------- basis probe
__global__ void k_basis_eval(DevBasis B, DevGrid G, int n_basis, const int* __restrict__ atom_fn0, int64_t n_pts,
                             const double* __restrict__ xyz, double* __restrict__ phi, double* __restrict__ grad) {
  const int64_t item = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (item >= n_pts * G.n_atoms) return;
  const int A = static_cast<int>(item / n_pts);
  const int64_t p = item - A * n_pts;
  const int f0 = atom_fn0[A];
  atom_functions(B, G.atom_sp[A], xyz[3 * p] - G.atom_xyz[3 * A], xyz[3 * p + 1] - G.atom_xyz[3 * A + 1],
                 xyz[3 * p + 2] - G.atom_xyz[3 * A + 2], [&](int k, double v, double gx, double gy, double gz) {
                   const int64_t o = static_cast<int64_t>(f0 + k) * n_pts + p;
                   phi[o] = v;
                   grad[3 * o] = gx;
                   grad[3 * o + 1] = gy;
                   grad[3 * o + 2] = gz;
                 });
}

q4c_status basis_eval(const q4c_tables* t, const q4c_grid* g, int64_t n_pts, const double* xyz, double* phi,
                      double* grad, cudaStream_t s) {
  if (n_pts == 0) return Q4C_OK;
  const int64_t items = n_pts * g->n_atoms;
  KernelScope ks("basis_eval", s);
  k_basis_eval<<<static_cast<unsigned>((items + 127) / 128), 128, 0, s>>>(t->view(), g->view(), g->n_basis,
                                                                         g->d_atom_fn0, n_pts, xyz, phi, grad);
  Q4C_CUDA(cudaGetLastError());
  return Q4C_OK;
}

}  // namespace q4c
