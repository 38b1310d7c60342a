// q4c_integrate_noalloc: the FP64 integration with its per-batch basis-tile
// workspace taken from a fixed, statically reserved device array instead of
// the grid's own workspace, so the call itself allocates nothing.
//
// It serves callers that cannot allocate device memory when they integrate:
// for example a host application that has handed the whole device memory to
// its own pool allocator, or a latency-bound loop that must not call
// cudaMalloc/cudaFree (they can synchronise the device and take
// milliseconds).  Such callers still pass inputs and outputs they own.
//
// The workspace is the file-scope array below (kNoAllocBytes = 64 MiB).
// Every GPU that loads this library reserves it until the process exits.
// Batches are processed in waves that fit it; a single batch whose tiles
// (4 n_b ceil8(n_p) doubles) exceed it is rejected with Q4C_EUNSUPPORTED.
// All calls share the array: calls that overlap on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.  Nothing in it needs to start at zero: every tile element a
// product kernel reads is written first by the basis kernel of the same wave.
//
// Host code cannot use the array's name as a device address; the first call
// on each device resolves it with cudaGetSymbolAddress (with that device
// current) and caches it for the rest of the process.  That first call should
// therefore come before any stream capture, and a process that destroys a
// device's primary context (cudaDeviceReset) must not call this entry point
// on that device again: the cached address belonged to the old context.
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace q4c {

constexpr int64_t kNoAllocBytes = int64_t(64) << 20;
constexpr int64_t kNoAllocDoubles = kNoAllocBytes / 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// kernels of the FP64 path (fp64.cu)
__global__ void k_basis_tiles(DevBasis B, DevGrid G, int64_t b0, const int64_t* __restrict__ scr_off,
                              int64_t scr_base, double* __restrict__ scratch, const double* __restrict__ v,
                              int* __restrict__ colexp);
__global__ void k_products_fp64(DevBasis B, DevGrid G, const int4* __restrict__ tiles, int64_t t0,
                                const int64_t* __restrict__ scr_off, int64_t scr_base,
                                const double* __restrict__ scratch,
                                const double* __restrict__ v, double* V, double* W0, double* SOx, double* SOy,
                                double* SOz);

namespace {
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// device address of the static workspace on the current device (resolved
// once per device)
q4c_status workspace(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error(std::string("q4c_integrate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return Q4C_ECUDA;
    }
    g_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_ptr[dev]);
  return Q4C_OK;
}
}  // namespace

}  // namespace q4c

using namespace q4c;

extern "C" q4c_status q4c_integrate_noalloc(const q4c_tables* t, const q4c_grid* g, const double* v,
                                           const q4c_matrices* out, q4c_stream stream) {
  Q4C_CHECK_ARG(t && g && v && out && out->V && out->W0 && out->SOx && out->SOy && out->SOz,
                "q4c_integrate_noalloc: NULL argument");
  Q4C_CHECK_ARG(g->tables == t, "q4c_integrate_noalloc: grid was partitioned with different tables");
  int dev = -1;
  Q4C_CUDA(cudaGetDevice(&dev));
  Q4C_CHECK_ARG(dev == g->device, "q4c_integrate_noalloc: current device differs from the grid's device");
  Q4C_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "q4c_integrate_noalloc: device index out of range");
  // reject before touching the device if some batch cannot fit
  for (int64_t b = 0; b < g->n_batches; ++b) {
    const int64_t np = g->h_pt_ptr[b + 1] - g->h_pt_ptr[b];
    const int64_t nb = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
    if (4 * nb * ((np + 7) / 8 * 8) > kNoAllocDoubles) {
      set_error("q4c_integrate_noalloc: a batch's basis tiles exceed the 64 MiB static workspace");
      return Q4C_EUNSUPPORTED;
    }
  }
  double* ws = nullptr;
  if (q4c_status st = workspace(dev, &ws)) return st;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* outs[5] = {out->V, out->W0, out->SOx, out->SOy, out->SOz};
  for (double* o : outs) Q4C_CUDA(cudaMemsetAsync(o, 0, sizeof(double) * g->nnz, s));
  const DevBasis B = t->view();
  const DevGrid G = g->view();
  // the grid's own waves keep per-batch tile offsets cumulative in batch
  // order; sub-waves of them that fit the static array reuse those offsets,
  // and the kernels subtract the sub-wave's first offset (base)
  int64_t tile = 0;
  for (size_t wv = 0; wv + 1 < g->wave_b0.size(); ++wv) {
    int64_t b = g->wave_b0[wv];
    const int64_t wb1 = g->wave_b0[wv + 1];
    tile = g->wave_t0[wv];
    while (b < wb1) {
      const int64_t b_first = b, t_first = tile, base = g->h_scr_off[b];
      while (b < wb1) {
        const int64_t np = g->h_pt_ptr[b + 1] - g->h_pt_ptr[b];
        const int64_t nb = g->h_bat_fn_ptr[b + 1] - g->h_bat_fn_ptr[b];
        const int64_t end = g->h_scr_off[b] + 4 * nb * ((np + 7) / 8 * 8) - base;
        if (end > kNoAllocDoubles) break;
        const int64_t nt = (nb + 31) / 32;
        tile += nt * (nt + 1) / 2;
        ++b;
      }
      {
        KernelScope ks("basis", s);
        k_basis_tiles<<<static_cast<unsigned>(b - b_first), 256, 0, s>>>(B, G, b_first, g->d_scr_off, base,
                                                                         ws, nullptr, nullptr);
      }
      Q4C_CUDA(cudaGetLastError());
      if (tile > t_first) {
        KernelScope ks("products_fp64", s);
        k_products_fp64<<<static_cast<unsigned>(tile - t_first), 256, 0, s>>>(
            B, G, g->d_tiles, t_first, g->d_scr_off, base, ws, v, out->V, out->W0, out->SOx, out->SOy, out->SOz);
      }
      Q4C_CUDA(cudaGetLastError());
    }
  }
  return mirror_and_spinor(g, out, s);
}
