// igks_noalloc.cu -- residual norms without any allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: code that runs while another
// component is capturing the stream into a CUDA graph, hosts whose GPU memory is handed
// out only by their own pool or arena, and real-time loops where an allocation's
// latency or failure is not acceptable. igks_residual_norms_noalloc gives them the
// per-solve residual norms of one iteration (the same reduction the iteration itself
// performs before its CFL update) using only memory the caller passes in plus a fixed
// scratch array that lives in this file's device data.
//
// The scratch array is a file-scope __device__ array: every GPU that loads the library
// holds IGKS_NOALLOC_MAX_CELLS / 256 * 2 doubles (64 KiB) of it until the process exits.
// Host code cannot use the array's name as a device address; the device address is
// looked up with cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device. Make that first call before any stream capture.
// All calls share the one array and it keeps the last call's contents: each call writes
// every partial it later reads, so nothing needs clearing, but calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/igks.h"

namespace {

constexpr int NB_THREADS = 256;
constexpr int MAX_BLOCKS = IGKS_NOALLOC_MAX_CELLS / NB_THREADS;
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) double g_norm_scratch[2 * MAX_BLOCKS];

// per-block max |M_rho| and sum of (M_rho / area)^2, same reduction order as the
// iteration's residual kernel (warp butterfly, then the warps in order)
__global__ void __launch_bounds__(NB_THREADS) k_norm_partials(const double* m_rho, const double* area, int n,
                                                              double* part, int nb) {
  const int i = blockIdx.x * NB_THREADS + threadIdx.x;
  double rmax = 0.0, r2 = 0.0;
  if (i < n) {
    double m = m_rho[i];
    rmax = fabs(m);
    double q = m / area[i];
    r2 = q * q;
  }
  __shared__ double smax[NB_THREADS / 32], ssum[NB_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if ((threadIdx.x & 31) == 0) { smax[threadIdx.x >> 5] = rmax; ssum[threadIdx.x >> 5] = r2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NB_THREADS / 32; w++) { a = fmax(a, smax[w]); b += ssum[w]; }
    part[blockIdx.x] = a;
    part[nb + blockIdx.x] = b;
  }
}

// blocks in order: out[0] = max |M_rho|, out[1] = RMS over cells of M_rho / area
__global__ void k_norm_final(const double* part, int nb, int n, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nb; k++) { a = fmax(a, part[k]); b += part[nb + k]; }
  out[0] = a;
  out[1] = sqrt(b / (double)n);
}

std::mutex g_mu;
double* g_scratch_addr[MAX_DEVICES] = {};
thread_local std::string g_err;

}  // namespace

// message of the last failed call of this entry point on the calling thread
const char* igks_noalloc_last_error_() { return g_err.c_str(); }

extern "C" int igks_residual_norms_noalloc(const double* m_rho, const double* area, int32_t n_cells,
                                           double* out, void* stream) {
  if (!m_rho || !area || !out || n_cells <= 0) {
    g_err = "igks_residual_norms_noalloc: null pointer or non-positive n_cells";
    return IGKS_EINVAL;
  }
  if (n_cells > IGKS_NOALLOC_MAX_CELLS) {
    g_err = "igks_residual_norms_noalloc: n_cells " + std::to_string(n_cells) + " exceeds the maximum " +
            std::to_string(IGKS_NOALLOC_MAX_CELLS) + " of its fixed scratch array";
    return IGKS_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_err = std::string("igks_residual_norms_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
    return IGKS_ECUDA;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    g_err = "igks_residual_norms_noalloc: device ordinal " + std::to_string(dev) +
            " is beyond the " + std::to_string(MAX_DEVICES) + " devices it keeps a scratch address for";
    return IGKS_EINVAL;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      // set-up, once per device: the device address of the file-scope scratch array
      e = cudaGetSymbolAddress((void**)&g_scratch_addr[dev], g_norm_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        g_err = std::string("igks_residual_norms_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return IGKS_ECUDA;
      }
    }
    scratch = g_scratch_addr[dev];
  }
  const int nb = (n_cells + NB_THREADS - 1) / NB_THREADS;
  cudaStream_t s = (cudaStream_t)stream;
  k_norm_partials<<<nb, NB_THREADS, 0, s>>>(m_rho, area, n_cells, scratch, nb);
  k_norm_final<<<1, 32, 0, s>>>(scratch, nb, n_cells, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("igks_residual_norms_noalloc: launch: ") + cudaGetErrorString(e);
    return IGKS_ECUDA;
  }
  return IGKS_OK;
}
