// Right-hand-side assembly that allocates nothing (see mp_poisson_rhs_noalloc
// in include/mp_poisson.h).
//
// Scratch lives in a file-scope device array instead of memory obtained from
// cudaMalloc: every GPU that loads this library holds it until the process
// exits.  Host code must not pass the array's name to a kernel (in host code
// the name is only a host-side stand-in for the symbol); the device address
// is looked up once per device with cudaGetSymbolAddress and that address is
// what the kernels receive.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mp_poisson.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_BLOCK = NA_THREADS * 8;
constexpr int NA_MAX_BLOCKS = 65536;          // partial sums held by the scratch array
constexpr int NA_MAX_DEVICES = 64;
// slot NA_MAX_BLOCKS holds the mean
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS + 32];

std::mutex g_mu;
double *g_addr[NA_MAX_DEVICES] = {};

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double na_block_sum(double v) {
  __shared__ double red[NA_THREADS / 32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = na_warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < NA_THREADS / 32 ? red[lane] : 0.0;
    s = na_warp_sum(s);
  }
  return s;
}

// b = rhs + J on this block's cells; partial sum of the block into scratch
__global__ void na_add_partial(const double *__restrict__ rhs, const double *__restrict__ J,
                               double *__restrict__ b, long long n, double *__restrict__ scratch) {
  long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  double acc = 0.0;
  for (int q = 0; q < NA_CELLS_PER_BLOCK / NA_THREADS; ++q) {
    long long e = base + (long long)q * NA_THREADS + threadIdx.x;
    if (e < n) {
      double v = rhs[e] + J[e];
      b[e] = v;
      acc += v;
    }
  }
  double s = na_block_sum(acc);
  if (threadIdx.x == 0) scratch[blockIdx.x] = s;
}

// one block: mean of the partials (fixed order) into scratch[NA_MAX_BLOCKS]
__global__ void na_mean(double *__restrict__ scratch, int nblocks, long long n) {
  double acc = 0.0;
  for (int e = threadIdx.x; e < nblocks; e += NA_THREADS) acc += scratch[e];
  double s = na_block_sum(acc);
  if (threadIdx.x == 0) scratch[NA_MAX_BLOCKS] = s / (double)n;
}

__global__ void na_sub_mean(double *__restrict__ b, long long n,
                            const double *__restrict__ scratch) {
  double m = scratch[NA_MAX_BLOCKS];
  long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  for (int q = 0; q < NA_CELLS_PER_BLOCK / NA_THREADS; ++q) {
    long long e = base + (long long)q * NA_THREADS + threadIdx.x;
    if (e < n) b[e] -= m;
  }
}

// Device address of the scratch array for the current device, looked up
// once per device (with that device current) and cached.
mp_status scratch_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return MP_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MP_ERR_CUDA;
    }
    g_addr[dev] = (double *)p;
  }
  *out = g_addr[dev];
  return MP_OK;
}

}  // namespace

extern "C" mp_status mp_poisson_rhs_noalloc(long long ncells, const double *rhs_dev,
                                            const double *J_dev, double *b_dev, void *stream) {
  if (ncells <= 0 || ncells > MP_NOALLOC_MAX_CELLS || !rhs_dev || !J_dev || !b_dev)
    return MP_ERR_INVALID_ARG;
  double *scratch = nullptr;
  mp_status s = scratch_address(&scratch);
  if (s != MP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int nblocks = (int)((ncells + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  na_add_partial<<<nblocks, NA_THREADS, 0, st>>>(rhs_dev, J_dev, b_dev, ncells, scratch);
  na_mean<<<1, NA_THREADS, 0, st>>>(scratch, nblocks, ncells);
  na_sub_mean<<<nblocks, NA_THREADS, 0, st>>>(b_dev, ncells, scratch);
  if (cudaGetLastError() != cudaSuccess) return MP_ERR_CUDA;
  return MP_OK;
}
