// Momentum and energy sums without any device allocation.
//
// The same sums the gravity call reports (sum m a, sum |m a|, 1/2 sum m Phi),
// computed over caller arrays by a two-pass reduction whose per-tile partial
// sums live in a fixed file-scope device array instead of context-owned
// scratch.  It exists for callers that cannot call cudaMalloc: code running
// under a custom or pre-reserved memory pool, or code that must not change the
// device's memory footprint once running.  The paper has no counterpart.
//
// Host code never passes the array's name to a kernel: in host code that name
// is only a host-side stand-in.  The device address is obtained once per
// device with cudaGetSymbolAddress (with that device current) and cached.
#include <mutex>

#include "sfmm_internal.cuh"

namespace {

constexpr int NOALLOC_TILE = 4096;                       // particles per partial
constexpr int NOALLOC_MAX_TILES = 16384;                 // 640 KB of partials
constexpr int64_t NOALLOC_MAX_N = (int64_t)NOALLOC_TILE * NOALLOC_MAX_TILES;  // 67,108,864
static_assert(NOALLOC_MAX_N == SFMM_NOALLOC_MAX_N, "header and implementation disagree");
constexpr int NOALLOC_NT = 256;
constexpr int NOALLOC_MAXDEV = 64;

// Per-tile partial sums: 5 doubles per tile.  Every call writes exactly the
// tiles it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_TILES * 5];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[NOALLOC_MAXDEV] = {};

__global__ void k_noalloc_tiles(int64_t n, const double* __restrict__ mass, const double* __restrict__ acc,
                                const double* __restrict__ pot, double* __restrict__ partials) {
  __shared__ double sh[5][NOALLOC_NT];
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t base = (int64_t)blockIdx.x * NOALLOC_TILE;
  for (int k = threadIdx.x; k < NOALLOC_TILE; k += NOALLOC_NT) {
    const int64_t i = base + k;
    if (i >= n) break;
    const double m = mass[i];
    const double ax = m * acc[3 * i], ay = m * acc[3 * i + 1], az = m * acc[3 * i + 2];
    s[0] += ax;
    s[1] += ay;
    s[2] += az;
    s[3] += fabs(ax) + fabs(ay) + fabs(az);
    if (pot) s[4] += m * pot[i];
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = NOALLOC_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) partials[5 * (int64_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_noalloc_final(int ntiles, const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sh[5][NOALLOC_NT];
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < ntiles; t += NOALLOC_NT)
    for (int c = 0; c < 5; ++c) s[c] += partials[5 * (int64_t)t + c];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = NOALLOC_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = (threadIdx.x == 4) ? 0.5 * sh[4][0] : sh[threadIdx.x][0];
}

// Device address of the partials array on the current device (first call on
// a device looks it up; later calls reuse it).
int noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= NOALLOC_MAXDEV) return SFMM_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SFMM_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return SFMM_OK;
}

}  // namespace

extern "C" int sfmm_reduce_noalloc(int64_t n, const double* mass, const double* acc, const double* pot,
                                   double* out, void* stream) {
  if (n < 1 || n > NOALLOC_MAX_N) return SFMM_EINVAL;
  if (!mass || !acc || !out) return SFMM_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SFMM_ECUDA;
  }
  double* partials = nullptr;
  int rc = noalloc_scratch(dev, &partials);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ntiles = (int)((n + NOALLOC_TILE - 1) / NOALLOC_TILE);
  k_noalloc_tiles<<<ntiles, NOALLOC_NT, 0, st>>>(n, mass, acc, pot, partials);
  k_noalloc_final<<<1, NOALLOC_NT, 0, st>>>(ntiles, partials, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFMM_OK : SFMM_ECUDA;
}
