// Momentum and energy sums without any device allocation.
//
// The same sums the gravity call reports (sum m a, sum |m a|, 1/2 sum m Phi),
// computed over caller arrays by a two-pass compensated reduction whose
// per-tile partial sums live in a fixed file-scope device array instead of
// context-owned scratch.  It exists for callers that cannot call cudaMalloc:
// code running under a custom or pre-reserved memory pool, or code that must
// not change the device's memory footprint once running.  The paper has no
// counterpart.
//
// Host code never passes the array's name to a kernel: in host code that name
// is only a host-side stand-in.  The device address is obtained with
// cudaGetSymbolAddress (with the device current) and cached per device and
// CUDA context: a device reset or a new primary context changes the context
// handle, and the next call then looks the address up again.
#include <mutex>

#include "sfmm_internal.cuh"

namespace {

constexpr int NOALLOC_TILE = 4096;                       // particles per partial
constexpr int NOALLOC_MAX_TILES = 16384;                 // 1.25 MB of partials
constexpr int64_t NOALLOC_MAX_N = (int64_t)NOALLOC_TILE * NOALLOC_MAX_TILES;  // 67,108,864
static_assert(NOALLOC_MAX_N == SFMM_NOALLOC_MAX_N, "header and implementation disagree");
constexpr int NOALLOC_NT = 256;
constexpr int NOALLOC_MAXDEV = 64;

// Per-tile partial sums: 5 compensated sums (s, then c) = 10 doubles per
// tile.  Every call writes exactly the tiles it reads, so nothing has to
// start at zero.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_TILES * 10];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[NOALLOC_MAXDEV] = {};
void* g_noalloc_ctx[NOALLOC_MAXDEV] = {};  // CUDA context the cached address belongs to

__device__ __forceinline__ void noalloc_block_merge(sfmm::csum (&s)[5], double (&sh)[10][NOALLOC_NT]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    sh[c][threadIdx.x] = s[c].s;
    sh[5 + c][threadIdx.x] = s[c].c;
  }
  __syncthreads();
  for (int w = NOALLOC_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) {
        sfmm::csum a{sh[c][threadIdx.x], sh[5 + c][threadIdx.x]};
        sfmm::cs_merge(a, sh[c][threadIdx.x + w], sh[5 + c][threadIdx.x + w]);
        sh[c][threadIdx.x] = a.s;
        sh[5 + c][threadIdx.x] = a.c;
      }
    __syncthreads();
  }
}

__global__ void k_noalloc_tiles(int64_t n, const double* __restrict__ mass, const double* __restrict__ acc,
                                const double* __restrict__ pot, double* __restrict__ partials) {
  __shared__ double sh[10][NOALLOC_NT];
  sfmm::csum s[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
  const int64_t base = (int64_t)blockIdx.x * NOALLOC_TILE;
  for (int k = threadIdx.x; k < NOALLOC_TILE; k += NOALLOC_NT) {
    const int64_t i = base + k;
    if (i >= n) break;
    const double m = mass[i];
    const double ax = m * acc[3 * i], ay = m * acc[3 * i + 1], az = m * acc[3 * i + 2];
    sfmm::cs_add(s[0], ax);
    sfmm::cs_add(s[1], ay);
    sfmm::cs_add(s[2], az);
    // same-sign sums: plain additions (no cancellation to compensate)
    s[3].s = __dadd_rn(s[3].s, __dadd_rn(__dadd_rn(fabs(ax), fabs(ay)), fabs(az)));
    if (pot) s[4].s = __dadd_rn(s[4].s, m * pot[i]);
  }
  noalloc_block_merge(s, sh);
  if (threadIdx.x < 10) partials[10 * (int64_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_noalloc_final(int ntiles, const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double sh[10][NOALLOC_NT];
  sfmm::csum s[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int t = threadIdx.x; t < ntiles; t += NOALLOC_NT)
    for (int c = 0; c < 5; ++c) sfmm::cs_merge(s[c], partials[10 * (int64_t)t + c], partials[10 * (int64_t)t + 5 + c]);
  noalloc_block_merge(s, sh);
  if (threadIdx.x < 5) {
    const double v = __dadd_rn(sh[threadIdx.x][0], sh[5 + threadIdx.x][0]);
    out[threadIdx.x] = (threadIdx.x == 4) ? 0.5 * v : v;
  }
}

// The CUDA context current on this thread, through the driver entry point the
// runtime hands out (no link-time dependency on the driver library).
void* current_context() {
  using Fn = int (*)(void**);
  static Fn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Fn>(p);
    else
      cudaGetLastError();
    looked = true;
  }
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

// Device address of the partials array on the current device and context
// (looked up on the first call in a context; later calls reuse it).
int noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= NOALLOC_MAXDEV) return SFMM_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  void* ctx = current_context();
  if (!g_noalloc_addr[dev] || !ctx || ctx != g_noalloc_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      g_noalloc_addr[dev] = nullptr;
      return SFMM_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
    g_noalloc_ctx[dev] = current_context();  // the lookup may have created the primary context
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
