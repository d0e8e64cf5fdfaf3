// Gravity-only leapfrog with the SFMM forces (the gravity part of the
// binary-polytrope test of Sect. 4).  Kick-drift-kick steps; the tree is
// rebuilt at every new position set.  Linear momentum is conserved to
// rounding because the SFMM pair forces are antisymmetric; the records of
// sum m v and sum m x cross v show it.
#include <cmath>

#include "sfmm_internal.cuh"

namespace sfmm {

namespace {

constexpr int LF_NT = 256;
constexpr int LF_TILE = 4096;  // particles per momentum partial
constexpr int LF_NSUM = 7;     // P (3), L (3), sum |m v_d|

// v += a hdt (each operation rounded as written: no fused multiply-add)
__global__ void k_kick(int64_t n, double* __restrict__ vel, const double* __restrict__ acc, double hdt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 3 * n) return;
  vel[k] = dadd(vel[k], dmul(acc[k], hdt));
}

// v += a hdt, then x += v dt
__global__ void k_kick_drift(int64_t n, double* __restrict__ pos, double* __restrict__ vel,
                             const double* __restrict__ acc, double hdt, double dt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 3 * n) return;
  const double v = dadd(vel[k], dmul(acc[k], hdt));
  vel[k] = v;
  pos[k] = dadd(pos[k], dmul(v, dt));
}

// Compensated (Neumaier) merge of one partial per thread: sh holds s then c.
__device__ __forceinline__ void block_sum7(csum (&s)[LF_NSUM], double (*sh)[LF_NT]) {
#pragma unroll
  for (int c = 0; c < LF_NSUM; ++c) {
    sh[c][threadIdx.x] = s[c].s;
    sh[LF_NSUM + c][threadIdx.x] = s[c].c;
  }
  __syncthreads();
  for (int w = LF_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < LF_NSUM; ++c) {
        csum a{sh[c][threadIdx.x], sh[LF_NSUM + c][threadIdx.x]};
        cs_merge(a, sh[c][threadIdx.x + w], sh[LF_NSUM + c][threadIdx.x + w]);
        sh[c][threadIdx.x] = a.s;
        sh[LF_NSUM + c][threadIdx.x] = a.c;
      }
    __syncthreads();
  }
}

// Per-tile compensated partial sums of m v, m x cross v and |m v_d| (fixed
// order): 2 x LF_NSUM doubles per tile (sums, then their error terms).
__global__ void k_momentum_tiles(int64_t n, const double* __restrict__ pos, const double* __restrict__ vel,
                                 const double* __restrict__ mass, double* __restrict__ part) {
  __shared__ double sh[2 * LF_NSUM][LF_NT];
  csum s[LF_NSUM] = {};
  const int64_t base = (int64_t)blockIdx.x * LF_TILE;
  for (int k = threadIdx.x; k < LF_TILE; k += LF_NT) {
    const int64_t i = base + k;
    if (i >= n) break;
    const double m = mass[i];
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    const double px = m * vel[3 * i], py = m * vel[3 * i + 1], pz = m * vel[3 * i + 2];
    cs_add(s[0], px);
    cs_add(s[1], py);
    cs_add(s[2], pz);
    cs_add(s[3], y * pz - z * py);
    cs_add(s[4], z * px - x * pz);
    cs_add(s[5], x * py - y * px);
    cs_add(s[6], fabs(px));
    cs_add(s[6], fabs(py));
    cs_add(s[6], fabs(pz));
  }
  block_sum7(s, sh);
  if (threadIdx.x < 2 * LF_NSUM) part[(int64_t)2 * LF_NSUM * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_momentum_final(int ntiles, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[2 * LF_NSUM][LF_NT];
  csum s[LF_NSUM] = {};
  for (int t = threadIdx.x; t < ntiles; t += LF_NT)
    for (int c = 0; c < LF_NSUM; ++c)
      cs_merge(s[c], part[(int64_t)2 * LF_NSUM * t + c], part[(int64_t)2 * LF_NSUM * t + LF_NSUM + c]);
  block_sum7(s, sh);
  if (threadIdx.x < LF_NSUM) out[threadIdx.x] = cs_value(csum{sh[threadIdx.x][0], sh[LF_NSUM + threadIdx.x][0]});
}

int blocks3(int64_t n) { return (int)((3 * n + LF_NT - 1) / LF_NT); }

// Makes the context's device current for the call and restores the caller's.
struct LfDevice {
  int prev = -1;
  explicit LfDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~LfDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// One record (t, P, L, sum |m v_d|) to the host.
int record_state(sfmm_ctx* c, int64_t n, const double* pos, const double* vel, const double* mass, double t,
                 double* rec) {
  const int ntiles = (int)((n + LF_TILE - 1) / LF_TILE);
  double* part = c->lf_part.as<double>();
  double* out = part + (size_t)2 * LF_NSUM * ntiles;
  k_momentum_tiles<<<ntiles, LF_NT, 0, c->stream>>>(n, pos, vel, mass, part);
  k_momentum_final<<<1, LF_NT, 0, c->stream>>>(ntiles, part, out);
  c->nlaunch += 2;
  SFMM_CUDA_TRY(cudaGetLastError());
  SFMM_CUDA_TRY(cudaMemcpyAsync(c->h_scalars + 32, out, sizeof(double) * LF_NSUM, cudaMemcpyDeviceToHost, c->stream));
  SFMM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  rec[0] = t;
  for (int k = 0; k < LF_NSUM; ++k) rec[1 + k] = c->h_scalars[32 + k];
  return SFMM_OK;
}

}  // namespace

}  // namespace sfmm

using namespace sfmm;

extern "C" int sfmm_leapfrog(sfmm_ctx* c, int64_t n, double* pos, double* vel, const double* mass, const double* h,
                             int leaf_size, double theta, int order, double dt, int64_t nsteps, int64_t record_every,
                             double* record, double* acc) {
  if (!c) return SFMM_EINVAL;
  if (!pos || !vel || !mass || !h) return set_error(c, SFMM_EINVAL, "NULL pointer");
  if (n < 1 || n > ((int64_t)1 << 31) - 2) return set_error(c, SFMM_EINVAL, "n must be in [1, 2^31 - 2]");
  if (!std::isfinite(dt)) return set_error(c, SFMM_EINVAL, "dt must be finite");
  if (nsteps < 0 || record_every < 1) return set_error(c, SFMM_EINVAL, "nsteps >= 0 and record_every >= 1");
  LfDevice g(c->device);
  int rc;
  const int ntiles = (int)((n + LF_TILE - 1) / LF_TILE);
  if ((rc = c->lf_acc.ensure(sizeof(double) * 3 * (size_t)n)) ||
      (rc = c->lf_part.ensure(sizeof(double) * 2 * LF_NSUM * ((size_t)ntiles + 1))))
    return set_error(c, rc, "leapfrog allocation failed");
  double* a = c->lf_acc.as<double>();
  if ((rc = sfmm_build(c, n, pos, mass, h, leaf_size))) return rc;
  if ((rc = sfmm_gravity(c, theta, order, a, nullptr))) return rc;
  int64_t irec = 0;
  if (record && (rc = record_state(c, n, pos, vel, mass, 0.0, record + 8 * irec++))) return set_error(c, rc, "record");
  for (int64_t s = 1; s <= nsteps; ++s) {
    k_kick_drift<<<blocks3(n), LF_NT, 0, c->stream>>>(n, pos, vel, a, 0.5 * dt, dt);
    ++c->nlaunch;
    SFMM_CUDA_TRY(cudaGetLastError());
    if ((rc = sfmm_build(c, n, pos, mass, h, leaf_size))) return rc;
    if ((rc = sfmm_gravity(c, theta, order, a, nullptr))) return rc;
    k_kick<<<blocks3(n), LF_NT, 0, c->stream>>>(n, vel, a, 0.5 * dt);
    ++c->nlaunch;
    SFMM_CUDA_TRY(cudaGetLastError());
    if (record && s % record_every == 0 &&
        (rc = record_state(c, n, pos, vel, mass, (double)s * dt, record + 8 * irec++)))
      return set_error(c, rc, "record");
  }
  if (acc) SFMM_CUDA_TRY(cudaMemcpyAsync(acc, a, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, c->stream));
  SFMM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return SFMM_OK;
}
