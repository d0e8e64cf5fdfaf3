// Momentum and energy sums of a gravity call, over the particles and per
// system (the solver's diagnostics: total momentum, which Newton's third law
// and the symmetric expansions keep at rounding level, and the potential
// energy W = 1/2 sum m Phi).
#include "sfmm_internal.cuh"

namespace sfmm {

// Momentum and energy sums over the particles: sum m a (3), sum |m a| (over
// components), sum m Phi, in FP64 in a fixed order (reruns are bitwise
// identical); the momentum components, whose terms cancel to ~1e-18 of
// sum |m a|, as Neumaier-compensated sums.  Every block takes a contiguous range of
// sorted positions (thread t: positions lo + t, lo + t + RED_NT, ...), merges
// its threads' sums in a fixed tree and writes one partial (s and c: 10
// doubles); one warp per sum merges the partials.  Accelerations and potentials are
// read in caller order through the permutation.  A separate pass costs fewer
// FP64 instructions per particle than sums formed in the near-field kernel,
// whose warps hold a leaf of ~11 particles.
#define RED_NT 256
#define RED_BLOCKS 304

__device__ __forceinline__ void block_merge(csum (&s)[5], double (&sh)[10][RED_NT]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    sh[c][threadIdx.x] = s[c].s;
    sh[5 + c][threadIdx.x] = s[c].c;
  }
  __syncthreads();
  for (int w = RED_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) {
        csum a{sh[c][threadIdx.x], sh[5 + c][threadIdx.x]};
        cs_merge(a, sh[c][threadIdx.x + w], sh[5 + c][threadIdx.x + w]);
        sh[c][threadIdx.x] = a.s;
        sh[5 + c][threadIdx.x] = a.c;
      }
    __syncthreads();
  }
}

// Compensated sums of sorted positions [lo, hi) into s (this thread's share).
__device__ __forceinline__ void particle_sums(int64_t lo, int64_t hi, const double* __restrict__ pm,
                                              const int* __restrict__ perm, const double* __restrict__ acc,
                                              const double* __restrict__ pot, csum (&s)[5]) {
  for (int64_t i = lo + threadIdx.x; i < hi; i += RED_NT) {
    const double m = pm[i];
    const int o = perm[i];
    const double ax = m * acc[3 * (size_t)o], ay = m * acc[3 * (size_t)o + 1], az = m * acc[3 * (size_t)o + 2];
    cs_add(s[0], ax);
    cs_add(s[1], ay);
    cs_add(s[2], az);
    // sums of same-sign terms cannot cancel: plain additions are accurate to
    // a few eps of the result there, and cost a seventh of a compensated one
    s[3].s = __dadd_rn(s[3].s, __dadd_rn(__dadd_rn(fabs(ax), fabs(ay)), fabs(az)));
    s[4].s = __dadd_rn(s[4].s, m * pot[o]);
  }
}

__global__ void __launch_bounds__(RED_NT) k_reduce_particles(int64_t n, const double* __restrict__ pm,
                                                             const int* __restrict__ perm,
                                                             const double* __restrict__ acc,
                                                             const double* __restrict__ pot,
                                                             double* __restrict__ part) {
  __shared__ double sh[10][RED_NT];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = min(n, lo + per);
  csum s[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
  particle_sums(lo, hi, pm, perm, acc, pot, s);
  block_merge(s, sh);
  if (threadIdx.x < 10) part[10 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// One warp per sum (block c: sum c), on five SMs: lane l merges partials l,
// l + 32, ... in order, then the lanes merge in a fixed tree.
__global__ void k_reduce_final(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  const int c = blockIdx.x, lane = threadIdx.x;
  csum s{0.0, 0.0};
  for (int q = lane; q < nparts; q += 32) cs_merge(s, part[10 * q + c], part[10 * q + 5 + c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double bs = __shfl_down_sync(SFMM_FULL, s.s, o), bc = __shfl_down_sync(SFMM_FULL, s.c, o);
    if (lane < o) cs_merge(s, bs, bc);
  }
  if (lane == 0) out[c] = __dadd_rn(s.s, s.c);
}

// Per-system sums of a batch: one block per system over its range of sorted
// positions (systems are contiguous in the sorted order).
__global__ void __launch_bounds__(RED_NT) k_reduce_sys(const int* __restrict__ sys_off, const double* __restrict__ pm,
                                                       const int* __restrict__ perm, const double* __restrict__ acc,
                                                       const double* __restrict__ pot, double* __restrict__ out) {
  __shared__ double sh[10][RED_NT];
  const int sys = blockIdx.x;
  csum s[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
  particle_sums(sys_off[sys], sys_off[sys + 1], pm, perm, acc, pot, s);
  block_merge(s, sh);
  if (threadIdx.x < 5) {
    const double v = __dadd_rn(sh[threadIdx.x][0], sh[5 + threadIdx.x][0]);
    out[5 * (size_t)sys + threadIdx.x] = (threadIdx.x == 4) ? 0.5 * v : v;
  }
}

int run_reduce_systems(sfmm_ctx* c) {
  int rc;
  if ((rc = c->sys_sums.ensure(sizeof(double) * 5 * (size_t)c->nsys))) return rc;
  k_reduce_sys<<<c->nsys, RED_NT, 0, c->stream>>>(c->sys_off.as<int>(), c->pm.as<double>(), c->perm.as<int>(),
                                                 c->red_acc, c->red_pot, c->sys_sums.as<double>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

int run_reduce(sfmm_ctx* c, double** out_dev) {
  int rc;
  if ((rc = c->red_part.ensure(sizeof(double) * 10 * ((size_t)RED_BLOCKS + 1)))) return rc;
  double* part = c->red_part.as<double>();
  double* out = part + 10 * RED_BLOCKS;
  k_reduce_particles<<<RED_BLOCKS, RED_NT, 0, c->stream>>>(c->n, c->pm.as<double>(), c->perm.as<int>(), c->red_acc,
                                                          c->red_pot, part);
  ++c->nlaunch;
  k_reduce_final<<<5, 32, 0, c->stream>>>(RED_BLOCKS, part, out);
  ++c->nlaunch;
  *out_dev = out;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

}  // namespace sfmm
