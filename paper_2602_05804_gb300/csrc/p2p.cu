// Near field of the SFMM solver: pairwise M4-softened gravity over each
// leaf's neighbour list (the cached neighbours of Algorithm 2, Sect. 3),
// combined with the far field, written in caller order, plus the momentum
// and energy sums (one partial per leaf, reduced in a fixed order).
//
// One warp per target leaf.  With n_t targets, lane l serves target
// l mod n_t and takes every (32 / n_t)-th source ("phase" l / n_t), so that
// all lanes work for any leaf size; sources are staged per warp in shared
// memory, converted once to coordinates relative to the target leaf's
// centre (FP32 form).
#include <type_traits>

#include "sfmm_internal.cuh"

namespace sfmm {

#define P2P_WARPS 8
#define P2P_NT (P2P_WARPS * 32)
#define P2P_SB 128

struct P2PArgs {
  int nleaves;
  const int* leaf_node;
  const int* nfirst;
  const int* ncount;
  const float4* geo_hi;
  const float4* geo_lo;
  const int* arena;
  const long long* p2p_off;
  const int* p2p_cnt;
  const float4* prel;
  const float* ph32;
  const double* px;
  const double* py;
  const double* pz;
  const double* pm;
  const double* ph;
  const int* perm;
  const float4* far32;
  const double* far64;
  double G;
  int self_pot;
  int* leaf_counter;
  double* acc;
  double* pot;
  double* leafsum;  // nleaves x 5: sum m a (3), sum |m a|, sum m Phi
};

// M4 softening kernel of one particle (compact support 2h): g = phi'(r)/r
// and phi, -> 1/r^3 and -1/r outside 2h.  rinv = 1/r (0 when r = 0).
template <typename R>
__device__ __forceinline__ void m4_kernel(R q, R hinv, R rinv, R& g, R& phi) {
  const R hinv3 = hinv * hinv * hinv;
  const R q2 = q * q;
  const R rinv3 = rinv * rinv * rinv;
  const R g_in = hinv3 * fma(q2, fma(R(0.5), q, R(-1.2)), R(4.0 / 3.0));
  const R p_in = hinv * fma(q2, fma(q2, fma(R(0.1), q, R(-0.3)), R(2.0 / 3.0)), R(-1.4));
  const R g_mid = fma(hinv3, fma(q, fma(q, fma(R(-1.0 / 6.0), q, R(1.2)), R(-3.0)), R(8.0 / 3.0)), R(-1.0 / 15.0) * rinv3);
  const R p_mid = fma(hinv, fma(q2, fma(q, fma(q, fma(R(-1.0 / 30.0), q, R(0.3)), R(-1.0)), R(4.0 / 3.0)), R(-1.6)),
                      R(1.0 / 15.0) * rinv);
  g = (q < R(1)) ? g_in : ((q < R(2)) ? g_mid : rinv3);
  phi = (q < R(1)) ? p_in : ((q < R(2)) ? p_mid : -rinv);
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <bool F32>
__global__ void __launch_bounds__(P2P_NT) k_p2p(const P2PArgs a) {
  using R = typename std::conditional<F32, float, double>::type;
  __shared__ R s_x[P2P_WARPS][P2P_SB], s_y[P2P_WARPS][P2P_SB], s_z[P2P_WARPS][P2P_SB];
  __shared__ R s_m[P2P_WARPS][P2P_SB], s_h2[P2P_WARPS][P2P_SB], s_hi[P2P_WARPS][P2P_SB];
  __shared__ int s_idx[P2P_WARPS][P2P_SB];
  __shared__ R s_red[P2P_WARPS][4][32];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    int leaf = 0;
    if (lane == 0) leaf = atomicAdd(a.leaf_counter, 1);
    leaf = __shfl_sync(SFMM_FULL, leaf, 0);
    if (leaf >= a.nleaves) break;
    const int L = a.leaf_node[leaf];
    const int fL = a.nfirst[L], nL = a.ncount[L];
    const float4 hiL = a.geo_hi[L], loL = a.geo_lo[L];
    // lane -> (target slot, phase)
    const int nph = (nL <= 16) ? (32 / nL) : 1;
    const int ntl = (nL <= 32) ? nL : 32;
    const int ph = lane / ntl;
    const bool lane_on = ph < nph;
    const int t0 = lane % ntl;
    const int t1 = t0 + 32;  // second target slot (leaves of 33..64)
    const bool on0 = lane_on && t0 < nL;
    const bool on1 = lane_on && nL > 32 && t1 < nL;
    R xi0 = R(0), yi0 = R(0), zi0 = R(0), h2i0 = R(0), hinvi0 = R(0);
    R xi1 = R(0), yi1 = R(0), zi1 = R(0), h2i1 = R(0), hinvi1 = R(0);
    auto load_t = [&](int t, R& x, R& y, R& z, R& h2, R& hinv) {
      const int i = fL + t;
      if constexpr (F32) {
        const float4 p = a.prel[i];
        x = p.x;
        y = p.y;
        z = p.z;
        const float h = a.ph32[i];
        h2 = 4.0f * h * h;
        hinv = 1.0f / h;
      } else {
        x = a.px[i];
        y = a.py[i];
        z = a.pz[i];
        const double h = a.ph[i];
        h2 = 4.0 * h * h;
        hinv = 1.0 / h;
      }
    };
    if (on0) load_t(t0, xi0, yi0, zi0, h2i0, hinvi0);
    if (on1) load_t(t1, xi1, yi1, zi1, h2i1, hinvi1);
    R ax0 = R(0), ay0 = R(0), az0 = R(0), pt0 = R(0);
    R ax1 = R(0), ay1 = R(0), az1 = R(0), pt1 = R(0);

    const long long off = a.p2p_off[leaf];
    const int cnt = a.p2p_cnt[leaf];
    int nb = 0;
    int e = 0;
    while (true) {
      // stage whole source leaves while they fit
      while (e < cnt) {
        const int S = a.arena[off + e];
        const int fS = a.nfirst[S], nS = a.ncount[S];
        if (nb + nS > P2P_SB) break;
        R ox = R(0), oy = R(0), oz = R(0);
        if constexpr (F32) {
          const float4 hS = a.geo_hi[S], lS = a.geo_lo[S];
          ox = df_diff(hS.x, lS.x, hiL.x, loL.x);
          oy = df_diff(hS.y, lS.y, hiL.y, loL.y);
          oz = df_diff(hS.z, lS.z, hiL.z, loL.z);
        }
        for (int j = lane; j < nS; j += 32) {
          const int i = fS + j;
          R x, y, z, m, h;
          if constexpr (F32) {
            const float4 p = a.prel[i];
            x = p.x + ox;
            y = p.y + oy;
            z = p.z + oz;
            m = p.w;
            h = a.ph32[i];
          } else {
            x = a.px[i];
            y = a.py[i];
            z = a.pz[i];
            m = a.pm[i];
            h = a.ph[i];
          }
          s_x[warp][nb + j] = x;
          s_y[warp][nb + j] = y;
          s_z[warp][nb + j] = z;
          s_m[warp][nb + j] = m;
          s_h2[warp][nb + j] = R(4) * h * h;
          s_hi[warp][nb + j] = R(1) / h;
          s_idx[warp][nb + j] = i;
        }
        nb += nS;
        ++e;
      }
      if (nb == 0) break;
      __syncwarp();
      const int iters = (nb + nph - 1) / nph;
      for (int it = 0; it < iters; ++it) {
        const int j = it * nph + ph;
        const bool vj = lane_on && j < nb;
        const int jj = vj ? j : 0;
        const R xj = s_x[warp][jj], yj = s_y[warp][jj], zj = s_z[warp][jj];
        const R mj = vj ? s_m[warp][jj] : R(0);
        const R h2j = s_h2[warp][jj], hinvj = s_hi[warp][jj];
        const int idxj = s_idx[warp][jj];
        // target slot 0
        {
          const R dx = xi0 - xj, dy = yi0 - yj, dz = zi0 - zj;
          const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
          const bool self = !on0 || !vj || (idxj == fL + t0);
          const R rinv = (r2 > R(0)) ? rsq(r2) : R(0);
          const bool near = !self && r2 < fmax(h2i0, h2j);
          R g, phi;
          if (__any_sync(SFMM_FULL, near)) {
            const R r = r2 * rinv;
            R gi, pi, gj, pj;
            m4_kernel<R>(r * hinvi0, hinvi0, rinv, gi, pi);
            m4_kernel<R>(r * hinvj, hinvj, rinv, gj, pj);
            g = R(0.5) * (gi + gj);
            phi = R(0.5) * (pi + pj);
          } else {
            g = rinv * rinv * rinv;
            phi = -rinv;
          }
          const R mg = self ? R(0) : mj * g;
          ax0 = fma(-mg, dx, ax0);
          ay0 = fma(-mg, dy, ay0);
          az0 = fma(-mg, dz, az0);
          pt0 = fma(self ? R(0) : mj, phi, pt0);
        }
        if (nL > 32) {
          const R dx = xi1 - xj, dy = yi1 - yj, dz = zi1 - zj;
          const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
          const bool self = !on1 || !vj || (idxj == fL + t1);
          const R rinv = (r2 > R(0)) ? rsq(r2) : R(0);
          const bool near = !self && r2 < fmax(h2i1, h2j);
          R g, phi;
          if (__any_sync(SFMM_FULL, near)) {
            const R r = r2 * rinv;
            R gi, pi, gj, pj;
            m4_kernel<R>(r * hinvi1, hinvi1, rinv, gi, pi);
            m4_kernel<R>(r * hinvj, hinvj, rinv, gj, pj);
            g = R(0.5) * (gi + gj);
            phi = R(0.5) * (pi + pj);
          } else {
            g = rinv * rinv * rinv;
            phi = -rinv;
          }
          const R mg = self ? R(0) : mj * g;
          ax1 = fma(-mg, dx, ax1);
          ay1 = fma(-mg, dy, ay1);
          az1 = fma(-mg, dz, az1);
          pt1 = fma(self ? R(0) : mj, phi, pt1);
        }
      }
      __syncwarp();
      nb = 0;
      if (e >= cnt) break;
    }

    // combine the phases of each target, add the far field, write out
    double sm[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int slot = 0; slot < 2; ++slot) {
      if (slot == 1 && nL <= 32) break;
      s_red[warp][0][lane] = slot ? ax1 : ax0;
      s_red[warp][1][lane] = slot ? ay1 : ay0;
      s_red[warp][2][lane] = slot ? az1 : az0;
      s_red[warp][3][lane] = slot ? pt1 : pt0;
      __syncwarp();
      const int t = lane + 32 * slot;
      if (lane < ntl && t < nL) {
        R v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          R s = R(0);
          for (int q = 0; q < nph; ++q) s += s_red[warp][c][q * ntl + lane];
          v[c] = s;
        }
        const int i = fL + t;
        double f[4];
        if constexpr (F32) {
          const float4 fr = a.far32[i];
          f[0] = (double)(v[0] + fr.x);
          f[1] = (double)(v[1] + fr.y);
          f[2] = (double)(v[2] + fr.z);
          f[3] = (double)(v[3] + fr.w);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) f[c] = v[c] + a.far64[4 * (size_t)i + c];
        }
        const double m = a.pm[i];
        double pot = a.G * f[3];
        if (a.self_pot) pot += a.G * m * (-1.4 / a.ph[i]);
        const int o = a.perm[i];
        double am[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double acc = a.G * f[c];
          a.acc[3 * (size_t)o + c] = acc;
          am[c] = m * acc;
        }
        if (a.pot) a.pot[o] = pot;
        sm[0] += am[0];
        sm[1] += am[1];
        sm[2] += am[2];
        sm[3] += fabs(am[0]) + fabs(am[1]) + fabs(am[2]);
        sm[4] += m * pot;
      }
      __syncwarp();
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double s = sm[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(SFMM_FULL, s, o);
      sm[c] = s;
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) a.leafsum[5 * (size_t)leaf + c] = sm[c];
    }
  }
}

// Fixed-order reduction of the per-leaf sums: one block, Neumaier
// compensated partial sums per thread, then a tree over threads.
__global__ void k_reduce_leafsum(int nleaves, const double* __restrict__ leafsum, double* __restrict__ out) {
  __shared__ double sh[5][256];
  double s[5] = {0, 0, 0, 0, 0}, cmp[5] = {0, 0, 0, 0, 0};
  for (int q = threadIdx.x; q < nleaves; q += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const double v = leafsum[5 * (size_t)q + c];
      const double t = s[c] + v;
      cmp[c] += (fabs(s[c]) >= fabs(v)) ? (s[c] - t) + v : (v - t) + s[c];
      s[c] = t;
    }
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = s[c] + cmp[c];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

int run_p2p(sfmm_ctx* c, double* acc, double* pot) {
  const int nl = c->nleaves;
  int rc;
  if ((rc = c->red_part.ensure(sizeof(double) * 5 * (size_t)nl + 64))) return rc;
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  SFMM_CUDA_TRY(cudaMemsetAsync(ctr + 10, 0, sizeof(unsigned long long), c->stream));
  P2PArgs a{};
  a.nleaves = nl;
  a.leaf_node = c->leaf_node.as<int>();
  a.nfirst = c->nfirst.as<int>();
  a.ncount = c->ncount.as<int>();
  a.geo_hi = c->geo_hi.as<float4>();
  a.geo_lo = c->geo_lo.as<float4>();
  a.arena = c->arena.as<int>();
  a.p2p_off = c->p2p_off.as<long long>();
  a.p2p_cnt = c->p2p_cnt.as<int>();
  a.prel = c->prel.as<float4>();
  a.ph32 = c->ph32.as<float>();
  a.px = c->px.as<double>();
  a.py = c->py.as<double>();
  a.pz = c->pz.as<double>();
  a.pm = c->pm.as<double>();
  a.ph = c->ph.as<double>();
  a.perm = c->perm.as<int>();
  a.far32 = c->far.as<float4>();
  a.far64 = c->far.as<double>();
  a.G = c->G;
  a.self_pot = c->self_potential;
  a.leaf_counter = reinterpret_cast<int*>(ctr + 10);
  a.acc = acc;
  a.pot = pot;
  a.leafsum = c->red_part.as<double>();
  const bool f32 = (c->precision == SFMM_FP32);
  int per_sm = 0;
  if (f32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<true>, P2P_NT, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<false>, P2P_NT, 0);
  if (per_sm < 1) per_sm = 1;
  const int nblocks = per_sm * num_sms(c->device);
  if (f32) k_p2p<true><<<nblocks, P2P_NT, 0, c->stream>>>(a);
  else k_p2p<false><<<nblocks, P2P_NT, 0, c->stream>>>(a);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

int run_reduce(sfmm_ctx* c, const double*, const double*) {
  double* out = c->red_part.as<double>() + 5 * (size_t)c->nleaves;
  k_reduce_leafsum<<<1, 256, 0, c->stream>>>(c->nleaves, c->red_part.as<double>(), out);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

}  // namespace sfmm
