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
#define P2P_SB 64

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
  const double* ncx;
  const double* ncy;
  const double* ncz;
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

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4; };

// Far pair (no softening): a -= m r^-3 d, phi -= m / r.
template <typename R>
__device__ __forceinline__ void pair_far(R xi, R yi, R zi, const typename Vec4<R>::T& s, R& ax, R& ay, R& az,
                                         R& pt) {
  const R dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
  const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const R ri = rsq(r2);
  const R mr = s.w * ri;
  const R mr3 = mr * (ri * ri);
  ax = fma(-mr3, dx, ax);
  ay = fma(-mr3, dy, ay);
  az = fma(-mr3, dz, az);
  pt -= mr;
}

// Softened pair (both particles' kernels, mean): returns the factor g-bar
// multiplying -m d and the potential factor phi-bar multiplying m.
template <typename R>
__device__ __forceinline__ void pair_soft(R r2, R hinvi, R hinvj, R& gbar, R& pbar) {
  const R ri = (r2 > R(0)) ? rsq(r2) : R(0);
  const R r = r2 * ri;
  R gi, pi, gj, pj;
  m4_kernel<R>(r * hinvi, hinvi, ri, gi, pi);
  m4_kernel<R>(r * hinvj, hinvj, ri, gj, pj);
  gbar = R(0.5) * (gi + gj);
  pbar = R(0.5) * (pi + pj);
}

// Sources are staged per warp, split once per source into those that may lie
// inside the kernel of some target of the leaf (|x_j - s_L| < l_L +
// 2 max(h_max,L, h_j), with a small safety factor) and those that cannot; the
// latter take the unsoftened branch-free loop.
template <bool F32> __host__ __device__ constexpr int p2p_warps() { return F32 ? P2P_WARPS : P2P_WARPS / 2; }

template <bool F32>
__global__ void __launch_bounds__(P2P_NT) k_p2p(const P2PArgs a) {
  using R = typename std::conditional<F32, float, double>::type;
  using V = typename Vec4<R>::T;
  constexpr int NW = p2p_warps<F32>();           // warps per block (48 KB static limit)
  constexpr int SB = P2P_SB;                     // staged sources per warp (>= 64, a full leaf)
  __shared__ V s_far[NW][SB];
  __shared__ V s_near[NW][SB];
  __shared__ R s_nhinv[NW][SB];
  __shared__ R s_nh2[NW][SB];                   // (2h)^2 of the candidate
  __shared__ int s_nidx[NW][SB];
  __shared__ R s_red[NW][4][32];
  __shared__ V s_tgt[NW][64];            // targets: x, y, z, 1/h
  __shared__ R s_acc[NW][64][4];                // softened part per target
  __shared__ int s_q[NW][64];            // queued pairs: target << 16 | candidate

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  while (true) {
    int leaf = 0;
    if (lane == 0) leaf = atomicAdd(a.leaf_counter, 1);
    leaf = __shfl_sync(SFMM_FULL, leaf, 0);
    if (leaf >= a.nleaves) break;
    const int L = a.leaf_node[leaf];
    const int fL = a.nfirst[L], nL = a.ncount[L];
    const float4 hiL = a.geo_hi[L], loL = a.geo_lo[L];
    // target leaf radius and largest smoothing length, with a safety factor
    // covering the float32 rounding of the relative coordinates
    const R lL = (R)hiL.w * R(1.0001), hL = (R)loL.w * R(1.0001);
    const double cLx = F32 ? 0.0 : a.ncx[L], cLy = F32 ? 0.0 : a.ncy[L], cLz = F32 ? 0.0 : a.ncz[L];
    // lane -> (target slot, phase)
    const int nph = (nL <= 16) ? (32 / nL) : 1;
    const int ntl = (nL <= 32) ? nL : 32;
    const int ph = lane / ntl;
    const bool lane_on = ph < nph;
    const int t0 = lane % ntl;
    const int t1 = t0 + 32;
    const bool on0 = lane_on && t0 < nL;
    const bool on1 = lane_on && nL > 32 && t1 < nL;
    R xi0 = R(0), yi0 = R(0), zi0 = R(0), hinvi0 = R(0);
    R xi1 = R(0), yi1 = R(0), zi1 = R(0), hinvi1 = R(0);
    if (on0) {
      const int i = fL + t0;
      if constexpr (F32) {
        const float4 p = a.prel[i];
        xi0 = p.x; yi0 = p.y; zi0 = p.z;
        hinvi0 = 1.0f / a.ph32[i];
      } else {
        xi0 = a.px[i]; yi0 = a.py[i]; zi0 = a.pz[i];
        hinvi0 = 1.0 / a.ph[i];
      }
    }
    if (on1) {
      const int i = fL + t1;
      if constexpr (F32) {
        const float4 p = a.prel[i];
        xi1 = p.x; yi1 = p.y; zi1 = p.z;
        hinvi1 = 1.0f / a.ph32[i];
      } else {
        xi1 = a.px[i]; yi1 = a.py[i]; zi1 = a.pz[i];
        hinvi1 = 1.0 / a.ph[i];
      }
    }
    // target table for the queued softened pairs
    for (int t = lane; t < nL; t += 32) {
      const int i = fL + t;
      if constexpr (F32) {
        const float4 p = a.prel[i];
        s_tgt[warp][t] = make_float4(p.x, p.y, p.z, 1.0f / a.ph32[i]);
      } else {
        s_tgt[warp][t] = make_double4(a.px[i], a.py[i], a.pz[i], 1.0 / a.ph[i]);
      }
      s_acc[warp][t][0] = s_acc[warp][t][1] = s_acc[warp][t][2] = s_acc[warp][t][3] = R(0);
    }
    __syncwarp();
    const R h2i0 = (hinvi0 > R(0)) ? R(4) / (hinvi0 * hinvi0) : R(0);
    const R h2i1 = (hinvi1 > R(0)) ? R(4) / (hinvi1 * hinvi1) : R(0);
    int nqp = 0;  // queued softened pairs
    // unsoftened accumulators per slot
    R ax0 = R(0), ay0 = R(0), az0 = R(0), pt0 = R(0);
    R ax1 = R(0), ay1 = R(0), az1 = R(0), pt1 = R(0);

    const long long off = a.p2p_off[leaf];
    const int cnt = a.p2p_cnt[leaf];
    int nfar = 0, nnear = 0, e = 0;
    while (true) {
      // stage whole source leaves while both buffers have room
      while (e < cnt) {
        const int S = a.arena[off + e];
        const int fS = a.nfirst[S], nS = a.ncount[S];
        if (nfar + nS > SB || nnear + nS > SB) break;
        R ox = R(0), oy = R(0), oz = R(0);
        if constexpr (F32) {
          const float4 hS = a.geo_hi[S], lS = a.geo_lo[S];
          ox = df_diff(hS.x, lS.x, hiL.x, loL.x);
          oy = df_diff(hS.y, lS.y, hiL.y, loL.y);
          oz = df_diff(hS.z, lS.z, hiL.z, loL.z);
        }
        for (int j0 = 0; j0 < nS; j0 += 32) {
          const int j = j0 + lane;
          const bool valid = j < nS;
          V v = {R(0), R(0), R(0), R(0)};
          R h = R(1);
          if (valid) {
            const int i = fS + j;
            if constexpr (F32) {
              const float4 p = a.prel[i];
              v = make_float4(p.x + ox, p.y + oy, p.z + oz, p.w);
              h = a.ph32[i];
            } else {
              v = make_double4(a.px[i], a.py[i], a.pz[i], a.pm[i]);
              h = a.ph[i];
            }
          }
          // distance to the target leaf's centre
          R rx = v.x, ry = v.y, rz = v.z;
          if constexpr (!F32) {
            rx -= cLx;
            ry -= cLy;
            rz -= cLz;
          }
          const R reach = lL + R(2) * fmax(hL, h * R(1.0001));
          const bool near = valid && (fma(rx, rx, fma(ry, ry, rz * rz)) < reach * reach);
          const unsigned bn = __ballot_sync(SFMM_FULL, near), bf = __ballot_sync(SFMM_FULL, valid && !near);
          if (near) {
            const int q = nnear + __popc(bn & lt);
            s_near[warp][q] = v;
            s_nhinv[warp][q] = R(1) / h;
            s_nh2[warp][q] = R(4) * h * h;
            s_nidx[warp][q] = fS + j;
          } else if (valid) {
            s_far[warp][nfar + __popc(bf & lt)] = v;
          }
          nnear += __popc(bn);
          nfar += __popc(bf);
        }
        ++e;
      }
      if (nfar == 0 && nnear == 0) break;
      __syncwarp();
      // unsoftened sources
      if (lane_on) {
        int j = ph;
        for (; j + nph < nfar; j += 2 * nph) {
          const V s0 = s_far[warp][j], s1 = s_far[warp][j + nph];
          pair_far<R>(xi0, yi0, zi0, s0, ax0, ay0, az0, pt0);
          pair_far<R>(xi0, yi0, zi0, s1, ax0, ay0, az0, pt0);
          if (nL > 32) {
            pair_far<R>(xi1, yi1, zi1, s0, ax1, ay1, az1, pt1);
            pair_far<R>(xi1, yi1, zi1, s1, ax1, ay1, az1, pt1);
          }
        }
        if (j < nfar) {
          const V s0 = s_far[warp][j];
          pair_far<R>(xi0, yi0, zi0, s0, ax0, ay0, az0, pt0);
          if (nL > 32) pair_far<R>(xi1, yi1, zi1, s0, ax1, ay1, az1, pt1);
        }
      }
      // one full batch of queued softened pairs, one per lane (queue <= 63)
      auto drain32 = [&]() {
        __syncwarp();
        // one full batch: each lane one queued softened pair
        const int qv = s_q[warp][nqp - 32 + lane];
        __syncwarp();
        const int tq = qv >> 16, jq = qv & 0xffff;
        const V T = s_tgt[warp][tq];
        const V S = s_near[warp][jq];
        const R ddx = T.x - S.x, ddy = T.y - S.y, ddz = T.z - S.z;
        R gb, pb;
        pair_soft<R>(fma(ddx, ddx, fma(ddy, ddy, ddz * ddz)), T.w, s_nhinv[warp][jq], gb, pb);
        const R mg = S.w * gb;
        atomicAdd(&s_acc[warp][tq][0], -mg * ddx);
        atomicAdd(&s_acc[warp][tq][1], -mg * ddy);
        atomicAdd(&s_acc[warp][tq][2], -mg * ddz);
        atomicAdd(&s_acc[warp][tq][3], S.w * pb);
        nqp -= 32;
      };
      // candidates: exact per-pair kernel test; pairs outside both kernels take
      // the unsoftened formula, pairs inside one are queued (self pairs drop out)
      {
        const int iters = (nnear + nph - 1) / nph;
        for (int it = 0; it < iters; ++it) {
          const int jn = it * nph + ph;
          const bool vj = lane_on && jn < nnear;
          const int jj = vj ? jn : 0;
          const V s0 = s_near[warp][jj];
          const R h2j = s_nh2[warp][jj];
          const int ij = s_nidx[warp][jj];
          bool soft;
          {
            const R dx = xi0 - s0.x, dy = yi0 - s0.y, dz = zi0 - s0.z;
            const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const bool live = vj && on0 && (ij != fL + t0);
            soft = live && r2 < fmax(h2i0, h2j);
            if (live && !soft) {
              const R ri = rsq(r2);
              const R mr = s0.w * ri;
              const R mr3 = mr * (ri * ri);
              ax0 = fma(-mr3, dx, ax0);
              ay0 = fma(-mr3, dy, ay0);
              az0 = fma(-mr3, dz, az0);
              pt0 -= mr;
            }
          }
          const unsigned bq = __ballot_sync(SFMM_FULL, soft);
          if (soft) s_q[warp][nqp + __popc(bq & lt)] = (t0 << 16) | jj;
          nqp += __popc(bq);
          if (nqp >= 32) drain32();
          if (nL > 32) {  // second target slot (leaves of 33..64 particles)
            const R dx = xi1 - s0.x, dy = yi1 - s0.y, dz = zi1 - s0.z;
            const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const bool live = vj && on1 && (ij != fL + t1);
            const bool soft1 = live && r2 < fmax(h2i1, h2j);
            if (live && !soft1) {
              const R ri = rsq(r2);
              const R mr = s0.w * ri;
              const R mr3 = mr * (ri * ri);
              ax1 = fma(-mr3, dx, ax1);
              ay1 = fma(-mr3, dy, ay1);
              az1 = fma(-mr3, dz, az1);
              pt1 -= mr;
            }
            const unsigned b1 = __ballot_sync(SFMM_FULL, soft1);
            if (soft1) s_q[warp][nqp + __popc(b1 & lt)] = (t1 << 16) | jj;
            nqp += __popc(b1);
            if (nqp >= 32) drain32();
          }
        }
      }
      __syncwarp();
      // drain the queue before the staged candidates are overwritten
      if (nqp > 0) {
        const int qv = (lane < nqp) ? s_q[warp][lane] : 0;
        __syncwarp();
        if (lane < nqp) {
          const int tq = qv >> 16, jq = qv & 0xffff;
          const V T = s_tgt[warp][tq];
          const V S = s_near[warp][jq];
          const R ddx = T.x - S.x, ddy = T.y - S.y, ddz = T.z - S.z;
          R gb, pb;
          pair_soft<R>(fma(ddx, ddx, fma(ddy, ddy, ddz * ddz)), T.w, s_nhinv[warp][jq], gb, pb);
          const R mg = S.w * gb;
          atomicAdd(&s_acc[warp][tq][0], -mg * ddx);
          atomicAdd(&s_acc[warp][tq][1], -mg * ddy);
          atomicAdd(&s_acc[warp][tq][2], -mg * ddz);
          atomicAdd(&s_acc[warp][tq][3], S.w * pb);
        }
        nqp = 0;
      }
      __syncwarp();
      nfar = 0;
      nnear = 0;
      if (e >= cnt) break;
    }
    if (!on0) { ax0 = ay0 = az0 = pt0 = R(0); }
    if (!on1) { ax1 = ay1 = az1 = pt1 = R(0); }

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
          R sacc = s_acc[warp][t][c];
          for (int q = 0; q < nph; ++q) sacc += s_red[warp][c][q * ntl + lane];
          v[c] = sacc;
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
      double sv = sm[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(SFMM_FULL, sv, o);
      sm[c] = sv;
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) a.leafsum[5 * (size_t)leaf + c] = sm[c];
    }
  }
}

// Fixed-order reduction of the per-leaf sums: every block sums a contiguous
// range of leaves (tree over threads), then one block sums the block
// partials; the order never changes, so reruns are bitwise identical.
#define RED_NT 256
#define RED_BLOCKS 152

__global__ void k_reduce_leafsum(int nleaves, const double* __restrict__ leafsum, double* __restrict__ part) {
  __shared__ double sh[5][RED_NT];
  const int per = (nleaves + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(nleaves, lo + per);
  double s[5] = {0, 0, 0, 0, 0};
  for (int q = lo + threadIdx.x; q < hi; q += RED_NT)
#pragma unroll
    for (int c = 0; c < 5; ++c) s[c] += leafsum[5 * (size_t)q + c];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = RED_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) part[5 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_reduce_final(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[5][RED_NT];
  double s[5] = {0, 0, 0, 0, 0};
  for (int q = threadIdx.x; q < nparts; q += RED_NT)
#pragma unroll
    for (int c = 0; c < 5; ++c) s[c] += part[5 * q + c];
#pragma unroll
  for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = RED_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 5; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

int run_p2p(sfmm_ctx* c, double* acc, double* pot) {
  const int nl = c->nleaves;
  int rc;
  if ((rc = c->red_part.ensure(sizeof(double) * 5 * ((size_t)nl + RED_BLOCKS + 1)))) return rc;
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
  a.ncx = c->ncx.as<double>();
  a.ncy = c->ncy.as<double>();
  a.ncz = c->ncz.as<double>();
  a.G = c->G;
  a.self_pot = c->self_potential;
  a.leaf_counter = reinterpret_cast<int*>(ctr + 10);
  a.acc = acc;
  a.pot = pot;
  a.leafsum = c->red_part.as<double>();
  const bool f32 = (c->precision == SFMM_FP32);
  const int nt = 32 * (f32 ? p2p_warps<true>() : p2p_warps<false>());
  int per_sm = 0;
  if (f32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<true>, nt, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<false>, nt, 0);
  if (per_sm < 1) per_sm = 1;
  const int nblocks = per_sm * num_sms(c->device);
  if (f32) k_p2p<true><<<nblocks, nt, 0, c->stream>>>(a);
  else k_p2p<false><<<nblocks, nt, 0, c->stream>>>(a);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

int run_reduce(sfmm_ctx* c, double** out_dev) {
  double* part = c->red_part.as<double>() + 5 * (size_t)c->nleaves;
  double* out = part + 5 * RED_BLOCKS;
  k_reduce_leafsum<<<RED_BLOCKS, RED_NT, 0, c->stream>>>(c->nleaves, c->red_part.as<double>(), part);
  ++c->nlaunch;
  k_reduce_final<<<1, RED_NT, 0, c->stream>>>(RED_BLOCKS, part, out);
  ++c->nlaunch;
  *out_dev = out;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

}  // namespace sfmm
