// Near field of the SFMM solver: pairwise M4-softened gravity over each
// leaf's neighbour list (the cached neighbours of Algorithm 2, Sect. 3),
// combined with the far field, written in caller order (the momentum and
// energy sums over the results are formed in reduce.cu).
//
// One warp per target leaf.  With n_t targets, lane l serves target
// l mod n_t and takes every (32 / n_t)-th source ("phase" l / n_t), so that
// all lanes work for any leaf size; sources are staged per warp in shared
// memory, converted once to coordinates relative to the target leaf's
// centre (FP32 form).
#include <algorithm>
#include <type_traits>

#include "sfmm_internal.cuh"

namespace sfmm {

#define P2P_WARPS 8
#define P2P_NT (P2P_WARPS * 32)
#define P2P_SB 128

struct P2PArgs {
  const uint32_t* counts;  // the build's node and leaf counts (device)
  const int* leaf_node;
  const int* nfirst;
  const int* ncount;
  const float4* geo_hi;
  const float4* geo_lo;
  const int* arena;
  const long long* p2p_off;
  const int* p2p_cnt;
  const float4* prel;
  const float4* phh;  // {1/h, (2h)^2, 2h rounded up, 0}
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
  // long lists: work items [0, nextra) are the further chunks (leaf, chunk)
  // of split lists, items [nextra, nextra + nleaves) the first chunk of every
  // leaf; a split leaf's chunk k writes its sums to partial slot split[leaf] + k.
  // The counts come from the split pass on the device: d_split[0] extra
  // items, [1] partial slots, [2] split leaves
  const unsigned long long* d_split;
  const int2* extra;
  const int* split;   // per leaf: first partial slot, -1 (or NULL array) if unsplit
  const int* slist;   // the split leaves
  void* part;         // [slot][lmax][4] partial sums in the form's type
  int lmax;
  int chunk;          // neighbour-list entries per work item of a split list
  unsigned long long* pair_counter;  // pair evaluations (statistics)
};

// M4 softening kernel of one particle (compact support 2h): g = phi'(r)/r
// and phi, -> 1/r^3 and -1/r outside 2h.  Both pieces' polynomials are
// evaluated in full and the piece chosen afterwards (fewer instructions than
// choosing coefficients).  q = r/h, hinv = 1/h, ri = 1/r.
template <typename R>
__device__ __forceinline__ void m4_kernel(R q, R hinv, R ri, R& g, R& phi) {
  const R hinv3 = hinv * hinv * hinv;
  const R ri3 = ri * ri * ri;
  const R q2 = q * q;
  // q < 1: g h^3 = 4/3 - 6/5 q^2 + 1/2 q^3, phi h = -7/5 + 2/3 q^2 - 3/10 q^4 + 1/10 q^5
  const R gA = fma(q2, fma(R(0.5), q, R(-1.2)), R(4.0 / 3.0));
  const R pA = fma(q2, fma(q2, fma(R(0.1), q, R(-0.3)), R(2.0 / 3.0)), R(-1.4));
  // 1 <= q < 2: g h^3 = 8/3 - 3 q + 6/5 q^2 - 1/6 q^3 - 1/(15 q^3),
  //             phi h = -8/5 + 4/3 q^2 - q^3 + 3/10 q^4 - 1/30 q^5 + 1/(15 q)
  const R gB = fma(q, fma(q, fma(R(-1.0 / 6.0), q, R(1.2)), R(-3)), R(8.0 / 3.0));
  const R pB = fma(q2, fma(q, fma(q, fma(R(-1.0 / 30.0), q, R(0.3)), R(-1)), R(4.0 / 3.0)), R(-1.6));
  const bool in1 = q < R(1);
  const R gk = fma(hinv3, in1 ? gA : gB, in1 ? R(0) : R(-1.0 / 15.0) * ri3);
  const R pk = fma(hinv, in1 ? pA : pB, in1 ? R(0) : R(1.0 / 15.0) * ri);
  const bool out2 = q >= R(2);
  g = out2 ? ri3 : gk;
  phi = out2 ? -ri : pk;
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; using T2 = float2; };
template <> struct Vec4<double> { using T = double4_16a; using T2 = double2; };

// Unsoftened pair: a -= m r^-3 d, phi -= m / r.
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

// Two unsoftened pairs of one target in the packed FP32 instructions (two
// lanes of FP32 per register pair, one issue slot): sources given negated,
// (-x, -y, -z, -m), so that every operation rounds exactly as pair_far's.
__device__ __forceinline__ void pair_far2(float2 xi, float2 yi, float2 zi, float2 nx, float2 ny, float2 nz,
                                          float2 nm, float2& ax, float2& ay, float2& az, float2& pt) {
  const float2 dx = __fadd2_rn(xi, nx), dy = __fadd2_rn(yi, ny), dz = __fadd2_rn(zi, nz);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
  const float2 mr = __fmul2_rn(nm, ri);                     // -m / r
  const float2 mr3 = __fmul2_rn(mr, __fmul2_rn(ri, ri));    // -m / r^3
  ax = __ffma2_rn(mr3, dx, ax);
  ay = __ffma2_rn(mr3, dy, ay);
  az = __ffma2_rn(mr3, dz, az);
  pt = __fadd2_rn(pt, mr);
}

// Candidate pair: softened when r < 2 max(h_i, h_j) (mean of both kernels),
// unsoftened otherwise; the self pair contributes nothing.
template <typename R>
__device__ __forceinline__ void pair_cand(R xi, R yi, R zi, R hinvi, R h2i, bool self,
                                          const typename Vec4<R>::T& s, const typename Vec4<R>::T2& hh, R& ax,
                                          R& ay, R& az, R& pt) {
  const R dx = xi - s.x, dy = yi - s.y, dz = zi - s.z;
  const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const R ri = (r2 > R(0)) ? rsq(r2) : R(0);
  R g, phi;
  if (r2 < fmax(h2i, hh.y)) {
    const R r = r2 * ri;
    R gi, pi, gj, pj;
    m4_kernel<R>(r * hinvi, hinvi, ri, gi, pi);
    m4_kernel<R>(r * hh.x, hh.x, ri, gj, pj);
    g = R(0.5) * (gi + gj);
    phi = R(0.5) * (pi + pj);
  } else {
    g = ri * ri * ri;
    phi = -ri;
  }
  const R m = self ? R(0) : s.w;
  const R mg = m * g;
  ax = fma(-mg, dx, ax);
  ay = fma(-mg, dy, ay);
  az = fma(-mg, dz, az);
  pt = fma(m, phi, pt);
}

template <bool F32> __host__ __device__ constexpr int p2p_warps() { return F32 ? P2P_WARPS : P2P_WARPS / 2; }

// Near sums v (a, Phi) of sorted particle i plus its far field: scaled by G
// and written in caller order.
template <bool F32, typename R>
__device__ __forceinline__ void p2p_finish(const P2PArgs& a, int i, const R (&v)[4]) {
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
  double pot = a.G * f[3];
  if (a.self_pot) pot += a.G * a.pm[i] * (-1.4 / a.ph[i]);
  const int o = a.perm[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) a.acc[3 * (size_t)o + c] = a.G * f[c];
  if (a.pot) a.pot[o] = pot;
}

// One warp per target leaf.  Sources: the particles of the leaf's neighbour
// list, streamed 32 at a time over consecutive list entries (every lane
// busy), moved to the target leaf's frame (FP32 form) and split once per
// source into those that may lie inside the kernel of some target
// (|x_j - s_L| < l_L + 2 max(h_max,L, h_j), with a small safety factor) and
// those that cannot; the latter take the unsoftened branch-free loop.
template <bool F32>
__global__ void __launch_bounds__(P2P_NT, F32 ? 3 : 1) k_p2p(const P2PArgs a) {
  using R = typename std::conditional<F32, float, double>::type;
  using V = typename Vec4<R>::T;
  using V2 = typename Vec4<R>::T2;
  constexpr int NW = p2p_warps<F32>();
  constexpr int SB = P2P_SB;
  __shared__ V s_far[NW][SB];
  __shared__ V s_near[NW][SB];
  __shared__ V2 s_nhh[NW][SB];
  __shared__ short s_nloc[NW][SB];  // candidate's index in the target leaf, -1 outside it
  __shared__ unsigned short s_sq[NW][F32 ? 1 : 64];  // FP64 softened pairs: candidate slot << 5 | owner lane
  // phase sums at the end of a leaf; the FP64 softened-pair results during its loop
  __shared__ __align__(4 * sizeof(R)) R s_red[NW][4][32];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int nextra = (int)a.d_split[0];
  const int nitems = nextra + (int)a.counts[1];
  unsigned long long pairs = 0;  // this lane's share of the pair evaluations
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(a.leaf_counter, 1);
    item = __shfl_sync(SFMM_FULL, item, 0);
    if (item >= nitems) break;
    int leaf, chunk = 0;
    if (item < nextra) {
      const int2 x = a.extra[item];
      leaf = x.x;
      chunk = x.y;
    } else {
      leaf = item - nextra;
    }
    const int pslot = a.split ? a.split[leaf] : -1;
    const int L = a.leaf_node[leaf];
    const int fL = a.nfirst[L], nL = a.ncount[L];
    const float4 hiL = a.geo_hi[L], loL = a.geo_lo[L];
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
    R xi0 = R(0), yi0 = R(0), zi0 = R(0), hinvi0 = R(0), h2i0 = R(0);
    R xi1 = R(0), yi1 = R(0), zi1 = R(0), hinvi1 = R(0), h2i1 = R(0);
    auto load_target = [&](int i, R& x, R& y, R& z, R& hinv, R& h2) {
      if constexpr (F32) {
        const float4 p = a.prel[i];
        const float4 hh = a.phh[i];
        x = p.x; y = p.y; z = p.z; hinv = hh.x; h2 = hh.y;
      } else {
        const double h = a.ph[i];
        x = a.px[i]; y = a.py[i]; z = a.pz[i]; hinv = 1.0 / h; h2 = 4.0 * h * h;
      }
    };
    if (on0) load_target(fL + t0, xi0, yi0, zi0, hinvi0, h2i0);
    if (on1) load_target(fL + t1, xi1, yi1, zi1, hinvi1, h2i1);
    R ax0 = R(0), ay0 = R(0), az0 = R(0), pt0 = R(0);
    R ax1 = R(0), ay1 = R(0), az1 = R(0), pt1 = R(0);

    const long long off = a.p2p_off[leaf] + (long long)chunk * a.chunk;
    const int cnt = (pslot < 0) ? a.p2p_cnt[leaf] : min(a.chunk, a.p2p_cnt[leaf] - chunk * a.chunk);
    int nfar = 0, nnear = 0;
    int e = 0;                 // next list entry to load
    int tot = 0, pdone = 0;    // particles of the loaded entries / staged so far
    int cum = 0, fS = 0;       // this lane's entry: first particle in the stream, first particle index
    R ox = R(0), oy = R(0), oz = R(0);
    while (true) {
      const bool stream_left = (pdone < tot) || (e < cnt);
      if (stream_left && pdone == tot) {
        // next 32 list entries, one per lane: prefix sum of their particle counts
        const int k = e + lane;
        int nS = 0;
        if (k < cnt) {
          const int S = a.arena[off + k];
          fS = a.nfirst[S];
          nS = a.ncount[S];
          pairs += (unsigned long long)nL * nS - (S == L ? nL : 0);
          if constexpr (F32) {
            const float4 hS = a.geo_hi[S], lS = a.geo_lo[S];
            ox = df_diff(hS.x, lS.x, hiL.x, loL.x);
            oy = df_diff(hS.y, lS.y, hiL.y, loL.y);
            oz = df_diff(hS.z, lS.z, hiL.z, loL.z);
          }
        }
        int incl = nS;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(SFMM_FULL, incl, o);
          if (lane >= o) incl += y;
        }
        cum = (nS > 0) ? incl - nS : INT_MAX;  // padding entries start nowhere
        tot = __shfl_sync(SFMM_FULL, incl, 31);
        pdone = 0;
        e += 32;
      }
      if (stream_left) {
        // stage one window of up to 32 particles of the stream
        const int p = pdone + lane;
        const bool valid = p < tot;
        // the entry holding position p: entries starting before the window
        // plus those starting inside it at or before p (every entry holds at
        // least one particle; the padding entries past the list hold none)
        const bool pre = cum < pdone;
        const int rs = cum - pdone;  // (no overflow: padding lanes test as neither)
        const unsigned starts = __reduce_or_sync(SFMM_FULL, (!pre && rs < 32) ? (1u << rs) : 0u);
        const int before = __popc(__ballot_sync(SFMM_FULL, pre));
        const int l = before + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
        const int d_l = __shfl_sync(SFMM_FULL, fS - cum, l);  // particle index minus stream position
        const R ox_l = __shfl_sync(SFMM_FULL, ox, l), oy_l = __shfl_sync(SFMM_FULL, oy, l),
                oz_l = __shfl_sync(SFMM_FULL, oz, l);
        V v;
        V2 hh;
        R h2j = R(0);  // 2 h_j (FP32 form: rounded up)
        int i = 0;
        if (valid) {
          i = d_l + p;
          if constexpr (F32) {
            const float4 q = a.prel[i];
            v = make_float4(q.x + ox_l, q.y + oy_l, q.z + oz_l, q.w);
            const float4 hr = a.phh[i];
            hh = make_float2(hr.x, hr.y);
            h2j = hr.z;
          } else {
            const double h = a.ph[i];
            v = make_double4_16a(a.px[i], a.py[i], a.pz[i], a.pm[i]);
            hh = make_double2(1.0 / h, 4.0 * h * h);
            h2j = 2.0 * h;
          }
        } else {
          v.x = v.y = v.z = v.w = R(0);
          hh.x = hh.y = R(0);
        }
        R rx = v.x, ry = v.y, rz = v.z;
        if constexpr (!F32) {
          rx -= cLx;
          ry -= cLy;
          rz -= cLz;
        }
        // reach = l_L + 2 max(h_L, h_j) (l_L and h_L carry a 1.0001 margin)
        const R reach = lL + fmax(R(2) * hL, h2j);
        const bool near = valid && (fma(rx, rx, fma(ry, ry, rz * rz)) < reach * reach);
        const unsigned bn = __ballot_sync(SFMM_FULL, near), bf = __ballot_sync(SFMM_FULL, valid && !near);
        if (near) {
          const int q = nnear + __popc(bn & lt);
          s_near[warp][q] = v;
          s_nhh[warp][q] = hh;
          s_nloc[warp][q] = (short)((i >= fL && i < fL + nL) ? i - fL : -1);
        } else if (valid) {
          const int q = nfar + __popc(bf & lt);
          if constexpr (F32) {
            // pairs of sources, negated: {x0, x1, y0, y1}, {z0, z1, m0, m1}
            float* const fxy = reinterpret_cast<float*>(&s_far[warp][q >> 1]);
            float* const fzm = reinterpret_cast<float*>(&s_far[warp][SB / 2 + (q >> 1)]);
            const int hb = q & 1;
            fxy[hb] = -v.x;
            fxy[2 + hb] = -v.y;
            fzm[hb] = -v.z;
            fzm[2 + hb] = -v.w;
          } else {
            s_far[warp][q] = v;
          }
        }
        nnear += __popc(bn);
        nfar += __popc(bf);
        pdone += min(32, tot - pdone);
      }
      const bool last = !((pdone < tot) || (e < cnt));
      if (!(nfar > SB - 32 || nnear > SB - 32 || last)) continue;
      __syncwarp();
      if constexpr (F32) {
        if (nfar & 1) {
          // odd count: the last pair's second source repeats the first with
          // no mass (outside every kernel, so r > 0)
          if (lane == 0) {
            float* const fxy = reinterpret_cast<float*>(&s_far[warp][nfar >> 1]);
            float* const fzm = reinterpret_cast<float*>(&s_far[warp][SB / 2 + (nfar >> 1)]);
            fxy[1] = fxy[0];
            fxy[3] = fxy[2];
            fzm[1] = fzm[0];
            fzm[3] = 0.0f;
          }
          __syncwarp();
        }
      }
      if (lane_on) {
        // unsoftened sources
        if constexpr (F32) {
          // one pass per target slot (the second only for leaves of more
          // than 32 particles)
          const int np = (nfar + 1) >> 1;
          auto far_pass = [&](float xi, float yi, float zi, float& ax, float& ay, float& az, float& pt) {
            const float2 x2 = make_float2(xi, xi), y2 = make_float2(yi, yi), z2 = make_float2(zi, zi);
            float2 fx = make_float2(0.0f, 0.0f), fy = fx, fz = fx, fp = fx;
            for (int pj = ph; pj < np; pj += nph) {
              const float4 a = s_far[warp][pj], b = s_far[warp][SB / 2 + pj];
              pair_far2(x2, y2, z2, make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                        make_float2(b.z, b.w), fx, fy, fz, fp);
            }
            ax += fx.x + fx.y;
            ay += fy.x + fy.y;
            az += fz.x + fz.y;
            pt += fp.x + fp.y;
          };
          far_pass(xi0, yi0, zi0, ax0, ay0, az0, pt0);
          if (nL > 32) far_pass(xi1, yi1, zi1, ax1, ay1, az1, pt1);
        } else if (nL > 32) {
        // FP64 form, more than 32 targets (up to 32: balanced, below)
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
        // candidates inside some kernel of the leaf, softened in place
        if (F32 || nL > 32) {
          for (int jn = ph; jn < nnear; jn += nph) {
            const V s0 = s_near[warp][jn];
            const V2 hh = s_nhh[warp][jn];
            const int loc = s_nloc[warp][jn];
            pair_cand<R>(xi0, yi0, zi0, hinvi0, h2i0, loc == t0, s0, hh, ax0, ay0, az0, pt0);
            if (nL > 32) pair_cand<R>(xi1, yi1, zi1, hinvi1, h2i1, loc == t1, s0, hh, ax1, ay1, az1, pt1);
          }
        }
      }
      if (!F32 && nL <= 32 && nfar > 0) {
        // FP64 form, up to 32 targets: the nL x nfar unsoftened pairs (target
        // major) cut into 32 equal runs, one per lane -- every lane busy, and
        // FP64 work costs per warp instruction whatever the active lanes.  A
        // run spans at most two targets; the partials go back to the lane
        // holding each target (lane t: target t, phase 0), which adds them in
        // lane order
        const int P = nL * nfar;
        const int b0 = (lane * P) >> 5, b1 = ((lane + 1) * P) >> 5;
        R fx = R(0), fy = R(0), fz = R(0), fp = R(0);  // the run's current target
        R gx = R(0), gy = R(0), gz = R(0), gp = R(0);  // its first target, once it moved on
        bool moved = false;
        if (b0 < b1) {
          int t = b0 / nfar, j = b0 - t * nfar;
          R x = a.px[fL + t], y = a.py[fL + t], z = a.pz[fL + t];
          for (int k = b0; k < b1; ++k) {
            if (j == nfar) {
              gx = fx; gy = fy; gz = fz; gp = fp;
              fx = fy = fz = fp = R(0);
              moved = true;
              ++t;
              j = 0;
              x = a.px[fL + t];
              y = a.py[fL + t];
              z = a.pz[fL + t];
            }
            pair_far<R>(x, y, z, s_far[warp][j], fx, fy, fz, fp);
            ++j;
          }
        }
        // lanes covering target t: from the one holding pair t nfar (which
        // may have started in target t - 1: then its second partial) to the
        // one holding pair (t + 1) nfar - 1
        int l0 = 0, l1 = -1;
        bool second = false;
        if (lane < nL) {
          l0 = (32 * lane * nfar + 31) / P;
          l1 = (32 * ((lane + 1) * nfar - 1) + 31) / P;
          second = ((l0 * P) >> 5) < lane * nfar;
        }
        R sx = R(0), sy = R(0), sz = R(0), sp = R(0);
        __syncwarp();
        s_red[warp][0][lane] = moved ? fx : R(0);
        s_red[warp][1][lane] = moved ? fy : R(0);
        s_red[warp][2][lane] = moved ? fz : R(0);
        s_red[warp][3][lane] = moved ? fp : R(0);
        __syncwarp();
        if (second) {
          sx = s_red[warp][0][l0];
          sy = s_red[warp][1][l0];
          sz = s_red[warp][2][l0];
          sp = s_red[warp][3][l0];
        }
        __syncwarp();
        s_red[warp][0][lane] = moved ? gx : fx;
        s_red[warp][1][lane] = moved ? gy : fy;
        s_red[warp][2][lane] = moved ? gz : fz;
        s_red[warp][3][lane] = moved ? gp : fp;
        __syncwarp();
        for (int l = second ? l0 + 1 : l0; l <= l1; ++l) {
          sx += s_red[warp][0][l];
          sy += s_red[warp][1][l];
          sz += s_red[warp][2][l];
          sp += s_red[warp][3][l];
        }
        if (lane < nL) {
          ax0 += sx;
          ay0 += sy;
          az0 += sz;
          pt0 += sp;
        }
        __syncwarp();
      }
      if (!F32 && nL <= 32 && nnear > 0) {
        // FP64 form, up to 32 targets: the unsoftened candidates in place; a
        // pair inside a kernel goes to the warp's queue, and every 32 queued
        // pairs are evaluated one per lane (target records by shuffle from the
        // lane holding them) and handed back to their owner lanes, which add
        // them in queue order.  The FP64 pipe costs the same per warp
        // instruction whatever the active lanes, so the softened branch pays
        // only once per 32 pairs; in the FP32 form the in-place branch is
        // faster (measured)
        V* const s_soft = reinterpret_cast<V*>(&s_red[warp][0][0]);
        auto soft_batch = [&](int cnt, unsigned mine) {
          __syncwarp();
          const int ent = (lane < cnt) ? (int)s_sq[warp][lane] : 0;
          const int o = ent & 31, jn = ent >> 5;
          const int t = o - (o / ntl) * ntl;  // the owner's target, held by lane t
          const R tx = __shfl_sync(SFMM_FULL, xi0, t), ty = __shfl_sync(SFMM_FULL, yi0, t),
                  tz = __shfl_sync(SFMM_FULL, zi0, t), thinv = __shfl_sync(SFMM_FULL, hinvi0, t);
          V c;
          c.x = c.y = c.z = c.w = R(0);
          if (lane < cnt) {
            const V s0 = s_near[warp][jn];
            const V2 hh = s_nhh[warp][jn];
            const R dx = tx - s0.x, dy = ty - s0.y, dz = tz - s0.z;
            const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            const R ri = (r2 > R(0)) ? rsq(r2) : R(0);
            const R r = r2 * ri;
            R gi, pi, gj, pj;
            m4_kernel<R>(r * thinv, thinv, ri, gi, pi);
            m4_kernel<R>(r * hh.x, hh.x, ri, gj, pj);
            const R mg = s0.w * (R(0.5) * (gi + gj));
            c.x = -mg * dx;
            c.y = -mg * dy;
            c.z = -mg * dz;
            c.w = s0.w * (R(0.5) * (pi + pj));
          }
          s_soft[lane] = c;
          __syncwarp();
          while (mine) {
            const int e = __ffs(mine) - 1;
            mine &= mine - 1;
            const V v = s_soft[e];
            ax0 += v.x;
            ay0 += v.y;
            az0 += v.z;
            pt0 += v.w;
          }
          __syncwarp();
        };
        int qn = 0;
        unsigned m0 = 0u, m1 = 0u;  // queue positions [0, 32) and [32, 64) this lane owns
        for (int base = 0; base < nnear; base += nph) {
          const int jn = base + ph;
          bool ins = false;
          if (lane_on && jn < nnear) {
            const V s0 = s_near[warp][jn];
            const V2 hh = s_nhh[warp][jn];
            const bool self = s_nloc[warp][jn] == t0;
            const R dx = xi0 - s0.x, dy = yi0 - s0.y, dz = zi0 - s0.z;
            const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            ins = !self && r2 < fmax(h2i0, hh.y);
            // outside both kernels: unsoftened (r >= 2 h > 0); else nothing here
            const bool skip = self || ins;
            const R ri = rsq(skip ? R(1) : r2);
            const R mr = (skip ? R(0) : s0.w) * ri;
            const R mr3 = mr * (ri * ri);
            ax0 = fma(-mr3, dx, ax0);
            ay0 = fma(-mr3, dy, ay0);
            az0 = fma(-mr3, dz, az0);
            pt0 -= mr;
          }
          const unsigned b = __ballot_sync(SFMM_FULL, ins);
          if (b) {
            if (ins) {
              const int pos = qn + __popc(b & lt);
              s_sq[warp][pos] = (unsigned short)((jn << 5) | lane);
              if (pos < 32) m0 |= 1u << pos;
              else m1 |= 1u << (pos - 32);
            }
            qn += __popc(b);
            if (qn >= 32) {
              soft_batch(32, m0);
              // carry the queued pairs beyond the batch to the front
              const int rest = qn - 32;
              const unsigned short carry = (lane < rest) ? s_sq[warp][32 + lane] : (unsigned short)0;
              __syncwarp();
              if (lane < rest) s_sq[warp][lane] = carry;
              qn = rest;
              m0 = m1;
              m1 = 0u;
            }
          }
        }
        if (qn > 0) soft_batch(qn, m0);
      }
      __syncwarp();
      nfar = 0;
      nnear = 0;
      if (last) break;
    }
    if (!on0) { ax0 = ay0 = az0 = pt0 = R(0); }
    if (!on1) { ax1 = ay1 = az1 = pt1 = R(0); }

    // combine the phases of each target, add the far field, write out
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
          R sacc = R(0);
          for (int q = 0; q < nph; ++q) sacc += s_red[warp][c][q * ntl + lane];
          v[c] = sacc;
        }
        if (pslot < 0) {
          p2p_finish<F32>(a, fL + t, v);
        } else {
          R* pp = static_cast<R*>(a.part) + ((size_t)(pslot + chunk) * a.lmax + t) * 4;
#pragma unroll
          for (int c = 0; c < 4; ++c) pp[c] = v[c];
        }
      }
      __syncwarp();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(SFMM_FULL, pairs, o);
  if (lane == 0 && pairs) atomicAdd(a.pair_counter, pairs);
}

// Long lists: thread per leaf; a list of more than `chunk` entries gets
// ceil(entries / chunk) partial slots and one extra work item
// per chunk after the first.  ctr[0]: extra items, ctr[1]: slots, ctr[2]:
// split leaves.  Which slots a leaf gets does not change any result.
__global__ void k_p2p_split(const uint32_t* __restrict__ counts, const int* __restrict__ p2p_cnt,
                            int* __restrict__ split, int2* __restrict__ extra, int* __restrict__ slist,
                            unsigned long long* __restrict__ ctr, int max_extra, int max_slots, int max_split,
                            int chunk, int* __restrict__ status) {
  const int nleaves = (int)counts[1];
  for (int leaf = blockIdx.x * blockDim.x + threadIdx.x; leaf < nleaves; leaf += gridDim.x * blockDim.x) {
    const int cnt = p2p_cnt[leaf];
    if (cnt <= chunk) {
      split[leaf] = -1;
      continue;
    }
    const int nch = (cnt + chunk - 1) / chunk;
    const int x = (int)atomicAdd(ctr, (unsigned long long)(nch - 1));
    const int base = (int)atomicAdd(ctr + 1, (unsigned long long)nch);
    const int q = (int)atomicAdd(ctr + 2, 1ull);
    if (x + nch - 1 > max_extra || base + nch > max_slots || q >= max_split) {
      // the walk counted these exactly: more means an internal inconsistency
      split[leaf] = -1;
      set_status(status, SFMM_ST_INTERNAL);
      continue;
    }
    split[leaf] = base;
    for (int k = 1; k < nch; ++k) extra[x + k - 1] = make_int2(leaf, k);
    slist[q] = leaf;
  }
}

// Split leaves: one warp per leaf sums the chunks' partial sums in chunk
// order (so reruns are bitwise identical) and finishes as an unsplit leaf.
template <bool F32>
__global__ void k_p2p_combine(const P2PArgs a) {
  const int nsplit = (int)a.d_split[2];
  using R = typename std::conditional<F32, float, double>::type;
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int q = w0; q < nsplit; q += nw) {
    const int leaf = a.slist[q];
    const int L = a.leaf_node[leaf];
    const int fL = a.nfirst[L], nL = a.ncount[L];
    const int nch = (a.p2p_cnt[leaf] + a.chunk - 1) / a.chunk;
    const int base = a.split[leaf];
    for (int t = lane; t < nL; t += 32) {
      R v[4] = {R(0), R(0), R(0), R(0)};
      for (int k = 0; k < nch; ++k) {
        const R* pp = static_cast<const R*>(a.part) + ((size_t)(base + k) * a.lmax + t) * 4;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] += pp[c];
      }
      p2p_finish<F32>(a, fL + t, v);
    }
  }
}

int run_p2p(sfmm_ctx* c, double* acc, double* pot) {
  const int nl = c->nleaves;
  int rc;
  // the sums read the potential: without a caller array it goes to scratch
  if (!pot) {
    if ((rc = c->out_pot.ensure(sizeof(double) * (size_t)c->n))) return rc;
    pot = c->out_pot.as<double>();
  }
  c->red_acc = acc;
  c->red_pot = pot;
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  SFMM_CUDA_TRY(cudaMemsetAsync(ctr + 10, 0, 4 * sizeof(unsigned long long), c->stream));
  const bool f32 = (c->precision == SFMM_FP32);
  // long lists: slots, extra items and split leaves are counted by the split
  // pass on the device; the buffers are sized from bounds on the host (a list
  // of cnt > chunk entries takes ceil(cnt / chunk) <= 2 cnt / chunk slots, so
  // all of them fit 2 arena / chunk), with no wait for the walk
  const int64_t arena_cap = (int64_t)(c->arena.bytes / sizeof(int));
  const int nslots = (int)std::min<int64_t>(2 * arena_cap / c->p2p_chunk + 2, INT32_MAX / 2);
  const int nsplit =
      (int)std::min<int64_t>(std::min<int64_t>(c->graph_mode ? c->n : nl, arena_cap / (c->p2p_chunk + 1) + 1), nslots);
  const int nextra = nslots;
  int lmax = c->leaf_size;
  for (int v : c->h_sys_lsz) lmax = v > lmax ? v : lmax;
  const int nl_b = c->graph_mode ? (int)c->n : nl;  // leaf-indexed: the bound for a captured step
  if ((rc = c->p2p_split.ensure(sizeof(int) * (size_t)nl_b))) return rc;
  if ((rc = c->p2p_extra.ensure(sizeof(int2) * (size_t)nextra))) return rc;
  if ((rc = c->p2p_slist.ensure(sizeof(int) * (size_t)nsplit))) return rc;
  if ((rc = c->p2p_part.ensure((f32 ? sizeof(float) : sizeof(double)) * 4 * (size_t)lmax * nslots))) return rc;
  const int sblocks = std::max(1, std::min((nl_b + 255) / 256, 8 * num_sms(c->device)));
  k_p2p_split<<<sblocks, 256, 0, c->stream>>>(c->d_counts, c->p2p_cnt.as<int>(), c->p2p_split.as<int>(),
                                                     c->p2p_extra.as<int2>(), c->p2p_slist.as<int>(), ctr + 11,
                                                     nextra, nslots, nsplit, c->p2p_chunk, c->d_status);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  P2PArgs a{};
  a.counts = c->d_counts;
  a.leaf_node = c->leaf_node.as<int>();
  a.nfirst = c->nfirst.as<int>();
  a.ncount = c->ncount.as<int>();
  a.geo_hi = c->geo_hi.as<float4>();
  a.geo_lo = c->geo_lo.as<float4>();
  a.arena = c->arena.as<int>();
  a.p2p_off = c->p2p_off.as<long long>();
  a.p2p_cnt = c->p2p_cnt.as<int>();
  a.prel = c->prel.as<float4>();
  a.phh = c->phh.as<float4>();
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
  a.d_split = ctr + 11;
  a.extra = c->p2p_extra.as<int2>();
  a.split = c->p2p_split.as<int>();
  a.slist = c->p2p_slist.as<int>();
  a.part = c->p2p_part.p;
  a.lmax = lmax;
  a.chunk = c->p2p_chunk;
  a.pair_counter = ctr + 3;
  const int nt = 32 * (f32 ? p2p_warps<true>() : p2p_warps<false>());
  int per_sm = 0;
  if (f32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<true>, nt, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<false>, nt, 0);
  if (per_sm < 1) per_sm = 1;
  if (c->p2p_blocks > 0 && c->p2p_blocks < per_sm) per_sm = c->p2p_blocks;  // option: fewer blocks per SM
  const int nblocks = per_sm * num_sms(c->device);
  if (f32) k_p2p<true><<<nblocks, nt, 0, c->stream>>>(a);
  else k_p2p<false><<<nblocks, nt, 0, c->stream>>>(a);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  {
    // split leaves (their count is on the device): a persistent grid
    const int cblocks = std::min(2 * num_sms(c->device), (nsplit + 7) / 8 + 1);
    if (f32) k_p2p_combine<true><<<cblocks, 256, 0, c->stream>>>(a);
    else k_p2p_combine<false><<<cblocks, 256, 0, c->stream>>>(a);
    ++c->nlaunch;
    SFMM_CUDA_TRY(cudaGetLastError());
  }
  return SFMM_OK;
}

int p2p_blocks_fit(sfmm_ctx* c) {
  const bool f32 = (c->precision == SFMM_FP32);
  const int nt = 32 * (f32 ? p2p_warps<true>() : p2p_warps<false>());
  int per_sm = 0;
  if (f32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<true>, nt, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<false>, nt, 0);
  return per_sm < 1 ? 1 : per_sm;
}

}  // namespace sfmm
