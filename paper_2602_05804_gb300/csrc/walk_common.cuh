// Device pieces shared by the two walk kernels (walk.cu: one warp per leaf,
// replaying Algorithm 1 for the leaf's branch; walk_shared.cu: one warp per
// node, each node's pairs evaluated once): the acceptance test of Sect. 3,
// the node-node expansion (Eq. dmkdeffmm) of one pair, the warp
// reduce-scatter of coefficients and the generated expansion dispatch.
#pragma once
#include <type_traits>

#include "expansion_gen.cuh"
#include "sfmm_internal.cuh"

namespace sfmm {

#define WALK_WARPS 4
#define WALK_NT (WALK_WARPS * 32)
#define WALK_MQ 64

enum { MODE_COMPUTE = 0, MODE_COUNT = 1, MODE_WRITE = 2 };

struct WalkArgs {
  int nleaves;
  const int* leaf_node;
  const int* nfirst;
  const int* ncount;
  const int* nright;
  const float4* geo_hi;
  const float4* geo_lo;
  const double* ncx;
  const double* ncy;
  const double* ncz;
  const double* nsize;
  const double* nhmax;
  const float* Qf;
  const double* Qd;
  int nqs;  // row stride of Qf
  const float4* prel;
  const double* px;
  const double* py;
  const double* pz;
  int* ring;
  int ring_cap;  // power of two
  int* leaf_counter;
  int* arena;
  unsigned long long* arena_counter;
  unsigned long long* split_counter;  // [0]: chunks of split lists, [1]: split lists
  int chunk;                          // neighbour-list entries per near-field work item
  long long arena_cap;
  long long* p2p_off;
  int* p2p_cnt;
  float4* far32;
  double* far64;
  int* status;
  unsigned long long* stat;  // m2l, m2l_unique, p2p_leaves, p2p_pairs, fallbacks
  double theta;
  float theta_f;
  float theta2_f;
  const int* psys;            // system of each particle (null: one system)
  const int* sys_root;        // root node of each system
  int* m2l_cnt;               // MODE_COUNT
  const long long* m2l_off;   // MODE_WRITE
  int* dump_level;
  int* dump_src;
};

template <int P> struct Exp;
#define SFMM_EXP(PP, PP1)                                                                                      \
  template <> struct Exp<PP> {                                                                                 \
    static constexpr int NM = SFMM_NM_##PP, NF = SFMM_NF_##PP, NC = NM + NF;                                   \
    static constexpr int NQ = ncoef(PP), NMONO1 = ncoef(PP + 1);                                               \
    template <typename T> __device__ static void derivs(T x, T y, T z, T ri, T* D) { sfmm_derivs_##PP1(x, y, z, ri, D); } \
    template <typename T> __device__ static void m2l(const T* D, const T* Q, T* C) { sfmm_m2l_##PP(D, Q, C); }  \
    template <typename T> __device__ static void m2l_nodip(const T* D, const T* Q, T* C) { sfmm_m2l_##PP##_nodip(D, Q, C); } \
    template <typename T, typename U> __device__ static void l2p(const T* am, const U* C, T* o) { sfmm_l2p_##PP(am, C, o); } \
    template <typename T> __device__ static void mono(T x, T y, T z, T* o) { sfmm_mono_##PP(x, y, z, o); }     \
    template <typename T> __device__ static void mono1(T x, T y, T z, T* o) { sfmm_mono_##PP1(x, y, z, o); }   \
    __device__ static const signed char* table() { return &sfmm_l2l_table_##PP[0][0]; }                       \
  };
SFMM_EXP(0, 1)
SFMM_EXP(1, 2)
SFMM_EXP(2, 3)
SFMM_EXP(3, 4)
SFMM_EXP(4, 5)
#undef SFMM_EXP

// Reduce-scatter over the warp: on entry every lane holds v[0..32); on exit
// v[0] on lane l is the warp sum of entry l.
template <typename T>
__device__ __forceinline__ T reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int step = 0; step < 5; ++step) {
    const int o = 16 >> step;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int c = 0; c < o; ++c) {
      T send = upper ? v[c] : v[c + o];
      T keep = upper ? v[c + o] : v[c];
      v[c] = keep + __shfl_xor_sync(SFMM_FULL, send, o);
    }
  }
  return v[0];
}

// Acceptance test of Sect. 3: accept iff (l_t + l_s) < theta d and not
// d < l_t + l_s + R_kern max(h_t, h_s).
__device__ __forceinline__ bool decide(const float4& hiA, const float4& loA, const float4& hiB, const float4& loB,
                                       int A, int B, const WalkArgs& a, int& nfb, float& dx, float& dy, float& dz) {
  dx = df_diff(hiB.x, loB.x, hiA.x, loA.x);
  dy = df_diff(hiB.y, loB.y, hiA.y, loA.y);
  dz = df_diff(hiB.z, loB.z, hiA.z, loA.z);
  // squared form (all terms non-negative): l^2 < theta^2 d^2 and d^2 >= (l + 2h)^2;
  // the float32 error is below 1.5e-6 relative, the tie band 1e-5
  const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float ls = hiA.w + hiB.w;
  const float hm = fmaxf(loA.w, loB.w);
  const float td2 = a.theta2_f * d2, ls2 = ls * ls;
  const float m1 = td2 - ls2, t1 = 1e-5f * (td2 + ls2);
  const float rhs = fmaf(2.0f, hm, ls);
  const float rhs2 = rhs * rhs;
  const float m2 = d2 - rhs2, t2 = 1e-5f * (d2 + rhs2);
  if (d2 >= 1e-30f && d2 <= 1e30f) {
    if (m1 < -t1 || m2 < -t2) return false;
    if (m1 > t1 && m2 > t2) return true;
  }
  ++nfb;
  const double ddx = dsub(a.ncx[B], a.ncx[A]);
  const double ddy = dsub(a.ncy[B], a.ncy[A]);
  const double ddz = dsub(a.ncz[B], a.ncz[A]);
  const double dd = __dsqrt_rn(dadd(dadd(dmul(ddx, ddx), dmul(ddy, ddy)), dmul(ddz, ddz)));
  const double lsd = dadd(a.nsize[A], a.nsize[B]);
  const double hmd = fmax(a.nhmax[A], a.nhmax[B]);
  const bool mac = lsd < dmul(a.theta, dd);
  const bool soft = dd < dadd(lsd, dmul(SFMM_RKERN, hmd));
  return mac && !soft;
}

// One node-node interaction (target centre A, source node s) accumulated
// into the lane's coefficients.  In the FP32 form r = s_B - s_A comes from
// the acceptance test (the same double-float difference).
template <int P, bool F32>
__device__ __forceinline__ void m2l_eval(int s, const float4& hiA, const float4& loA, double cAx, double cAy,
                                         double cAz, const WalkArgs& a,
                                         typename std::conditional<F32, float, double>::type* C,
                                         const float4& r) {
  using E = Exp<P>;
  if (s < 0) return;
  if constexpr (F32) {
    const float rx = r.x, ry = r.y, rz = r.z;
    const float ri = rsqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
    float D[E::NMONO1];
    E::derivs(rx * ri, ry * ri, rz * ri, ri, D);
    constexpr int NQ4 = (E::NQ + 3) / 4;
    float Q[NQ4 * 4];
    const float4* q4 = reinterpret_cast<const float4*>(a.Qf + (size_t)s * a.nqs);
#pragma unroll
    for (int t = 0; t < NQ4; ++t) {
      float4 v = __ldg(q4 + t);
      Q[4 * t] = v.x;
      Q[4 * t + 1] = v.y;
      Q[4 * t + 2] = v.z;
      Q[4 * t + 3] = v.w;
    }
    // moments are about the centre of mass: the dipole vanishes to rounding
    E::m2l_nodip(D, Q, C);
  } else {
    const double rx = a.ncx[s] - cAx, ry = a.ncy[s] - cAy, rz = a.ncz[s] - cAz;
    const double ri = rsqrt(fma(rx, rx, fma(ry, ry, rz * rz)));
    double D[E::NMONO1];
    E::derivs(rx * ri, ry * ri, rz * ri, ri, D);
    double Q[E::NQ];
    const double* q = a.Qd + (size_t)s * E::NQ;
#pragma unroll
    for (int t = 0; t < E::NQ; ++t) Q[t] = __ldg(q + t);
    E::m2l(D, Q, C);
  }
}

// Sign (-1)^|gamma| of entry t of a derivative vector (entries are ordered by
// degree: ncoef(k) of them have degree <= k).
__host__ __device__ constexpr int deriv_degree(int t) {
  int k = 0;
  while (ncoef(k) <= t) ++k;
  return k;
}

// One-sided symmetric interaction (Sect. 5, after Dehnen 2002): D_gamma(r) is
// evaluated once for the pair; the target's coefficients from the source's
// moments are added to C as in m2l_eval, and the source's coefficients from
// the target's moments QA, with D_gamma(-r) = (-1)^|gamma| D_gamma(r), are
// added to the source's received sums EB (FP64 atomics).
template <int P, bool F32>
__device__ __forceinline__ void m2l_eval_sym(int s, double cAx, double cAy, double cAz, const WalkArgs& a,
                                             typename std::conditional<F32, float, double>::type* C,
                                             const float4& r,
                                             const typename std::conditional<F32, float, double>::type* QA,
                                             double* EB) {
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  if (s < 0) return;
  R D[E::NMONO1];
  R Q[F32 ? ((E::NQ + 3) / 4) * 4 : E::NQ];
  if constexpr (F32) {
    const float ri = rsqrtf(fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z)));
    E::derivs(r.x * ri, r.y * ri, r.z * ri, ri, D);
    const float4* q4 = reinterpret_cast<const float4*>(a.Qf + (size_t)s * a.nqs);
#pragma unroll
    for (int t = 0; t < (E::NQ + 3) / 4; ++t) {
      const float4 v = __ldg(q4 + t);
      Q[4 * t] = v.x;
      Q[4 * t + 1] = v.y;
      Q[4 * t + 2] = v.z;
      Q[4 * t + 3] = v.w;
    }
    E::m2l_nodip(D, Q, C);
  } else {
    const double rx = a.ncx[s] - cAx, ry = a.ncy[s] - cAy, rz = a.ncz[s] - cAz;
    const double ri = rsqrt(fma(rx, rx, fma(ry, ry, rz * rz)));
    E::derivs(rx * ri, ry * ri, rz * ri, ri, D);
    const double* q = a.Qd + (size_t)s * E::NQ;
#pragma unroll
    for (int t = 0; t < E::NQ; ++t) Q[t] = __ldg(q + t);
    E::m2l(D, Q, C);
  }
#pragma unroll
  for (int t = 0; t < E::NMONO1; ++t)
    if (deriv_degree(t) & 1) D[t] = -D[t];
  R Cp[E::NC];
#pragma unroll
  for (int t = 0; t < E::NC; ++t) Cp[t] = R(0);
  if constexpr (F32) E::m2l_nodip(D, QA, Cp);
  else E::m2l(D, QA, Cp);
#pragma unroll
  for (int t = 0; t < E::NC; ++t) atomicAdd(EB + t, (double)Cp[t]);
}

// The same with r computed here from the node records (FP32 form).
template <int P, bool F32>
__device__ __forceinline__ void m2l_eval(int s, const float4& hiA, const float4& loA, double cAx, double cAy,
                                         double cAz, const WalkArgs& a,
                                         typename std::conditional<F32, float, double>::type* C) {
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (F32 && s >= 0) {
    const float4 hB = a.geo_hi[s], lB = a.geo_lo[s];
    r.x = df_diff(hB.x, lB.x, hiA.x, loA.x);
    r.y = df_diff(hB.y, lB.y, hiA.y, loA.y);
    r.z = df_diff(hB.z, lB.z, hiA.z, loA.z);
  }
  m2l_eval<P, F32>(s, hiA, loA, cAx, cAy, cAz, a, C, r);
}

// Acceptance test without the separation output.
__device__ __forceinline__ bool decide(const float4& hiA, const float4& loA, const float4& hiB, const float4& loB,
                                       int A, int B, const WalkArgs& a, int& nfb) {
  float dx, dy, dz;
  return decide(hiA, loA, hiB, loB, A, B, a, nfb, dx, dy, dz);
}

}  // namespace sfmm
