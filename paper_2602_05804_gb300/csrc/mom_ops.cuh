// Moment operators of order P from the generated expansion code: monomials
// x^a/a! (Eq. massmom) and the translation of scaled moments to a parent
// centre (Eq. massmomtrans).
#pragma once
#include "expansion_gen.cuh"
#include "sfmm_common.cuh"

namespace sfmm {

template <int P> struct MomOps;
#define SFMM_MOMOPS(PP)                                                                               \
  template <> struct MomOps<PP> {                                                                     \
    static constexpr int NQ = ncoef(PP);                                                              \
    template <typename T> __device__ static void mono(T x, T y, T z, T* o) { sfmm_mono_##PP(x, y, z, o); } \
    template <typename T> __device__ static void m2m(const T* g, const T* qc, T* qp) { sfmm_m2m_##PP(g, qc, qp); } \
  };
SFMM_MOMOPS(0)
SFMM_MOMOPS(1)
SFMM_MOMOPS(2)
SFMM_MOMOPS(3)
SFMM_MOMOPS(4)
#undef SFMM_MOMOPS

}  // namespace sfmm
