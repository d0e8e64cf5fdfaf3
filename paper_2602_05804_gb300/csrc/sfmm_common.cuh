// Shared device helpers of the SFMM gravity library (CUDA, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sfmm.h"

#define SFMM_FULL 0xffffffffu
#define SFMM_PMAX 4
#define SFMM_RKERN 2.0

// Device status bits (one int per context, OR-ed by kernels, read once per call).
#define SFMM_ST_NONFINITE   0x01  // a non-finite position, mass or smoothing length
#define SFMM_ST_NONPOSITIVE 0x02  // mass <= 0 or h <= 0
#define SFMM_ST_RING        0x04  // walk frontier ring overflow (capacity)
#define SFMM_ST_ARENA       0x08  // P2P list arena overflow (capacity)
#define SFMM_ST_DEPTH       0x10  // branch deeper than SFMM_MAXDEPTH
#define SFMM_ST_INTERNAL    0x20  // internal consistency check failed
#define SFMM_ST_CHILDLIST   0x40  // child-frontier arena overflow (capacity)

#define SFMM_MAXDEPTH 128
#define SFMM_WALK_ATTEMPTS 6  // walk runs: the first plus regrow-and-retry of short buffers

// Default of the option "p2p_chunk": neighbour lists longer than this many
// entries are split into chunks of it, each a separate near-field work item
// (long lists would otherwise leave one warp working alone at the end of the
// pass).
#define SFMM_P2P_CHUNK_DEFAULT 256

namespace sfmm {

// ---------------------------------------------------------------------------
// Exact-rounding FP64 helpers: every operation rounded as written, no FMA
// contraction, so that acceptance decisions match a plain FP64 evaluation of
// the same expression bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

// ---------------------------------------------------------------------------
// Double-float helpers (Dekker 1971; Knuth's TwoSum): a value carried as an
// unevaluated sum hi + lo of two floats.
// ---------------------------------------------------------------------------
struct dfloat { float hi, lo; };

__device__ __forceinline__ void split_double(double v, float& hi, float& lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ dfloat two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// (hi, lo) + b, renormalised.
__device__ __forceinline__ dfloat df_add_f(dfloat a, float b) {
  dfloat s = two_sum(a.hi, b);
  float lo = __fadd_rn(s.lo, a.lo);
  return two_sum(s.hi, lo);
}

// Difference of two double-float centres as a float (|error| ~ 2^-24 |d|).
__device__ __forceinline__ float df_diff(float ahi, float alo, float bhi, float blo) {
  return __fadd_rn(__fsub_rn(ahi, bhi), __fsub_rn(alo, blo));
}

// ---------------------------------------------------------------------------
// Compensated FP64 sums (Neumaier's variant of Kahan summation, 1974): a sum
// is carried as the rounded running sum s plus the accumulated rounding
// errors c of every addition, each error taken exactly, so the order of the
// operands' magnitudes does not matter.  Two partial sums merge by adding
// one's s to the other and both c's: the total error is about eps |sum| +
// O(n eps^2) sum |x|, instead of O(n eps) sum |x| for a plain sum.  Every
// operation is rounded as written.
//
// The error of t = fl(a + b) is taken as (big - t) + small, with big the
// operand of larger magnitude (Dekker's Fast2Sum, exact under that ordering:
// the same value as Knuth's branch-free TwoSum, in three FP64 operations
// instead of six).  The magnitudes are compared on the bit patterns (for
// finite doubles |a| >= |b| iff the sign-cleared patterns compare so as
// unsigned integers), on the integer pipe: GB300's FP64 pipe is the narrow one.
// ---------------------------------------------------------------------------
struct csum { double s, c; };

__device__ __forceinline__ void cs_add(csum& a, double x) {
  const double t = __dadd_rn(a.s, x);
  const unsigned long long ma = (unsigned long long)__double_as_longlong(a.s) & 0x7fffffffffffffffull;
  const unsigned long long mx = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const bool a_big = ma >= mx;
  const double big = a_big ? a.s : x, small = a_big ? x : a.s;
  const double e = __dadd_rn(__dsub_rn(big, t), small);
  a.s = t;
  a.c = __dadd_rn(a.c, e);
}
__device__ __forceinline__ void cs_merge(csum& a, double bs, double bc) {
  cs_add(a, bs);
  a.c = __dadd_rn(a.c, bc);
}
__device__ __forceinline__ double cs_value(const csum& a) { return __dadd_rn(a.s, a.c); }

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void set_status(int* status, int bits) { atomicOr(status, bits); }

// Number of scaled multi-index coefficients with |alpha| <= p.
__host__ __device__ constexpr int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

}  // namespace sfmm

// Host-side helpers shared by the .cu files.
#define SFMM_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return sfmm_internal_cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

int sfmm_internal_cuda_fail(cudaError_t e, const char* expr, const char* file, int line);
