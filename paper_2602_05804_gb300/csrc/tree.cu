// Tree build of the SFMM solver (Sect. 3): bounding box, Morton keys, radix
// sort, binary radix tree collapsed to leaves of <= leaf_size particles,
// pre-order node layout, node centres of mass, maximum smoothing lengths and
// exact sizes l = max_j |x_j - s| over each node's particles.
#include <cfloat>
#include <climits>
#include <cuda/atomic>

#include "mom_ops.cuh"
#include <type_traits>

#include "sfmm_internal.cuh"

namespace sfmm {

// ---------------------------------------------------------------------------
// Block-wide helpers
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(SFMM_FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < NT / 32) ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(SFMM_FULL, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) warp_tot[lane] = w;  // inclusive per-warp totals
  }
  __syncthreads();
  uint32_t base = warp ? warp_tot[warp - 1] : 0u;
  total = warp_tot[NT / 32 - 1];
  __syncthreads();
  return base + x - v;
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (three passes: tile sums, scan of sums, rescan)
// ---------------------------------------------------------------------------
#define SCAN_NT 512
#define SCAN_ITEMS 8
#define SCAN_TILE (SCAN_NT * SCAN_ITEMS)

__global__ void k_scan_tile_sums(const uint32_t* __restrict__ d, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[SCAN_NT / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * SCAN_NT + threadIdx.x;
    if (i < n) s += d[i];
  }
  uint32_t tot;
  block_exclusive_scan<SCAN_NT>(s, wt, tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums (any count, serial chunks).
__global__ void k_scan_sums(uint32_t* __restrict__ sums, int nt, uint32_t* __restrict__ total_out) {
  __shared__ uint32_t wt[SCAN_NT / 32];
  uint32_t carry = 0;
  for (int base = 0; base < nt; base += SCAN_NT) {
    int i = base + threadIdx.x;
    uint32_t v = (i < nt) ? sums[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<SCAN_NT>(v, wt, tot);
    if (i < nt) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_apply(uint32_t* __restrict__ d, int64_t n, const uint32_t* __restrict__ sums) {
  __shared__ uint32_t wt[SCAN_NT / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  uint32_t carry = sums[blockIdx.x];
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * SCAN_NT + threadIdx.x;
    uint32_t v = (i < n) ? d[i] : 0u;
    uint32_t tot;
    uint32_t ex = block_exclusive_scan<SCAN_NT>(v, wt, tot);
    if (i < n) d[i] = carry + ex;
    carry += tot;
  }
}

int exclusive_scan_u32(sfmm_ctx* c, uint32_t* data, int64_t n, uint32_t* total_dev) {
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nt < 1) nt = 1;
  int rc = c->scan_tmp.ensure(sizeof(uint32_t) * (size_t)nt);
  if (rc) return rc;
  uint32_t* sums = c->scan_tmp.as<uint32_t>();
  k_scan_tile_sums<<<(unsigned)nt, SCAN_NT, 0, c->stream>>>(data, n, sums);
  ++c->nlaunch;
  k_scan_sums<<<1, SCAN_NT, 0, c->stream>>>(sums, (int)nt, total_dev);
  ++c->nlaunch;
  k_scan_apply<<<(unsigned)nt, SCAN_NT, 0, c->stream>>>(data, n, sums);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

// ---------------------------------------------------------------------------
// S1: bounding box + input validation
// ---------------------------------------------------------------------------
#define BB_NT 256

// Order-preserving integer key of a finite double and its inverse (signed
// comparison of keys orders the values; -0 sorts just below +0): extrema and
// checks on the integer pipe instead of GB300's narrow FP64 pipe.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_inv(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// 1 / M for M > 0, within about one unit in the last place: Newton's
// iteration for the reciprocal, r <- r + r (1 - M r), twice from the FP32
// reciprocal of M rounded to FP32 (relative error below 2^-22, so below
// 2^-44 after one step and at FP64 rounding after the second).  Four FP64
// operations in a dependent chain instead of a correctly rounded division;
// magnitudes outside FP32's normal range take the division.
__device__ __forceinline__ double recip_pos(double M) {
  const float mf = __double2float_rn(M);
  if (!(mf > 1e-36f && mf < 1e36f)) return 1.0 / M;
  double r = (double)__frcp_rn(mf);
  r = fma(r, fma(-M, r, 1.0), r);
  r = fma(r, fma(-M, r, 1.0), r);
  return r;
}

// A node's centre as double-float walk records (w fields: filled later).
__device__ __forceinline__ void store_centre_df(int v, double cx, double cy, double cz, float4* __restrict__ geo_hi,
                                                float4* __restrict__ geo_lo) {
  float xh, xl, yh, yl, zh, zl;
  split_double(cx, xh, xl);
  split_double(cy, yh, yl);
  split_double(cz, zh, zl);
  geo_hi[v] = make_float4(xh, yh, zh, 0.0f);
  geo_lo[v] = make_float4(xl, yl, zl, 0.0f);
}

// One particle into a thread's box (as keys) and validity bits: positions,
// masses and h finite (exponent field not all ones), masses and h > 0 (a
// positive double's bit pattern is a positive integer; zero, -0 and
// negatives are not, and NaN fails the test as it fails m > 0).
__device__ __forceinline__ void bbox_take(const double* __restrict__ pos, const double* __restrict__ mass,
                                          const double* __restrict__ h, int i, long long (&mn)[3],
                                          long long (&mx)[3], int& bad) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long b = __double_as_longlong(pos[3 * (int64_t)i + c]);
    if (((b >> 52) & 0x7ff) == 0x7ff) bad |= SFMM_ST_NONFINITE;
    const long long k = b ^ ((b >> 63) & 0x7fffffffffffffffLL);
    mn[c] = min(mn[c], k);
    mx[c] = max(mx[c], k);
  }
  const long long bm = __double_as_longlong(mass[i]), bh = __double_as_longlong(h[i]);
  if (((bm >> 52) & 0x7ff) == 0x7ff || ((bh >> 52) & 0x7ff) == 0x7ff) bad |= SFMM_ST_NONFINITE;
  const long long inf = 0x7ff0000000000000LL, mag = 0x7fffffffffffffffLL;
  if (bm <= 0 || bh <= 0 || (bm & mag) > inf || (bh & mag) > inf) bad |= SFMM_ST_NONPOSITIVE;
}

// Block-wide extrema of the keys: s[c][w] per warp (min c < 3, max c >= 3).
__device__ __forceinline__ void bbox_block(long long (&mn)[3], long long (&mx)[3], long long (&s)[6][BB_NT / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[c] = min(mn[c], __shfl_xor_sync(SFMM_FULL, mn[c], o));
      mx[c] = max(mx[c], __shfl_xor_sync(SFMM_FULL, mx[c], o));
    }
    if (lane == 0) {
      s[c][warp] = mn[c];
      s[3 + c][warp] = mx[c];
    }
  }
  __syncthreads();
}

// Block partials as keys; the last block to finish (a counter the caller
// zeroes) combines them into bbox: [0..2] min, [3..5] max, [6] cube extent
// E, [7] key scale 2^21 / E (0 if E == 0).
__global__ void k_bbox_partial(const double* __restrict__ pos, const double* __restrict__ mass,
                               const double* __restrict__ h, int n, long long* __restrict__ part,
                               unsigned* __restrict__ done, double* __restrict__ bbox, int* __restrict__ status) {
  long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bbox_take(pos, mass, h, i, mn, mx, bad);
  __shared__ long long s[6][BB_NT / 32];
  __shared__ bool s_last;
  bbox_block(mn, mx, s);
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    long long v = s[c][0];
    for (int w = 1; w < BB_NT / 32; ++w) v = (c < 3) ? min(v, s[c][w]) : max(v, s[c][w]);
    part[6 * blockIdx.x + c] = v;
  }
  if (bad) atomicOr(status, bad);
  // publish the partial, then count: the last block sees every partial
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    long long a[6] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int b = lane; b < (int)gridDim.x; b += 32)
  #pragma unroll
      for (int c = 0; c < 6; ++c) {
        const long long v = __ldcg(&part[6 * b + c]);
        a[c] = (c < 3) ? min(a[c], v) : max(a[c], v);
      }
  #pragma unroll
    for (int c = 0; c < 6; ++c)
      for (int o = 16; o > 0; o >>= 1) {
        const long long y = __shfl_xor_sync(SFMM_FULL, a[c], o);
        a[c] = (c < 3) ? min(a[c], y) : max(a[c], y);
      }
    if (lane == 0) {
      double E = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double lo = dkey_inv(a[c]), hi = dkey_inv(a[3 + c]);
        bbox[c] = lo;
        bbox[3 + c] = hi;
        const double e = dsub(hi, lo);
        if (e > E) E = e;
      }
      bbox[6] = E;
      bbox[7] = (E > 0.0) ? __ddiv_rn(2097152.0, E) : 0.0;
    }
  }
}

// Per-system bounding boxes for a batch: one block per system; bbox[8 s ..].
__global__ void k_bbox_seg(const double* __restrict__ pos, const double* __restrict__ mass,
                           const double* __restrict__ h, const int* __restrict__ off, double* __restrict__ bbox,
                           int* __restrict__ status) {
  const int sys = blockIdx.x;
  const int lo = off[sys], hi = off[sys + 1];
  long long mn[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, mx[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  int bad = 0;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) bbox_take(pos, mass, h, i, mn, mx, bad);
  __shared__ long long s[6][BB_NT / 32];
  bbox_block(mn, mx, s);
  if (threadIdx.x == 0) {
    double E = 0.0;
    for (int c = 0; c < 3; ++c) {
      long long a = s[c][0], b = s[3 + c][0];
      for (int w = 1; w < BB_NT / 32; ++w) {
        a = min(a, s[c][w]);
        b = max(b, s[3 + c][w]);
      }
      const double da = dkey_inv(a), db = dkey_inv(b);
      bbox[8 * sys + c] = da;
      bbox[8 * sys + 3 + c] = db;
      double e = dsub(db, da);
      if (e > E) E = e;
    }
    bbox[8 * sys + 6] = E;
    bbox[8 * sys + 7] = (E > 0.0) ? __ddiv_rn(2097152.0, E) : 0.0;
  }
  if (bad) atomicOr(status, bad);
}

// System of every particle (sorted and input positions of a system coincide:
// systems are packed back to back and the sort keeps them in order).
__global__ void k_fill_psys(int n, int nsys, const int* __restrict__ off, int* __restrict__ psys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = nsys;  // largest s with off[s] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  psys[i] = lo;
}


// ---------------------------------------------------------------------------
// Morton keys: 21 bits per axis, x highest (bit 3b+2 = x_b, 3b+1 = y_b, 3b = z_b)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// floor((x - mn) scale) clamped to [0, 2^21 - 1]: the conversion rounds
// down (exactly floor, saturating out of range), the clamp is on integers.
__device__ __forceinline__ uint64_t quantise(double x, double mn, double scale) {
  const long long v = __double2ll_rd(dmul(dsub(x, mn), scale));
  return (uint64_t)min(max(v, 0LL), 2097151LL);
}

__global__ void k_morton(const double* __restrict__ pos, int n, const double* __restrict__ bbox0,
                         const int* __restrict__ psys, uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* bbox = bbox0 + (psys ? 8 * psys[i] : 0);
  double scale = bbox[7];
  uint64_t kx = quantise(pos[3 * (int64_t)i], bbox[0], scale);
  uint64_t ky = quantise(pos[3 * (int64_t)i + 1], bbox[1], scale);
  uint64_t kz = quantise(pos[3 * (int64_t)i + 2], bbox[2], scale);
  keys[i] = (spread3(kx) << 2) | (spread3(ky) << 1) | spread3(kz);
  idx[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// S2: stable LSD radix sort of (key, index), 8-bit digits.  Sets below 2^30
// particles take the onesweep passes further down (k_rs_upfront,
// k_rs_onesweep); larger ones the reduce-then-scan passes here (per-tile
// histograms, a scan over them, the scatter).
// ---------------------------------------------------------------------------
#define RS_NT 256
#define RS_ITEMS 4
#define RS_TILE (RS_NT * RS_ITEMS)
#define RS_WARPS (RS_NT / 32)

// Digit of element i: bits [shift, shift+8) of its key, or of its system id
// (psys of the carried input index) for the final passes of a batch sort.
__device__ __forceinline__ unsigned rs_digit(const uint64_t* keys, const uint32_t* vals, const int* psys, int64_t i,
                                             int shift) {
  if (psys) return ((unsigned)psys[vals[i]] >> shift) & 255u;
  return (unsigned)(keys[i] >> shift) & 255u;
}

__global__ void __launch_bounds__(RS_NT) k_rs_hist(const uint64_t* __restrict__ keys,
                                                   const uint32_t* __restrict__ vals, const int* __restrict__ psys,
                                                   int n, int shift, uint32_t* __restrict__ counts, int ntiles) {
  __shared__ uint32_t hw[RS_WARPS][256];
  const int warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_NT) (&hw[0][0])[t] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; ++k) {
    int64_t i = base + (int64_t)k * RS_NT + threadIdx.x;
    if (i < n) atomicAdd(&hw[warp][rs_digit(keys, vals, psys, i, shift)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_NT) {
    uint32_t s = 0;
    for (int w = 0; w < RS_WARPS; ++w) s += hw[w][d];
    counts[(int64_t)d * ntiles + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(RS_NT) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                      const int* __restrict__ psys, int n, int shift,
                                                      const uint32_t* __restrict__ offs, int ntiles) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wc[RS_WARPS][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < 256; d += RS_NT) run[d] = offs[(int64_t)d * ntiles + blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_NT) (&wc[0][0])[t] = 0;
    __syncthreads();
    int64_t i = base + (int64_t)r * RS_NT + threadIdx.x;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0ull;
    int d = valid ? (int)rs_digit(kin, vin, psys, i, shift) : 256;
    unsigned peers = __match_any_sync(SFMM_FULL, d);
    unsigned rank = __popc(peers & lanemask_lt());
    bool leader = (__ffs(peers) - 1) == lane;
    if (valid && leader) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t s = run[threadIdx.x];
      for (int w = 0; w < RS_WARPS; ++w) {
        uint32_t cnt = wc[w][threadIdx.x];
        wc[w][threadIdx.x] = s;
        s += cnt;
      }
      run[threadIdx.x] = s;
    }
    __syncthreads();
    if (valid) {
      uint32_t dst = wc[warp][d] + rank;
      kout[dst] = key;
      vout[dst] = vin[i];
    }
    __syncthreads();
  }
}

// Onesweep passes (Adinets and Merrill's single-pass radix sort): the digit
// histograms of every pass are counted once up front; each pass is then one
// launch in which a tile (numbered in start order by an atomic counter)
// publishes its digit counts, adds those of all earlier tiles by decoupled
// look-back and scatters its keys stably.  A published word holds a 2-bit
// flag (1: this tile's count, 2: inclusive of all earlier tiles) and a
// 30-bit count.
#define RS_FLAG_AGG (1u << 30)
#define RS_FLAG_INC (2u << 30)
#define RS_COUNT_MASK ((1u << 30) - 1u)
// Bounded wait on an earlier tile's word (it is running, so the wait ends;
// the limit only turns a fault into an error status)
#define RS_SPIN (1 << 22)
#define RS_LOOK 4  // predecessor tiles read per look-back round trip
#ifndef OS_ITEMS
#define OS_ITEMS 8  // keys per thread of a onesweep tile (4, 8, 16 measured: 8 best)
#endif
#define OS_TILE (RS_NT * OS_ITEMS)

__global__ void __launch_bounds__(RS_NT) k_rs_upfront(const uint64_t* __restrict__ keys,
                                                      const uint32_t* __restrict__ vals,
                                                      const int* __restrict__ psys, int n, int nkey,
                                                      int nsysd, uint32_t* __restrict__ gh) {
  __shared__ uint32_t h[12][256];
  const int npass = nkey + nsysd;
  for (int t = threadIdx.x; t < npass * 256; t += RS_NT) (&h[0][0])[t] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * RS_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RS_NT) {
    const uint64_t k = keys[i];
    for (int p = 0; p < nkey; ++p) atomicAdd(&h[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
    if (nsysd) {
      const unsigned sv = (unsigned)psys[vals[i]];
      for (int p = 0; p < nsysd; ++p) atomicAdd(&h[nkey + p][(sv >> (8 * p)) & 255u], 1u);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < npass * 256; t += RS_NT) {
    const uint32_t v = (&h[0][0])[t];
    if (v) atomicAdd(&gh[t], v);
  }
}

__global__ void __launch_bounds__(RS_NT) k_rs_onesweep(const uint64_t* __restrict__ kin,
                                                       const uint32_t* __restrict__ vin,
                                                       uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                       const int* __restrict__ psys, int n, int shift,
                                                       const uint32_t* __restrict__ ghist, uint32_t* tstat,
                                                       int* tile_ctr, int* status) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wc[RS_WARPS][256];
  __shared__ uint32_t s_tot[256];
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1);
  for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_NT) (&wc[0][0])[t] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t base = (int64_t)tile * OS_TILE;
  // the tile's keys and digits, and its digit counts
  uint64_t key[OS_ITEMS];
  uint32_t val[OS_ITEMS];
  int dig[OS_ITEMS];
#pragma unroll
  for (int r = 0; r < OS_ITEMS; ++r) {
    const int64_t i = base + (int64_t)r * RS_NT + threadIdx.x;
    const bool valid = i < n;
    key[r] = valid ? kin[i] : 0ull;
    val[r] = valid ? vin[i] : 0u;
    dig[r] = valid ? (int)(psys ? (((unsigned)psys[val[r]] >> shift) & 255u) : ((unsigned)(key[r] >> shift) & 255u))
                   : 256;
    if (valid) atomicAdd(&wc[warp][dig[r]], 1u);
  }
  __syncthreads();
  // publish, look back, and the digit's start in the output
  if (threadIdx.x < 256) {
    const int d = threadIdx.x;
    uint32_t cnt = 0;
    for (int w = 0; w < RS_WARPS; ++w) cnt += wc[w][d];
    volatile uint32_t* st = tstat;
    st[(int64_t)tile * 256 + d] = (tile == 0 ? RS_FLAG_INC : RS_FLAG_AGG) | cnt;
    // look back RS_LOOK tiles per round trip: their words are read at once
    // and taken in order up to the first inclusive one (done) or the first
    // not yet published (read again from there); tile 0 is always inclusive
    uint32_t excl = 0;
    int t = tile - 1, spins = 0;
    while (t >= 0) {
      uint32_t w[RS_LOOK];
#pragma unroll
      for (int k = 0; k < RS_LOOK; ++k) w[k] = (t - k >= 0) ? st[(int64_t)(t - k) * 256 + d] : 0u;
      int k = 0;
      bool done = false;
#pragma unroll
      for (int q = 0; q < RS_LOOK; ++q) {
        if (k == q && t - q >= 0 && (w[q] & ~RS_COUNT_MASK) != 0u) {
          excl += w[q] & RS_COUNT_MASK;
          if ((w[q] & ~RS_COUNT_MASK) == RS_FLAG_INC) done = true;
          else k = q + 1;
        }
      }
      if (done) break;
      t -= k;
      if (k == 0 && ++spins > RS_SPIN) {
        set_status(status, SFMM_ST_INTERNAL);
        break;
      }
    }
    if (tile > 0) st[(int64_t)tile * 256 + d] = RS_FLAG_INC | (excl + cnt);
    s_tot[d] = ghist[d];
    run[d] = excl;
  }
  __syncthreads();
  // exclusive scan of the pass's digit totals (the digit starts), added in
  if (threadIdx.x < 256) {
    uint32_t v = s_tot[threadIdx.x];
    // warp-level inclusive scan, then across the 8 warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(SFMM_FULL, v, o);
      if (lane >= o) v += y;
    }
    wc[0][threadIdx.x] = v;  // inclusive within the warp
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += wc[0][32 * w + 31];
    run[threadIdx.x] += pre + wc[0][threadIdx.x] - s_tot[threadIdx.x];
  }
  __syncthreads();
  // stable scatter in input order: item r of every thread, warp by warp
#pragma unroll
  for (int r = 0; r < OS_ITEMS; ++r) {
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_NT) (&wc[0][0])[t] = 0;
    __syncthreads();
    const int d = dig[r];
    const unsigned peers = __match_any_sync(SFMM_FULL, d);
    const unsigned rank = __popc(peers & lanemask_lt());
    const bool leader = (__ffs(peers) - 1) == lane;
    if (d < 256 && leader) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t s = run[threadIdx.x];
      for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = wc[w][threadIdx.x];
        wc[w][threadIdx.x] = s;
        s += c;
      }
      run[threadIdx.x] = s;
    }
    __syncthreads();
    if (d < 256) {
      const uint32_t dst = wc[warp][d] + rank;
      if (dst < (uint32_t)n) {  // always, unless a look-back gave up (status set)
        kout[dst] = key[r];
        vout[dst] = val[r];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Gather the sorted particles (float64 SoA)
// ---------------------------------------------------------------------------
// FP32 softening record of a particle: {1/h, (2h)^2, 2h rounded up, 0}.
// The first two in FP32 from h rounded to FP32 (within an ulp or two of the
// FP32 roundings of the exact values: the FP32 form's M4 kernels and its
// inside-the-kernel test take them as they are); 2h rounded up from the
// FP64 value, since the near-field candidate test needs a bound.
__device__ __forceinline__ float4 softening_record(double h) {
  const float hf = __double2float_rn(h);
  const float h2 = 2.0f * hf;
  return make_float4(__frcp_rn(hf), h2 * h2, __double2float_ru(2.0 * h), 0.0f);
}

// Sorted particles (and their softening records, formed while the gather
// waits on its loads).
__global__ void k_gather(const double* __restrict__ pos, const double* __restrict__ mass,
                         const double* __restrict__ h, const uint32_t* __restrict__ idx, int n,
                         double* __restrict__ px, double* __restrict__ py, double* __restrict__ pz,
                         double* __restrict__ pm, double* __restrict__ ph, int* __restrict__ perm,
                         float4* __restrict__ phh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t j = idx[i];
  px[i] = pos[3 * j];
  py[i] = pos[3 * j + 1];
  pz[i] = pos[3 * j + 2];
  pm[i] = mass[j];
  const double hj = h[j];
  ph[i] = hj;
  perm[i] = (int)j;
  phh[i] = softening_record(hj);
}

// ---------------------------------------------------------------------------
// S3: binary radix tree over the augmented keys (key, sorted position)
// (Karras 2012 construction; split at the highest differing bit)
// ---------------------------------------------------------------------------
// Common prefix length of the augmented keys (system, Morton key, position
// within the system) of sorted elements i and j (-1 outside [0, n)).
struct SysView {
  const int* psys;  // null: one system
  const int* off;
};
__device__ __forceinline__ int prefix_len(const uint64_t* __restrict__ keys, int n, int i, int64_t j,
                                          const SysView sv) {
  if (j < 0 || j >= n) return -1;
  int si = 0, sj = 0, oi = 0;
  if (sv.psys) {
    si = sv.psys[i];
    sj = sv.psys[j];
    if (si != sj) return __clz(si ^ sj);
    oi = sv.off[si];
  }
  uint64_t a = keys[i], b = keys[j];
  if (a != b) return 32 + __clzll((long long)(a ^ b));
  return 96 + __clz((i - oi) ^ ((int)j - oi));
}

// Children encoding: >= 0 internal node index, < 0 leaf (particle) ~index.
__global__ void k_radix_tree(const uint64_t* __restrict__ keys, int n, const SysView sv, int* __restrict__ kl,
                             int* __restrict__ kr, int* __restrict__ kf, int* __restrict__ kla,
                             int* __restrict__ par_int, int* __restrict__ par_leaf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (prefix_len(keys, n, i, i + 1, sv) - prefix_len(keys, n, i, i - 1, sv)) >= 0 ? 1 : -1;
  int dmin = prefix_len(keys, n, i, (int64_t)i - d, sv);
  int64_t lmax = 2;
  while (prefix_len(keys, n, i, i + lmax * d, sv) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (prefix_len(keys, n, i, i + (l + t) * d, sv) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = prefix_len(keys, n, i, j, sv);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (prefix_len(keys, n, i, i + (s + t) * d, sv) > dnode) s += t;
  } while (t > 1);
  int gamma = (int)(i + s * d + (d < 0 ? -1 : 0));
  int first = (int)min((int64_t)i, j), last = (int)max((int64_t)i, j);
  int left = (first == gamma) ? ~gamma : gamma;
  int right = (last == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  kl[i] = left;
  kr[i] = right;
  kf[i] = first;
  kla[i] = last;
  if (left >= 0) par_int[left] = i; else par_leaf[~left] = i;
  if (right >= 0) par_int[right] = i; else par_leaf[~right] = i;
  if (i == 0) par_int[0] = -1;
}

// A node is split (internal) when it holds more than its system's leaf size
// or particles of more than one system.
struct LeafRule {
  const int* psys;  // null: one system
  const int* lsz;
  int leaf_size;
  __device__ __forceinline__ bool splits(int first, int last) const {
    if (psys) {
      const int sf = psys[first];
      if (sf != psys[last]) return true;
      return last - first + 1 > lsz[sf];
    }
    return last - first + 1 > leaf_size;
  }
};

// Tree nodes of the collapsed tree: the root and every child of a node with
// more than leaf_size particles.  chain[f] counts the tree nodes whose range
// starts at f (a nested chain: each is the left child of the previous).
__global__ void k_mark(int n, const LeafRule lr, const int* __restrict__ kf, const int* __restrict__ kla,
                       const int* __restrict__ par_int, const int* __restrict__ par_leaf,
                       uint32_t* __restrict__ chain) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n - 1) {
    int p = par_int[i];
    bool tree = (i == 0) || lr.splits(kf[p], kla[p]);
    if (tree) atomicAdd(&chain[kf[i]], 1u);
  }
  if (i < n) {
    int p = par_leaf[i];
    bool tree = lr.splits(kf[p], kla[p]);
    if (tree) atomicAdd(&chain[i], 1u);
  }
}

// Pre-order index = (# tree nodes starting before) + (# tree ancestors
// starting at the same particle).
__global__ void k_preorder(int n, const LeafRule lr, const int* __restrict__ kf, const int* __restrict__ kla,
                           const int* __restrict__ par_int, const int* __restrict__ par_leaf,
                           const uint32_t* __restrict__ base, int* __restrict__ pre_int,
                           int* __restrict__ pre_leaf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n - 1) {
    int p = par_int[i];
    bool tree = (i == 0) || lr.splits(kf[p], kla[p]);
    int v = -1;
    if (tree) {
      int f = kf[i], r = 0, u = i;
      while (u != 0) {
        int q = par_int[u];
        if (kf[q] != f) break;
        ++r;
        u = q;
      }
      v = (int)base[f] + r;
    }
    pre_int[i] = v;
  }
  if (i < n) {
    int p = par_leaf[i];
    bool tree = lr.splits(kf[p], kla[p]);
    int v = -1;
    if (tree) {
      int r = 0, u = p;
      while (u >= 0 && kf[u] == i) {
        ++r;
        u = (u == 0) ? -1 : par_int[u];
      }
      v = (int)base[i] + r;
    }
    pre_leaf[i] = v;
  }
}

__global__ void k_fill_nodes(int n, const LeafRule lr, const int* __restrict__ kl, const int* __restrict__ kr,
                             const int* __restrict__ kf, const int* __restrict__ kla,
                             const int* __restrict__ par_int, const int* __restrict__ par_leaf,
                             const int* __restrict__ pre_int, const int* __restrict__ pre_leaf,
                             int* __restrict__ nfirst, int* __restrict__ ncount, int* __restrict__ nright,
                             int* __restrict__ nparent, uint32_t* __restrict__ lstart, int* __restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n - 1) {
    int v = pre_int[i];
    if (v >= 0) {
      int cnt = kla[i] - kf[i] + 1;
      nfirst[v] = kf[i];
      ncount[v] = cnt;
      nparent[v] = (i == 0) ? -1 : pre_int[par_int[i]];
      if (!lr.splits(kf[i], kla[i])) {
        nright[v] = -1;
        lstart[kf[i]] = 1u;
      } else {
        int L = kl[i], R = kr[i];
        int pl = (L >= 0) ? pre_int[L] : pre_leaf[~L];
        int pr = (R >= 0) ? pre_int[R] : pre_leaf[~R];
        if (pl != v + 1) atomicOr(status, SFMM_ST_INTERNAL);
        nright[v] = pr;
      }
    }
  }
  if (i < n) {
    int v = pre_leaf[i];
    if (v >= 0) {
      nfirst[v] = i;
      ncount[v] = 1;
      nright[v] = -1;
      nparent[v] = pre_int[par_leaf[i]];
      lstart[i] = 1u;
    }
  }
}

// Walk parent of every node: the parent, -1 at a system's root, -2 for nodes
// spanning several systems (never walked); the root node of each system.
__global__ void k_sysroots(const uint32_t* __restrict__ counts, const int* __restrict__ psys, const int* __restrict__ nfirst,
                           const int* __restrict__ ncount, const int* __restrict__ nparent, int* __restrict__ wparent,
                           int* __restrict__ sys_root) {
  const int nn = (int)counts[0];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
    const int f = nfirst[v], l = f + ncount[v] - 1;
    const int p = nparent[v];
    if (!psys) {
      wparent[v] = p;
      if (p < 0) sys_root[0] = v;
      continue;
    }
    const int sv = psys[f];
    if (sv != psys[l]) {
      wparent[v] = -2;
      continue;
    }
    const bool root = (p < 0) || (psys[nfirst[p]] != psys[nfirst[p] + ncount[p] - 1]);
    wparent[v] = root ? -1 : p;
    if (root) sys_root[sv] = v;
  }
}

// Leaf numbers: lstart holds the exclusive scan over particles of the
// leaf-start flags, so the leaves before node v in pre-order are those that
// start before its first particle: leaf_index[v] = lstart[first[v]] (a
// leaf's own number).  Records the leaves, and clears each node's arrival
// flag and size bits for the passes that follow.
__global__ void k_leaf_list(const uint32_t* __restrict__ counts, const int* __restrict__ nfirst,
                            const int* __restrict__ nright, const uint32_t* __restrict__ lstart,
                            uint32_t* __restrict__ leaf_index, int* __restrict__ leaf_node, int* __restrict__ flags,
                            unsigned long long* __restrict__ l2bits) {
  const int nn = (int)counts[0];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
    const uint32_t q = lstart[nfirst[v]];
    leaf_index[v] = q;
    if (nright[v] < 0) leaf_node[q] = v;
    flags[v] = 0;
    l2bits[v] = 0ull;
  }
}

// ---------------------------------------------------------------------------
// S4 geometry: leaf mass / centre of mass / h_max (one warp per leaf), then
// bottom-up for internal nodes; particle -> leaf node map.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dadd(v, __shfl_xor_sync(SFMM_FULL, v, o));
  return v;
}

// The larger of two non-negative doubles, compared as bit patterns (exact).
__device__ __forceinline__ double dmax_pos(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

// A node's moments: FP64 (the FP64 form; FP32 rows rounded from them) or
// FP32 only (the FP32 form, whose walk reads nothing else; the monopole is
// the FP64 mass, rounded once).
template <int NQ, typename QT>
__device__ __forceinline__ void store_moments(int v, QT (&q)[NQ], double M, double* __restrict__ Qd,
                                              float* __restrict__ Qf) {
  constexpr int NQS = (NQ + 3) & ~3;
  if constexpr (std::is_same<QT, double>::value) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) Qd[(int64_t)v * NQ + k] = q[k];
  } else {
    q[0] = __double2float_rn(M);
  }
#pragma unroll
  for (int k = 0; k < NQS; ++k) Qf[(int64_t)v * NQS + k] = (k < NQ) ? (float)q[k] : 0.0f;
}

// A child's moments, read through L2 (written by another thread of the same
// launch in the climb).
template <int NQ, typename QT>
__device__ __forceinline__ void load_moments(int u, QT (&q)[NQ], const double* Qd, const float* Qf) {
  constexpr int NQS = (NQ + 3) & ~3;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    if constexpr (std::is_same<QT, double>::value) q[k] = __ldcg(&Qd[(int64_t)u * NQ + k]);
    else q[k] = __ldcg(&Qf[(int64_t)u * NQS + k]);
  }
}

// One thread per leaf (the FP64 sums of a leaf are short; warp reductions in
// FP64 would cost more than the sums themselves).
// P >= 0: also the leaf's scaled moments of order P about its centre of mass
// (P2M, Eq. massmom) in FP64 and their FP32 copy; P < 0: geometry only.
template <int P, typename QT>
__global__ void k_leaf_geom(const uint32_t* __restrict__ counts, const int* __restrict__ leaf_node, const int* __restrict__ nfirst,
                            const int* __restrict__ ncount, const double* __restrict__ px,
                            const double* __restrict__ py, const double* __restrict__ pz,
                            const double* __restrict__ pm, const double* __restrict__ ph,
                            double* __restrict__ ncx, double* __restrict__ ncy, double* __restrict__ ncz,
                            double* __restrict__ nmass, double* __restrict__ nhmax, int* __restrict__ pnode,
                            int* __restrict__ nlu, double* __restrict__ extv, int* __restrict__ exti,
                            float4* __restrict__ prel, float4* __restrict__ geo_hi, float4* __restrict__ geo_lo,
                            double* __restrict__ Qd, float* __restrict__ Qf, int nqs) {
  const int nleaves = (int)counts[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nleaves; q += gridDim.x * blockDim.x) {
    const int v = leaf_node[q];
    const int f = nfirst[v], cnt = ncount[v];
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, hm = 0.0;
    // extreme particles per axis (min x, y, z, max x, y, z; first one on ties)
    double ev[6] = {px[f], py[f], pz[f], px[f], py[f], pz[f]};
    long long ek[6];
  #pragma unroll
    for (int c = 0; c < 6; ++c) ek[c] = dkey(ev[c]);
    int ei[6] = {f, f, f, f, f, f};
    for (int i = f; i < f + cnt; ++i) {
      const double m = pm[i];
      M = dadd(M, m);
      sx = dadd(sx, dmul(m, px[i]));
      sy = dadd(sy, dmul(m, py[i]));
      sz = dadd(sz, dmul(m, pz[i]));
      hm = dmax_pos(hm, ph[i]);
      pnode[i] = v;
      const double xc[3] = {px[i], py[i], pz[i]};
  #pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long k = dkey(xc[c]);
        if (k < ek[c]) { ek[c] = k; ev[c] = xc[c]; ei[c] = i; }
        if (k > ek[3 + c]) { ek[3 + c] = k; ev[3 + c] = xc[c]; ei[3 + c] = i; }
      }
    }
  #pragma unroll
    for (int c = 0; c < 6; ++c) {
      extv[6 * (size_t)v + c] = ev[c];
      exti[6 * (size_t)v + c] = ei[c];
    }
    nmass[v] = M;
    // the leaf centre as the oracle forms it (sums of rounded products, one
    // correctly rounded division per axis): degenerate leaves (coincident
    // particles) then have exactly its zero offsets
    const double cx = __ddiv_rn(sx, M), cy = __ddiv_rn(sy, M), cz = __ddiv_rn(sz, M);
    ncx[v] = cx;
    ncy[v] = cy;
    ncz[v] = cz;
    store_centre_df(v, cx, cy, cz, geo_hi, geo_lo);
    nhmax[v] = hm;
    nlu[v] = 1;
    // the particles' FP32 records (offsets from the leaf centre, mass) and,
    // P >= 0, the leaf's moments from the same offsets
    constexpr int NQ = (P >= 0) ? MomOps<(P >= 0 ? P : 0)>::NQ : 1;
    QT acc[NQ];
  #pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = QT(0);
    for (int i = f; i < f + cnt; ++i) {
      const double dx = dsub(px[i], cx), dy = dsub(py[i], cy), dz = dsub(pz[i], cz);
      const float fx = __double2float_rn(dx), fy = __double2float_rn(dy), fz = __double2float_rn(dz);
      const float fm = __double2float_rn(pm[i]);
      prel[i] = make_float4(fx, fy, fz, fm);
      if constexpr (P >= 0) {
        QT mono[NQ];
        if constexpr (std::is_same<QT, float>::value) MomOps<P>::mono(fx, fy, fz, mono);
        else MomOps<P>::mono(dx, dy, dz, mono);
        const QT m = std::is_same<QT, float>::value ? (QT)fm : (QT)pm[i];
  #pragma unroll
        for (int k = 0; k < NQ; ++k) acc[k] = fma(m, mono[k], acc[k]);
      }
    }
    if constexpr (P >= 0) store_moments<NQ>(v, acc, M, Qd, Qf);
  }
}

// Node v from its children L = v + 1 and R: centre of mass, moments (P >= 0:
// both children's translated to v's centre, Eq. massmomtrans), h_max, leaf
// count and the axis-extreme particles (the left child's on ties).  The
// children's records are read through L2: another thread of this launch may
// have written them.
template <int P, typename QT>
__device__ __forceinline__ void upward_node(int v, int R, double* ncx, double* ncy, double* ncz, double* nmass,
                                            double* nhmax, int* nlu, double* extv, int* exti, double* Qd,
                                            float* Qf) {
  const int L = v + 1;
  // every load first: the stores below may alias them as far as the
  // compiler knows, and loads left after a store would wait for the work
  // before it, one L2 round trip per group
  const double mL = __ldcg(&nmass[L]), mR = __ldcg(&nmass[R]);
  const double cLx = __ldcg(&ncx[L]), cLy = __ldcg(&ncy[L]), cLz = __ldcg(&ncz[L]);
  const double cRx = __ldcg(&ncx[R]), cRy = __ldcg(&ncy[R]), cRz = __ldcg(&ncz[R]);
  const double hL = __ldcg(&nhmax[L]), hR = __ldcg(&nhmax[R]);
  const int uL = __ldcg(&nlu[L]), uR = __ldcg(&nlu[R]);
  double ea[6], eb[6];
  int ia[6], ib[6];
  #pragma unroll
  for (int c = 0; c < 6; ++c) {
    ea[c] = __ldcg(&extv[6 * (size_t)L + c]);
    eb[c] = __ldcg(&extv[6 * (size_t)R + c]);
    ia[c] = __ldcg(&exti[6 * (size_t)L + c]);
    ib[c] = __ldcg(&exti[6 * (size_t)R + c]);
  }
  constexpr int NQ = (P >= 0) ? MomOps<(P >= 0 ? P : 0)>::NQ : 1;
  QT qL[NQ], qR[NQ];
  if constexpr (P >= 0) {
    load_moments<NQ>(L, qL, Qd, Qf);
    load_moments<NQ>(R, qR, Qd, Qf);
  }
  const double M = dadd(mL, mR);
  // one reciprocal per node (GB300's FP64 pipe is narrow): the centre is
  // within rounding of the quotient, like the oracle's own sum
  const double iM = recip_pos(M);
  const double cx = dmul(dadd(dmul(mL, cLx), dmul(mR, cRx)), iM);
  const double cy = dmul(dadd(dmul(mL, cLy), dmul(mR, cRy)), iM);
  const double cz = dmul(dadd(dmul(mL, cLz), dmul(mR, cRz)), iM);
  ncx[v] = cx;
  ncy[v] = cy;
  ncz[v] = cz;
  if constexpr (P >= 0) {
    QT qp[NQ];
  #pragma unroll
    for (int k = 0; k < NQ; ++k) qp[k] = QT(0);
    QT g[NQ];
    MomOps<P>::mono((QT)(cLx - cx), (QT)(cLy - cy), (QT)(cLz - cz), g);
    MomOps<P>::m2m(g, qL, qp);
    MomOps<P>::mono((QT)(cRx - cx), (QT)(cRy - cy), (QT)(cRz - cz), g);
    MomOps<P>::m2m(g, qR, qp);
    store_moments<NQ>(v, qp, M, Qd, Qf);
  }
  nmass[v] = M;
  nhmax[v] = dmax_pos(hL, hR);
  nlu[v] = uL + uR;
  #pragma unroll
  for (int c = 0; c < 6; ++c) {
    const long long ka = dkey(ea[c]), kb = dkey(eb[c]);
    const bool right = (c < 3) ? (kb < ka) : (kb > ka);
    extv[6 * (size_t)v + c] = right ? eb[c] : ea[c];
    exti[6 * (size_t)v + c] = right ? ib[c] : ia[c];
  }
}

// Bottom-up: the second child to finish computes its parent.  The climb's
// cost is its longest chain of dependent arrivals (one device-scope fence,
// atomic and round of loads per level: about 30 levels on a Plummer sphere
// of 10^6), so the node body issues all its loads at once.  (Measured on
// GB300: computing the top of the tree -- the ~1500 nodes of more than 10^3
// particles, 23 levels deep -- level by level in one block after a climb
// that stops below it was slower, 0.18 against 0.13 ms.)
template <int P, typename QT>
__global__ void k_upward(const uint32_t* __restrict__ counts, const int* __restrict__ leaf_node, const int* __restrict__ nparent,
                         const int* __restrict__ nright, double* ncx, double* ncy, double* ncz, double* nmass,
                         double* nhmax, int* nlu, int* flags, double* extv, int* exti, double* Qd, float* Qf,
                         int nqs) {
  const int nleaves = (int)counts[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nleaves; q += gridDim.x * blockDim.x) {
    int v = nparent[leaf_node[q]];
    while (v >= 0) {
      // the tree's links (written by earlier launches) load ahead of the arrival
      const int R = nright[v], up = nparent[v];
      {
        // release this child's records, acquire the sibling's
        cuda::atomic_ref<int, cuda::thread_scope_device> arrive(flags[v]);
        if (arrive.fetch_add(1, cuda::memory_order_acq_rel) == 0) break;
      }
      upward_node<P, QT>(v, R, ncx, ncy, ncz, nmass, nhmax, nlu, extv, exti, Qd, Qf);
      v = up;
    }
  }
}

// Exact node sizes l_v = max over the node's particles of |x_i - s_v| (the
// squared distance rounded as written, then one square root).  Most
// (particle, ancestor) pairs cannot hold the maximum, so only candidates are
// evaluated:
//  * LB(v): the largest distance from s_v among the node's six axis-extreme
//    particles -- real particles, so LB(v) <= l_v;
//  * a leaf L (exact size l_L) can hold the maximum of an ancestor v only if
//    l_L + |s_L - s_v| >= LB(v); the test uses margins of 1e-12, far above
//    the rounding of these few operations, so a skipped particle's distance
//    is strictly below LB(v);
//  * every particle then visits its ancestors and evaluates only those its
//    leaf is a candidate for.
__device__ __forceinline__ double exact_d2(double x, double y, double z, double cx, double cy, double cz) {
  const double dx = dsub(x, cx), dy = dsub(y, cy), dz = dsub(z, cz);
  return dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
}

// Upper bound on the error of an FP32 distance assembled from double-float
// centre differences (each within a few units of 2^-24 of its value, the
// centres within 2^-48 of theirs) and FP32 offsets: generous by two orders.
__device__ __forceinline__ float df_dist_err(float ox, float oy, float oz, float4 a, float4 b) {
  return 2e-6f * (fabsf(ox) + fabsf(oy) + fabsf(oz)) +
         1e-13f * (fabsf(a.x) + fabsf(a.y) + fabsf(a.z) + fabsf(b.x) + fabsf(b.y) + fabsf(b.z));
}

// An internal node's centre as double-float walk records (the leaf pass
// wrote the leaves'), and LB(v) in FP32, rounded down: the largest distance
// from s_v among the node's six axis-extreme particles, each assembled from
// the particle's FP32 offset in its leaf and the double-float difference of
// the leaf's and v's centres, less that sum's error bound (so LB(v) never
// exceeds the real distance, nor, hence, l_v), in the w field of v's record.
// A thread reads the records of leaves only, besides its own node's.
__global__ void k_node_lb(const uint32_t* __restrict__ counts, const int* __restrict__ wparent,
                          const int* __restrict__ nright, const int* __restrict__ exti,
                          const int* __restrict__ pnode, const double* __restrict__ ncx,
                          const double* __restrict__ ncy, const double* __restrict__ ncz,
                          const float4* __restrict__ prel, float4* __restrict__ geo_hi,
                          float4* __restrict__ geo_lo) {
  const int nn = (int)counts[0];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
    float4 hv, ov;
    if (nright[v] >= 0) {
      float xh, xl, yh, yl, zh, zl;
      split_double(ncx[v], xh, xl);
      split_double(ncy[v], yh, yl);
      split_double(ncz[v], zh, zl);
      hv = make_float4(xh, yh, zh, 0.0f);
      ov = make_float4(xl, yl, zl, 0.0f);
      geo_lo[v] = ov;
    } else {
      hv = geo_hi[v];
      ov = geo_lo[v];
    }
    float lbv = 0.0f;
    if (wparent[v] != -2) {
  #pragma unroll
      for (int c = 0; c < 6; ++c) {
        const int e = exti[6 * (size_t)v + c];
        const int L = pnode[e];
        const float4 r = prel[e], hL = geo_hi[L], oL = geo_lo[L];
        const float ox = df_diff(hL.x, oL.x, hv.x, ov.x), oy = df_diff(hL.y, oL.y, hv.y, ov.y),
                    oz = df_diff(hL.z, oL.z, hv.z, ov.z);
        const float dx = r.x + ox, dy = r.y + oy, dz = r.z + oz;
        const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        const float err = 2e-6f * (fabsf(r.x) + fabsf(r.y) + fabsf(r.z)) + df_dist_err(ox, oy, oz, hL, hv);
        lbv = fmaxf(lbv, (d - err) * (1.0f - 1e-6f));
      }
    }
    hv.w = lbv;
    if (nright[v] >= 0) geo_hi[v] = hv;
    else reinterpret_cast<float*>(&geo_hi[v])[3] = lbv;  // only w: other threads read a leaf's centre
  }
}

// Thread per leaf: the leaf's exact size, and the ancestors it is a
// candidate for (a short list; a leaf with more tries every ancestor).
#define SIZE_LIST 8
__global__ void k_size_leaf(const uint32_t* __restrict__ counts, const int* __restrict__ leaf_node, const int* __restrict__ nfirst,
                            const int* __restrict__ ncount, const int* __restrict__ wparent,
                            const double* __restrict__ px, const double* __restrict__ py,
                            const double* __restrict__ pz, const double* __restrict__ ncx,
                            const double* __restrict__ ncy, const double* __restrict__ ncz,
                            const float4* __restrict__ geo_hi, const float4* __restrict__ geo_lo,
                            const float4* __restrict__ prel, unsigned long long* __restrict__ l2bits,
                            int* __restrict__ cand) {
  const int nleaves = (int)counts[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nleaves; q += gridDim.x * blockDim.x) {
    const int L = leaf_node[q];
    const int f = nfirst[L], cnt = ncount[L];
    const double cx = ncx[L], cy = ncy[L], cz = ncz[L];
    // the particles' FP32 offsets give their squared distances within 2^-21
    // (relative): only those within 4e-6 of the FP32 maximum can hold the
    // exact maximum, and only they are evaluated in FP64 (one, as a rule);
    // offsets too small or too large for that bound take every particle
    float best = -1.0f;
    int bi = f;
    for (int i = f; i < f + cnt; ++i) {
      const float4 r = prel[i];
      const float d2 = fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z));
      if (d2 > best) {
        best = d2;
        bi = i;
      }
    }
    double l2 = exact_d2(px[bi], py[bi], pz[bi], cx, cy, cz);
    const float thr = (best > 1e-30f && best < 1e30f) ? best * (1.0f - 4e-6f) : -1.0f;
    for (int i = f; i < f + cnt; ++i) {
      const float4 r = prel[i];
      if (i != bi && fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z)) >= thr)
        l2 = fmax(l2, exact_d2(px[i], py[i], pz[i], cx, cy, cz));
    }
    l2bits[L] = (unsigned long long)__double_as_longlong(l2);
    const float lL = __double2float_ru(__dsqrt_rn(l2));
    const float4 hL = geo_hi[L], oL = geo_lo[L];
    // an ancestor v is skipped when every particle of the leaf is certainly
    // closer to s_v than LB(v) (a real particle's distance): |s_L - s_v| + l_L,
    // with its error bound and one more relative margin for the FP32 sums,
    // below LB(v) rounded down.  The others are listed (count, then ids);
    // more than SIZE_LIST - 1 of them: count -1, and every ancestor is tried
    int* const lst = cand + SIZE_LIST * (size_t)q;
    int nc = 0;
    for (int v = (wparent[L] >= 0) ? wparent[L] : -1; v >= 0; v = wparent[v]) {
      const float4 hv = geo_hi[v], ov = geo_lo[v];
      const float dx = df_diff(hL.x, oL.x, hv.x, ov.x), dy = df_diff(hL.y, oL.y, hv.y, ov.y),
                  dz = df_diff(hL.z, oL.z, hv.z, ov.z);
      const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      const float reach = (d + df_dist_err(dx, dy, dz, hL, hv) + lL) * (1.0f + 1e-6f);
      if (!(reach < hv.w) && nc >= 0) {
        if (nc < SIZE_LIST - 1) lst[1 + nc++] = v;
        else nc = -1;
      }
    }
    lst[0] = nc;
  }
}

// Thread per particle: candidate ancestors only.  A (particle, ancestor)
// pair that passes the FP32 test goes to its warp's queue; every 32 queued
// pairs are evaluated exactly, one per lane (FP64 work costs per warp
// instruction, whatever the active lanes), and lanes at the same node
// combine their squared distances, one atomic max per group.
#define SIZE_NT 256
__device__ __forceinline__ void size_flush(const int2* q, int cnt, const double* __restrict__ px,
                                           const double* __restrict__ py, const double* __restrict__ pz,
                                           const double* __restrict__ ncx, const double* __restrict__ ncy,
                                           const double* __restrict__ ncz, unsigned long long* __restrict__ l2bits) {
  const int lane = threadIdx.x & 31;
  const bool on = lane < cnt;
  const int2 e = on ? q[lane] : make_int2(0, -1);
  const unsigned act = __ballot_sync(SFMM_FULL, on);
  if (on) {
    const int i = e.x, v = e.y;
    const double d2 = exact_d2(px[i], py[i], pz[i], ncx[v], ncy[v], ncz[v]);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d2);
    const unsigned grp = __match_any_sync(act, v);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const unsigned mhi = __reduce_max_sync(grp, hi);
    const unsigned mlo = __reduce_max_sync(grp, hi == mhi ? lo : 0u);
    if ((__ffs(grp) - 1) == lane) atomicMax(&l2bits[v], ((unsigned long long)mhi << 32) | mlo);
  }
}

__global__ void __launch_bounds__(SIZE_NT) k_size(int n, const double* __restrict__ px, const double* __restrict__ py,
                       const double* __restrict__ pz, const int* __restrict__ pnode,
                       const uint32_t* __restrict__ leaf_index, const int* __restrict__ cand,
                       const int* __restrict__ wparent, const double* __restrict__ ncx,
                       const double* __restrict__ ncy, const double* __restrict__ ncz,
                       const float4* __restrict__ geo_hi, const float4* __restrict__ geo_lo,
                       const float4* __restrict__ prel, unsigned long long* __restrict__ l2bits) {
  __shared__ int2 s_q[SIZE_NT / 32][64];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2* const q = s_q[warp];
  int nq = 0;
  const int* lst = nullptr;
  int nc = 0, L = -1;
  float4 hL = make_float4(0.f, 0.f, 0.f, 0.f), oL = hL, r = hL;
  if (i < n) {
    L = pnode[i];  // the leaf itself was done by k_size_leaf
    lst = cand + SIZE_LIST * (size_t)leaf_index[L];
    nc = lst[0];
    hL = geo_hi[L];
    oL = geo_lo[L];
    r = prel[i];  // x - s_L in FP32
  }
  const float er = 2e-6f * (fabsf(r.x) + fabsf(r.y) + fabsf(r.z));
  // candidate ancestor number k of this particle's leaf: from the list, or
  // (count -1) every ancestor in turn
  int v = (i < n && nc < 0) ? wparent[L] : -1;
  for (int k = 0;; ++k) {
    int u = -1;
    if (i < n) {
      if (nc >= 0) u = (k < nc) ? lst[1 + k] : -1;
      else u = v;
    }
    const unsigned act = __ballot_sync(SFMM_FULL, u >= 0);
    if (act == 0u) break;
    bool want = false;
    if (u >= 0) {
      // certainly closer than LB(u)? then not the maximum: skip the exact test
      const float4 hv = geo_hi[u], ov = geo_lo[u];
      const float ox = df_diff(hL.x, oL.x, hv.x, ov.x), oy = df_diff(hL.y, oL.y, hv.y, ov.y),
                  oz = df_diff(hL.z, oL.z, hv.z, ov.z);
      const float dx = r.x + ox, dy = r.y + oy, dz = r.z + oz;
      const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      want = !((d + er + df_dist_err(ox, oy, oz, hL, hv)) * (1.0f + 1e-6f) < hv.w);
    }
    const unsigned bw = __ballot_sync(SFMM_FULL, want);
    if (want) q[nq + __popc(bw & lanemask_lt())] = make_int2(i, u);
    nq += __popc(bw);
    __syncwarp();
    if (nq >= 32) {
      size_flush(q, 32, px, py, pz, ncx, ncy, ncz, l2bits);
      __syncwarp();
      const int rest = nq - 32;  // carry the pairs beyond the batch to the front
      const int2 c = (lane < rest) ? q[32 + lane] : make_int2(0, 0);
      __syncwarp();
      if (lane < rest) q[lane] = c;
      __syncwarp();
      nq = rest;
    }
    if (nc < 0 && v >= 0) v = wparent[v];  // stops after the system root (-1)
  }
  if (nq > 0) size_flush(q, nq, px, py, pz, ncx, ncy, ncz, l2bits);
}

// Final node records: the sizes and h_max into the w fields (the centres
// were written with the nodes).
__global__ void k_finalize_nodes(const uint32_t* __restrict__ counts, const unsigned long long* __restrict__ l2bits,
                                 const double* __restrict__ nhmax, double* __restrict__ nsize,
                                 float4* __restrict__ geo_hi, float4* __restrict__ geo_lo) {
  const int nn = (int)counts[0];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
    const double l = __dsqrt_rn(__longlong_as_double((long long)l2bits[v]));
    nsize[v] = l;
    reinterpret_cast<float*>(&geo_hi[v])[3] = __double2float_rn(l);
    reinterpret_cast<float*>(&geo_lo[v])[3] = __double2float_rn(nhmax[v]);
  }
}

// FP32 softening records of every particle: {1/h, (2h)^2, 2h rounded up}
// (the offsets and masses come from the leaf pass).
__global__ void k_particles_hh(int n, const double* __restrict__ ph, float4* __restrict__ phh) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  phh[i] = softening_record(ph[i]);
}

// Node depths, and counts[2]: the walkable internal nodes whose children are
// both leaves (the node-queue walk takes both in the parent's warp and
// queues neither, so its queue holds that many items fewer).
__global__ void k_depth(uint32_t* __restrict__ counts, const int* __restrict__ nparent,
                        const int* __restrict__ nright, const int* __restrict__ wparent, int* __restrict__ depth) {
  const int nn = (int)counts[0];
  const int lane = threadIdx.x & 31;
  // warp-aligned strides, so that every lane of a warp runs the same trips
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nn; base += gridDim.x * blockDim.x) {
    const int v = base + lane;
    bool pair = false;
    if (v < nn) {
      int d = 0, u = nparent[v];
      while (u >= 0) {
        ++d;
        u = nparent[u];
      }
      depth[v] = d;
      const int r = nright[v];
      pair = r >= 0 && wparent[v] != -2 && nright[v + 1] < 0 && nright[r] < 0;
    }
    const unsigned b = __ballot_sync(SFMM_FULL, pair);
    if (lane == 0 && b) atomicAdd(&counts[2], (unsigned)__popc(b));
  }
}

// Internal nodes grouped by depth (level lists for the per-node walk), and
// the leaves ordered by depth, shallowest first (the per-node walk processes
// all leaves in one launch; shallow leaves run the longest lowering).
// Warp-aggregated counting: one atomic per (warp, depth) group.
__global__ void k_level_count(int nn, const int* __restrict__ depth, const int* __restrict__ nright,
                              const int* __restrict__ wparent, uint32_t* __restrict__ cnt_int,
                              uint32_t* __restrict__ cnt_leaf) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = v < nn && wparent[v] != -2;
  const int d = ok ? depth[v] : -1;
  const bool leaf = ok && nright[v] < 0;
  const int key = ok ? (2 * d + (leaf ? 1 : 0)) : -1;
  const unsigned grp = __match_any_sync(SFMM_FULL, key);
  if (ok && (__ffs(grp) - 1) == (int)(threadIdx.x & 31))
    atomicAdd(leaf ? &cnt_leaf[d] : &cnt_int[d], (unsigned)__popc(grp));
}

__global__ void k_level_scatter(int nn, const int* __restrict__ depth, const int* __restrict__ nright,
                                const int* __restrict__ wparent, const uint32_t* __restrict__ off_int,
                                const uint32_t* __restrict__ off_leaf, uint32_t* __restrict__ cur_int,
                                uint32_t* __restrict__ cur_leaf, int* __restrict__ level_nodes,
                                int* __restrict__ leaf_order) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nn || wparent[v] == -2) return;
  const int d = depth[v];
  if (nright[v] < 0) leaf_order[off_leaf[d] + atomicAdd(&cur_leaf[d], 1u)] = v;
  else level_nodes[off_int[d] + atomicAdd(&cur_int[d], 1u)] = v;
}

static inline unsigned nblk(int64_t n, int nt) { return (unsigned)((n + nt - 1) / nt); }

int build_levels(sfmm_ctx* c) {
  const int nn = c->nnodes;
  int rc;
  // depth < nn always; counts sized for the worst case.  Layout of level_off:
  // [0, nn + 1) internal-node offsets by depth, [nn + 1, 2 nn + 2) leaf offsets
  const size_t nc = (size_t)nn + 1;
  if ((rc = c->level_off.ensure(sizeof(uint32_t) * 2 * (nc + 1)))) return rc;
  if ((rc = c->level_cur.ensure(sizeof(uint32_t) * 2 * (nc + 1)))) return rc;
  if ((rc = c->level_nodes.ensure(sizeof(int) * (size_t)nn))) return rc;
  if ((rc = c->leaf_order.ensure(sizeof(int) * (size_t)c->nleaves))) return rc;
  cudaStream_t st = c->stream;
  uint32_t* off = c->level_off.as<uint32_t>();
  uint32_t* cur = c->level_cur.as<uint32_t>();
  SFMM_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(uint32_t) * 2 * (nc + 1), st));
  SFMM_CUDA_TRY(cudaMemsetAsync(cur, 0, sizeof(uint32_t) * 2 * (nc + 1), st));
  k_level_count<<<nblk(nn, 256), 256, 0, st>>>(nn, c->ndepth.as<int>(), c->nright.as<int>(), c->wparent.as<int>(),
                                               off, off + nc);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  // totals (walkable internal nodes, leaves) land in the two spare slots
  if ((rc = exclusive_scan_u32(c, off, (int64_t)nc, off + 2 * nc))) return rc;
  if ((rc = exclusive_scan_u32(c, off + nc, (int64_t)nc, off + 2 * nc + 1))) return rc;
  k_level_scatter<<<nblk(nn, 256), 256, 0, st>>>(nn, c->ndepth.as<int>(), c->nright.as<int>(), c->wparent.as<int>(),
                                                 off, off + nc, cur,
                                                 cur + nc, c->level_nodes.as<int>(), c->leaf_order.as<int>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

// Grids of the node- and leaf-indexed passes: their counts stay on the
// device (read by the kernels), so the grids cover the bound and stride.
static inline unsigned node_grid(const sfmm_ctx* c) {
  return std::min<unsigned>(nblk(2 * c->n, 256), 16u * num_sms(c->device));
}
static inline unsigned leaf_grid(const sfmm_ctx* c) {
  return std::min<unsigned>(nblk(c->n, 128), 32u * num_sms(c->device));
}

int compute_depth(sfmm_ctx* c) {
  int rc = c->ndepth.ensure(sizeof(int) * 2 * (size_t)c->n);
  if (rc) return rc;
  SFMM_CUDA_TRY(cudaMemsetAsync(c->d_counts + 2, 0, sizeof(uint32_t), c->stream));
  k_depth<<<node_grid(c), 256, 0, c->stream>>>(c->d_counts, c->nparent.as<int>(), c->nright.as<int>(),
                                               c->wparent.as<int>(), c->ndepth.as<int>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

// ---------------------------------------------------------------------------
// Host orchestration of the build
// ---------------------------------------------------------------------------
// The upward pass climbs from every leaf with acquire-release arrival
// counters (one launch; measured on GB300 faster than one launch per depth
// at 10^6 and at 1.6 x 10^7 particles).

template <int P, typename QT>
static int geom_upward_t(sfmm_ctx* c, int nqs) {
  cudaStream_t st = c->stream;
  k_leaf_geom<P, QT><<<leaf_grid(c), 128, 0, st>>>(
      c->d_counts, c->leaf_node.as<int>(), c->nfirst.as<int>(), c->ncount.as<int>(), c->px.as<double>(),
      c->py.as<double>(), c->pz.as<double>(), c->pm.as<double>(), c->ph.as<double>(), c->ncx.as<double>(),
      c->ncy.as<double>(), c->ncz.as<double>(), c->nmass.as<double>(), c->nhmax.as<double>(), c->pnode.as<int>(),
      c->nlu.as<int>(), c->n_extv.as<double>(), c->n_exti.as<int>(), c->prel.as<float4>(), c->geo_hi.as<float4>(),
      c->geo_lo.as<float4>(), c->Qd.as<double>(), c->Qf.as<float>(), nqs);
  ++c->nlaunch;
  // the second child to finish climbs on (arrival flags cleared by the leaf
  // numbering pass)
  k_upward<P, QT><<<leaf_grid(c), 128, 0, st>>>(c->d_counts, c->leaf_node.as<int>(), c->nparent.as<int>(), c->nright.as<int>(),
                                                 c->ncx.as<double>(), c->ncy.as<double>(), c->ncz.as<double>(),
                                                 c->nmass.as<double>(), c->nhmax.as<double>(), c->nlu.as<int>(),
                                                 c->flags.as<int>(), c->n_extv.as<double>(), c->n_exti.as<int>(),
                                                 c->Qd.as<double>(), c->Qf.as<float>(), nqs);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

// Moments in the context's form: FP32 for the FP32 form, FP64 otherwise.
template <int P>
static int geom_upward(sfmm_ctx* c, int nqs) {
  if (P >= 0 && c->precision == SFMM_FP32) return geom_upward_t<P, float>(c, nqs);
  return geom_upward_t<P, double>(c, nqs);
}

// The per-depth lists of walkable internal nodes and the leaves by depth,
// built on first use: the per-depth walk launches and the one-sided
// symmetric walk run over them; the readiness-queue walk needs only the
// number of walkable nodes.  Their offsets come back to pinned host memory
// (one synchronisation).
#define SFMM_LEVEL_COPY 130  // the tree is at most 128 levels deep
int ensure_levels(sfmm_ctx* c) {
  if (c->levels_ready) return SFMM_OK;
  int rc;
  if ((rc = build_levels(c))) return rc;
  if (!c->h_level_pin && cudaMallocHost(&c->h_level_pin, sizeof(int) * (SFMM_LEVEL_COPY + 1)) != cudaSuccess) {
    c->h_level_pin = nullptr;
    return SFMM_ENOMEM;
  }
  // system, key and position bits distinguish every particle: at most 128
  // levels, so 130 offsets cover every depth
  const int ncopy = (int)std::min<int64_t>((int64_t)c->nnodes + 1, SFMM_LEVEL_COPY);
  SFMM_CUDA_TRY(cudaMemcpyAsync(c->h_level_pin, c->level_off.p, sizeof(int) * ncopy, cudaMemcpyDeviceToHost,
                                c->stream));
  SFMM_CUDA_TRY(cudaMemcpyAsync(c->h_level_pin + SFMM_LEVEL_COPY,
                                c->level_off.as<uint32_t>() + 2 * ((size_t)c->nnodes + 1), sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, c->stream));
  SFMM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  // deepest level holding a walkable internal node (-1: none)
  const int nint = c->h_level_pin[SFMM_LEVEL_COPY];
  c->h_level_off.assign(c->h_level_pin, c->h_level_pin + ncopy);
  c->max_depth = -2;
  for (int d = 0; d < (int)c->h_level_off.size(); ++d)
    if (c->h_level_off[d] >= nint) {
      c->max_depth = d - 1;
      break;
    }
  if (c->max_depth < -1) return SFMM_ESTACK;
  c->h_level_off.resize(c->max_depth + 2);
  c->levels_ready = true;
  return SFMM_OK;
}

int build_tree(sfmm_ctx* c, const double* pos, const double* mass, const double* h) {
  const int n = (int)c->n;
  cudaStream_t st = c->stream;
  int rc;
  const size_t nn_max = (size_t)2 * n;
#define ENS(buf, bytes) \
  if ((rc = c->buf.ensure(bytes)) != SFMM_OK) return rc;
  ENS(keys_a, sizeof(uint64_t) * n);
  ENS(keys_b, sizeof(uint64_t) * n);
  ENS(idx_a, sizeof(uint32_t) * n);
  ENS(idx_b, sizeof(uint32_t) * n);
  ENS(misc, 256 + 64 * (size_t)c->nsys);
  ENS(px, sizeof(double) * n);
  ENS(py, sizeof(double) * n);
  ENS(pz, sizeof(double) * n);
  ENS(pm, sizeof(double) * n);
  ENS(ph, sizeof(double) * n);
  ENS(perm, sizeof(int) * n);
  ENS(pnode, sizeof(int) * n);
  ENS(prel, sizeof(float4) * n);
  ENS(phh, sizeof(float4) * n);
  ENS(k_left, sizeof(int) * n);
  ENS(k_right, sizeof(int) * n);
  ENS(k_first, sizeof(int) * n);
  ENS(k_last, sizeof(int) * n);
  ENS(par_int, sizeof(int) * n);
  ENS(par_leaf, sizeof(int) * n);
  ENS(chain, sizeof(uint32_t) * (n + 1));
  ENS(pre_int, sizeof(int) * n);
  ENS(pre_leaf, sizeof(int) * n);
  ENS(nfirst, sizeof(int) * nn_max);
  ENS(ncount, sizeof(int) * nn_max);
  ENS(nright, sizeof(int) * nn_max);
  ENS(nparent, sizeof(int) * nn_max);
  ENS(isleaf, sizeof(uint32_t) * (nn_max + 1));
  ENS(ncx, sizeof(double) * nn_max);
  ENS(ncy, sizeof(double) * nn_max);
  ENS(ncz, sizeof(double) * nn_max);
  ENS(nsize, sizeof(double) * nn_max);
  ENS(nhmax, sizeof(double) * nn_max);
  ENS(nmass, sizeof(double) * nn_max);
  ENS(l2bits, sizeof(unsigned long long) * nn_max);
  ENS(flags, sizeof(int) * nn_max);
  ENS(geo_hi, sizeof(float4) * nn_max);
  ENS(geo_lo, sizeof(float4) * nn_max);
  ENS(leaf_node, sizeof(int) * nn_max);
  ENS(nlu, sizeof(int) * nn_max);
  ENS(n_extv, sizeof(double) * 6 * nn_max);
  ENS(n_exti, sizeof(int) * 6 * nn_max);
  ENS(size_cand, sizeof(unsigned long long) * 2 * nn_max);
  const int nbb = 2 * num_sms(c->device);
  ENS(bbox_part, sizeof(long long) * 6 * nbb + 16);
#undef ENS
  const int nsys = c->nsys;
  double* bbox = c->misc.as<double>();             // 8 doubles per system
  // scan totals: [0] node count, [1] leaf count (read on the device by every
  // node- and leaf-indexed pass, and by the host with the closing status)
  uint32_t* totals = (uint32_t*)(bbox + 8 * nsys);
  c->d_counts = totals;
  const int* psys = nullptr;                       // system of each particle (batches only)
  if (nsys > 1) {
    if ((rc = c->psys.ensure(sizeof(int) * (size_t)n))) return rc;
    k_fill_psys<<<nblk(n, 256), 256, 0, st>>>(n, nsys, c->sys_off.as<int>(), c->psys.as<int>());
    ++c->nlaunch;
    psys = c->psys.as<int>();
  }
  if ((rc = c->sys_root.ensure(sizeof(int) * (size_t)nsys))) return rc;
  if ((rc = c->wparent.ensure(sizeof(int) * nn_max))) return rc;

  // S1: bounding box (per system), validation, Morton keys
  if (nsys == 1) {
    unsigned* done = reinterpret_cast<unsigned*>(c->bbox_part.as<long long>() + 6 * (size_t)nbb);
    SFMM_CUDA_TRY(cudaMemsetAsync(done, 0, sizeof(unsigned), st));
    k_bbox_partial<<<nbb, BB_NT, 0, st>>>(pos, mass, h, n, c->bbox_part.as<long long>(), done, bbox, c->d_status);
    ++c->nlaunch;
  } else {
    k_bbox_seg<<<nsys, BB_NT, 0, st>>>(pos, mass, h, c->sys_off.as<int>(), bbox, c->d_status);
    ++c->nlaunch;
  }
  uint64_t* ka_final = c->keys_a.as<uint64_t>();  // where the sorted keys end up
  if (c->tree_kind == 1) {
    // centre-of-mass-pivot kd tree: topology, sorted particles, pre-order
    // nodes (level-synchronous on the host, so its counts are known here)
    if ((rc = build_kd_topology(c, pos, mass, h))) return rc;
    const uint32_t hc[2] = {(uint32_t)c->nnodes, (uint32_t)c->nleaves};
    SFMM_CUDA_TRY(cudaMemcpyAsync(totals, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    SFMM_CUDA_TRY(cudaMemsetAsync(c->flags.p, 0, sizeof(int) * (size_t)c->nnodes, st));
    SFMM_CUDA_TRY(cudaMemsetAsync(c->l2bits.p, 0, sizeof(unsigned long long) * (size_t)c->nnodes, st));
  } else {
    k_morton<<<nblk(n, 256), 256, 0, st>>>(pos, n, bbox, psys, c->keys_a.as<uint64_t>(), c->idx_a.as<uint32_t>());
    ++c->nlaunch;
    SFMM_CUDA_TRY(cudaGetLastError());

    // S2: radix sort, 8 passes of 8 bits (the top pass holds 7 key bits)
    const int ntiles = (n + RS_TILE - 1) / RS_TILE;
    const int otiles = (n + OS_TILE - 1) / OS_TILE;
    uint64_t *ka = c->keys_a.as<uint64_t>(), *kb = c->keys_b.as<uint64_t>();
    uint32_t *va = c->idx_a.as<uint32_t>(), *vb = c->idx_b.as<uint32_t>();
    // Morton passes, then (batches) the system id as the most significant digits:
    // the result is ordered by (system, key, input index)
    int sys_bits = 0;
    while ((1 << sys_bits) < nsys) ++sys_bits;
    const int nsysd = (sys_bits + 7) / 8;
    const int npass = 8 + nsysd;
    // digit histograms of all passes at once, then one launch per pass (the
    // published counts have 30 bits; larger sets take the three-step passes)
    const bool onesweep = n < (1 << 30);
    // tile counts: one region per onesweep pass, all zeroed by one memset
    const size_t tstat = sizeof(uint32_t) * 256 * (size_t)otiles;
    if ((rc = c->sort_counts.ensure(onesweep ? tstat * npass : sizeof(uint32_t) * 256 * (size_t)ntiles)) != SFMM_OK)
      return rc;
    if (onesweep) SFMM_CUDA_TRY(cudaMemsetAsync(c->sort_counts.p, 0, tstat * npass, st));
    const size_t aux = sizeof(uint32_t) * 256 * (size_t)npass + sizeof(int) * (size_t)npass;
    if ((rc = c->sort_aux.ensure(aux))) return rc;
    uint32_t* gh = c->sort_aux.as<uint32_t>();
    int* tctr = reinterpret_cast<int*>(gh + 256 * (size_t)npass);
    SFMM_CUDA_TRY(cudaMemsetAsync(gh, 0, aux, st));
    if (onesweep) {
      k_rs_upfront<<<std::min(ntiles, 4 * num_sms(c->device)), RS_NT, 0, st>>>(ka, va, psys, n, 8,
                                                                             psys ? nsysd : 0, gh);
      ++c->nlaunch;
    }
    for (int pass = 0; pass < npass; ++pass) {
      const bool by_sys = pass >= 8;
      const int shift = by_sys ? 8 * (pass - 8) : 8 * pass;
      const int* dsys = by_sys ? psys : nullptr;
      if (onesweep) {
        k_rs_onesweep<<<otiles, RS_NT, 0, st>>>(ka, va, kb, vb, dsys, n, shift, gh + 256 * (size_t)pass,
                                                c->sort_counts.as<uint32_t>() + 256 * (size_t)otiles * pass,
                                                tctr + pass, c->d_status);
        ++c->nlaunch;
      } else {
        k_rs_hist<<<ntiles, RS_NT, 0, st>>>(ka, va, dsys, n, shift, c->sort_counts.as<uint32_t>(), ntiles);
        ++c->nlaunch;
        SFMM_CUDA_TRY(cudaGetLastError());
        if ((rc = exclusive_scan_u32(c, c->sort_counts.as<uint32_t>(), (int64_t)256 * ntiles, nullptr))) return rc;
        k_rs_scatter<<<ntiles, RS_NT, 0, st>>>(ka, va, kb, vb, dsys, n, shift, c->sort_counts.as<uint32_t>(),
                                               ntiles);
        ++c->nlaunch;
      }
      SFMM_CUDA_TRY(cudaGetLastError());
      std::swap(ka, kb);
      std::swap(va, vb);
    }
    // the sorted data is in ka / va
    ka_final = ka;
    k_gather<<<nblk(n, 256), 256, 0, st>>>(pos, mass, h, va, n, c->px.as<double>(), c->py.as<double>(),
                                           c->pz.as<double>(), c->pm.as<double>(), c->ph.as<double>(),
                                           c->perm.as<int>(), c->phh.as<float4>());
    ++c->nlaunch;
    SFMM_CUDA_TRY(cudaGetLastError());

    // S3: radix tree, collapse, pre-order
    if (n == 1) {
      int one = 1, zero = 0, minus = -1;
      SFMM_CUDA_TRY(cudaMemcpyAsync(c->nfirst.as<int>(), &zero, sizeof(int), cudaMemcpyHostToDevice, st));
      SFMM_CUDA_TRY(cudaMemcpyAsync(c->ncount.as<int>(), &one, sizeof(int), cudaMemcpyHostToDevice, st));
      SFMM_CUDA_TRY(cudaMemcpyAsync(c->nright.as<int>(), &minus, sizeof(int), cudaMemcpyHostToDevice, st));
      SFMM_CUDA_TRY(cudaMemcpyAsync(c->nparent.as<int>(), &minus, sizeof(int), cudaMemcpyHostToDevice, st));
      // one leaf, starting at particle 0: its number is 0
      SFMM_CUDA_TRY(cudaMemsetAsync(c->chain.p, 0, sizeof(uint32_t), st));
      static const uint32_t one_node[2] = {1u, 1u};
      SFMM_CUDA_TRY(cudaMemcpyAsync(totals, one_node, sizeof(one_node), cudaMemcpyHostToDevice, st));
    } else {
      const SysView sv{psys, c->sys_off.as<int>()};
      const LeafRule lr{psys, c->sys_lsz.as<int>(), c->leaf_size};
      k_radix_tree<<<nblk(n - 1, 256), 256, 0, st>>>(ka, n, sv, c->k_left.as<int>(), c->k_right.as<int>(),
                                                       c->k_first.as<int>(), c->k_last.as<int>(),
                                                       c->par_int.as<int>(), c->par_leaf.as<int>());
      ++c->nlaunch;
      SFMM_CUDA_TRY(cudaMemsetAsync(c->chain.p, 0, sizeof(uint32_t) * (n + 1), st));
      k_mark<<<nblk(n, 256), 256, 0, st>>>(n, lr, c->k_first.as<int>(), c->k_last.as<int>(),
                                           c->par_int.as<int>(), c->par_leaf.as<int>(), c->chain.as<uint32_t>());
      ++c->nlaunch;
      SFMM_CUDA_TRY(cudaGetLastError());
      // the node count (totals[0]) stays on the device: every node-indexed
      // pass reads it there, and the host learns it with the status word
      if ((rc = exclusive_scan_u32(c, c->chain.as<uint32_t>(), n, totals))) return rc;
      k_preorder<<<nblk(n, 256), 256, 0, st>>>(n, lr, c->k_first.as<int>(), c->k_last.as<int>(),
                                               c->par_int.as<int>(), c->par_leaf.as<int>(),
                                               c->chain.as<uint32_t>(), c->pre_int.as<int>(), c->pre_leaf.as<int>());
      ++c->nlaunch;
      SFMM_CUDA_TRY(cudaGetLastError());
      // leaf-start flags per particle (chain is free again), scanned into
      // leaf numbers; their total is the leaf count (totals[1])
      SFMM_CUDA_TRY(cudaMemsetAsync(c->chain.p, 0, sizeof(uint32_t) * (n + 1), st));
      k_fill_nodes<<<nblk(n, 256), 256, 0, st>>>(n, lr, c->k_left.as<int>(), c->k_right.as<int>(),
                                                 c->k_first.as<int>(), c->k_last.as<int>(), c->par_int.as<int>(),
                                                 c->par_leaf.as<int>(), c->pre_int.as<int>(), c->pre_leaf.as<int>(),
                                                 c->nfirst.as<int>(), c->ncount.as<int>(), c->nright.as<int>(),
                                                 c->nparent.as<int>(), c->chain.as<uint32_t>(), c->d_status);
      ++c->nlaunch;
      SFMM_CUDA_TRY(cudaGetLastError());
      if ((rc = exclusive_scan_u32(c, c->chain.as<uint32_t>(), n, totals + 1))) return rc;
    }
    k_leaf_list<<<node_grid(c), 256, 0, st>>>(c->d_counts, c->nfirst.as<int>(), c->nright.as<int>(),
                                              c->chain.as<uint32_t>(), c->isleaf.as<uint32_t>(),
                                              c->leaf_node.as<int>(), c->flags.as<int>(),
                                              c->l2bits.as<unsigned long long>());
    ++c->nlaunch;
    SFMM_CUDA_TRY(cudaGetLastError());
  }
  // walk parents and system roots
  k_sysroots<<<node_grid(c), 256, 0, st>>>(c->d_counts, psys, c->nfirst.as<int>(), c->ncount.as<int>(),
                                           c->nparent.as<int>(), c->wparent.as<int>(), c->sys_root.as<int>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());

  // S4 geometry, and the moments of the order the last gravity call used
  // (P2M at the leaves, M2M on the way up: the same passes)
  const int P = c->pref_order;
  const int NQ = (int)ncoef(P), nqs = (NQ + 3) & ~3;
  if ((rc = c->Qd.ensure(sizeof(double) * nn_max * NQ)) || (rc = c->Qf.ensure(sizeof(float) * nn_max * nqs)))
    return rc;
  // node depths (exported, and ranks of the one-sided symmetric walk); the
  // per-depth lists are built when a walk first needs them
  if ((rc = compute_depth(c))) return rc;
  c->levels_ready = false;
  switch (P) {
    case 0: rc = geom_upward<0>(c, nqs); break;
    case 1: rc = geom_upward<1>(c, nqs); break;
    case 2: rc = geom_upward<2>(c, nqs); break;
    case 3: rc = geom_upward<3>(c, nqs); break;
    default: rc = geom_upward<4>(c, nqs); break;
  }
  if (rc) return rc;
  k_node_lb<<<node_grid(c), 256, 0, st>>>(c->d_counts, c->wparent.as<int>(), c->nright.as<int>(), c->n_exti.as<int>(),
                                          c->pnode.as<int>(), c->ncx.as<double>(), c->ncy.as<double>(),
                                          c->ncz.as<double>(), c->prel.as<float4>(), c->geo_hi.as<float4>(),
                                          c->geo_lo.as<float4>());
  if (c->tree_kind == 1) {  // (the Morton build's gather wrote them)
    k_particles_hh<<<nblk(n, 256), 256, 0, st>>>(n, c->ph.as<double>(), c->phh.as<float4>());
    ++c->nlaunch;
  }
  k_size_leaf<<<leaf_grid(c), 128, 0, st>>>(c->d_counts, c->leaf_node.as<int>(), c->nfirst.as<int>(),
                                            c->ncount.as<int>(), c->wparent.as<int>(), c->px.as<double>(),
                                            c->py.as<double>(), c->pz.as<double>(), c->ncx.as<double>(),
                                            c->ncy.as<double>(), c->ncz.as<double>(), c->geo_hi.as<float4>(),
                                            c->geo_lo.as<float4>(), c->prel.as<float4>(),
                                            c->l2bits.as<unsigned long long>(), c->size_cand.as<int>());
  k_size<<<nblk(n, SIZE_NT), SIZE_NT, 0, st>>>(n, c->px.as<double>(), c->py.as<double>(), c->pz.as<double>(),
                                       c->pnode.as<int>(), c->isleaf.as<uint32_t>(),
                                       c->size_cand.as<int>(), c->wparent.as<int>(),
                                       c->ncx.as<double>(), c->ncy.as<double>(), c->ncz.as<double>(),
                                       c->geo_hi.as<float4>(), c->geo_lo.as<float4>(), c->prel.as<float4>(),
                                       c->l2bits.as<unsigned long long>());
  c->nlaunch += 3;  // node_lb, size_leaf, size
  k_finalize_nodes<<<node_grid(c), 256, 0, st>>>(c->d_counts, c->l2bits.as<unsigned long long>(),
                                                 c->nhmax.as<double>(), c->nsize.as<double>(), c->geo_hi.as<float4>(),
                                                 c->geo_lo.as<float4>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  c->moments_order = P;
  c->moments_fp64 = (P >= 0 && c->precision != SFMM_FP32);
  if (c->keys_a.p != (void*)ka_final) {
    // keep the sorted keys in keys_a for export (even number of passes: no-op)
    SFMM_CUDA_TRY(cudaMemcpyAsync(c->keys_a.p, ka_final, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
  }
  return SFMM_OK;
}

}  // namespace sfmm
