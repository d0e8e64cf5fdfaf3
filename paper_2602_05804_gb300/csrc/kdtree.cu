// Centre-of-mass-pivot kd tree (Sect. 3: the centre of mass is the pivot of
// the kd-tree build; the axis rule is not printed).  Reading, shared with the
// oracle: split a node with more than leaf_size particles along the axis of
// largest extent of its particles (ties: lowest axis) at its centre of mass
// on that axis; particles below the pivot go left, the others right, both in
// their current order; if one side would be empty, split in the middle.
//
// Level-synchronous build.  Every level's active nodes (more than leaf_size
// particles) are cut into chunks of KD_CH particles.  Each chunk reduces its
// bounding box and mass moments in a fixed order, a thread per node combines
// its chunks in chunk order (so the pivot never depends on scheduling), each
// chunk counts the particles below the pivot, a thread per node turns the
// counts into chunk offsets, and each chunk scatters its particles stably.
// Children get breadth-first ids 2a, 2a + 1 after the level's base, so the
// ids are reproducible.  At the end subtree sizes and pre-order indices are
// computed level by level and the nodes are laid out in pre-order, which is
// the layout every later pass uses.
#include <cfloat>
#include <utility>
#include <vector>

#include "sfmm_internal.cuh"

namespace sfmm {

namespace {

constexpr int KD_CH = 4096;  // particles per chunk
constexpr int KD_NT = 256;
constexpr int KD_NRED = 10;  // min xyz, max xyz, mass, mass-weighted xyz

struct KdChunk {
  int act;    // index of the node in the level's active list
  int start;  // first position of the chunk
  int len;
  int pad;
};

inline unsigned nb(int64_t n, int nt) { return (unsigned)((n + nt - 1) / nt); }

__global__ void k_kd_nchunks(int na, const int* __restrict__ act, const int* __restrict__ cnt,
                             uint32_t* __restrict__ nch) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < na) nch[a] = (uint32_t)((cnt[act[a]] + KD_CH - 1) / KD_CH);
}

__global__ void k_kd_fill(int na, const int* __restrict__ act, const int* __restrict__ first,
                          const int* __restrict__ cnt, const uint32_t* __restrict__ off, KdChunk* __restrict__ ch) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int v = act[a], f = first[v], c = cnt[v];
  const uint32_t o = off[a];
  for (int k = 0; k * KD_CH < c; ++k) ch[o + k] = KdChunk{a, f + k * KD_CH, min(KD_CH, c - k * KD_CH), 0};
}

// Bounding box and mass moments of each chunk (block tree reduction: fixed order).
__global__ void __launch_bounds__(KD_NT) k_kd_reduce(const uint32_t* __restrict__ nchunks,
                                                     const KdChunk* __restrict__ ch, const int* __restrict__ perm,
                                                     const double* __restrict__ pos,
                                                     const double* __restrict__ mass, double* __restrict__ part) {
  const uint32_t b = blockIdx.x;
  if (b >= *nchunks) return;
  const KdChunk k = ch[b];
  double r[KD_NRED] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < k.len; i += KD_NT) {
    const int64_t j = perm[k.start + i];
    const double m = mass[j];
    r[6] += m;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = pos[3 * j + c];
      r[c] = fmin(r[c], x);
      r[3 + c] = fmax(r[3 + c], x);
      r[7 + c] += m * x;
    }
  }
  __shared__ double sh[KD_NRED][KD_NT];
#pragma unroll
  for (int q = 0; q < KD_NRED; ++q) sh[q][threadIdx.x] = r[q];
  __syncthreads();
  for (int w = KD_NT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = fmin(sh[q][threadIdx.x], sh[q][threadIdx.x + w]);
      for (int q = 3; q < 6; ++q) sh[q][threadIdx.x] = fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + w]);
      for (int q = 6; q < KD_NRED; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < KD_NRED) part[(size_t)KD_NRED * b + threadIdx.x] = sh[threadIdx.x][0];
}

// Thread per active node: combine its chunks in order, pick axis and pivot.
__global__ void k_kd_pivot(int na, const int* __restrict__ act, const int* __restrict__ cnt,
                           const uint32_t* __restrict__ off, const double* __restrict__ part, int* __restrict__ axis,
                           double* __restrict__ pivot) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int nch = (cnt[act[a]] + KD_CH - 1) / KD_CH;
  double r[KD_NRED] = {DBL_MAX, DBL_MAX, DBL_MAX, -DBL_MAX, -DBL_MAX, -DBL_MAX, 0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < nch; ++k) {
    const double* p = part + (size_t)KD_NRED * (off[a] + k);
    for (int q = 0; q < 3; ++q) r[q] = fmin(r[q], p[q]);
    for (int q = 3; q < 6; ++q) r[q] = fmax(r[q], p[q]);
    for (int q = 6; q < KD_NRED; ++q) r[q] += p[q];
  }
  int ax = 0;
  for (int c = 1; c < 3; ++c)
    if (r[3 + c] - r[c] > r[3 + ax] - r[ax]) ax = c;
  axis[a] = ax;
  pivot[a] = r[7 + ax] / r[6];
}

__device__ __forceinline__ bool kd_below(const double* pos, int64_t j, int ax, double piv) {
  return pos[3 * j + ax] < piv;
}

// Particles of each chunk below its node's pivot.
__global__ void __launch_bounds__(KD_NT) k_kd_count(const uint32_t* __restrict__ nchunks,
                                                    const KdChunk* __restrict__ ch, const int* __restrict__ perm,
                                                    const double* __restrict__ pos, const int* __restrict__ axis,
                                                    const double* __restrict__ pivot, uint32_t* __restrict__ cl) {
  const uint32_t b = blockIdx.x;
  if (b >= *nchunks) return;
  const KdChunk k = ch[b];
  const int ax = axis[k.act];
  const double piv = pivot[k.act];
  int n = 0;
  for (int i = threadIdx.x; i < k.len; i += KD_NT) n += kd_below(pos, perm[k.start + i], ax, piv) ? 1 : 0;
  __shared__ int sh[KD_NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(SFMM_FULL, n, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < KD_NT / 32; ++w) s += sh[w];
    cl[b] = (uint32_t)s;
  }
}

// Thread per active node: chunk offsets of the left side, the split, and the
// two children (breadth-first ids base + 2a, base + 2a + 1).
__global__ void k_kd_split(int na, const int* __restrict__ act, int* __restrict__ kfirst, int* __restrict__ kcount,
                           int* __restrict__ kparent, int* __restrict__ kleft, int* __restrict__ kright,
                           const uint32_t* __restrict__ off, uint32_t* __restrict__ cl, int* __restrict__ nl_enc,
                           int base) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int v = act[a], f = kfirst[v], c = kcount[v];
  const int nch = (c + KD_CH - 1) / KD_CH;
  uint32_t run = 0;
  for (int k = 0; k < nch; ++k) {
    const uint32_t t = cl[off[a] + k];
    cl[off[a] + k] = run;
    run += t;
  }
  int nl = (int)run;
  const bool mid = (nl == 0 || nl == c);
  if (mid) nl = c / 2;
  nl_enc[a] = mid ? -1 : nl;
  const int L = base + 2 * a, R = L + 1;
  kfirst[L] = f;
  kcount[L] = nl;
  kparent[L] = v;
  kleft[L] = kright[L] = -1;
  kfirst[R] = f + nl;
  kcount[R] = c - nl;
  kparent[R] = v;
  kleft[R] = kright[R] = -1;
  kleft[v] = L;
  kright[v] = R;
}

// Stable scatter of each chunk to its side (middle splits keep the order:
// their particles were copied before this launch).
__global__ void __launch_bounds__(KD_NT) k_kd_scatter(const uint32_t* __restrict__ nchunks,
                                                      const KdChunk* __restrict__ ch, const int* __restrict__ act,
                                                      const int* __restrict__ kfirst,
                                                      const uint32_t* __restrict__ cl, const int* __restrict__ nl_enc,
                                                      const int* __restrict__ axis, const double* __restrict__ pivot,
                                                      const int* __restrict__ pin, const double* __restrict__ pos,
                                                      int* __restrict__ pout) {
  const uint32_t b = blockIdx.x;
  if (b >= *nchunks) return;
  const KdChunk k = ch[b];
  const int nl = nl_enc[k.act];
  if (nl < 0) return;
  const int f = kfirst[act[k.act]];
  const int ax = axis[k.act];
  const double piv = pivot[k.act];
  __shared__ int wl[KD_NT / 32];
  __shared__ int tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int loff = (int)cl[b];                 // lefts of this node before this chunk
  int roff = (k.start - f) - loff;       // rights of this node before this chunk
  for (int base = 0; base < k.len; base += KD_NT) {
    const int i = base + (int)threadIdx.x;
    const bool valid = i < k.len;
    int j = 0;
    bool left = false;
    if (valid) {
      j = pin[k.start + i];
      left = kd_below(pos, j, ax, piv);
    }
    const unsigned bl = __ballot_sync(SFMM_FULL, left);
    if (lane == 0) wl[warp] = __popc(bl);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < KD_NT / 32; ++w) {
      if (w < warp) before += wl[w];
      all += wl[w];
    }
    const int rl = before + __popc(bl & lanemask_lt());   // lefts before me in this round
    const int rr = (int)threadIdx.x - rl;                  // rights before me in this round
    if (valid) pout[left ? f + loff + rl : f + nl + roff + rr] = j;
    const int nvalid = min(KD_NT, k.len - base);
    if (threadIdx.x == 0) tot = all;
    __syncthreads();
    loff += tot;
    roff += nvalid - tot;
    __syncthreads();
  }
}

// Next level's active nodes: children with more than leaf_size particles,
// in child-id order.
__global__ void k_kd_flags(int nch2, int base, const int* __restrict__ kcount, int leaf_size,
                           uint32_t* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nch2) flag[i] = kcount[base + i] > leaf_size ? 1u : 0u;
}

__global__ void k_kd_next(int nch2, int base, const int* __restrict__ kcount, int leaf_size,
                          const uint32_t* __restrict__ scan, int* __restrict__ act) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nch2 && kcount[base + i] > leaf_size) act[scan[i]] = base + i;
}

// Subtree sizes (deepest level first) and pre-order indices (top down).
__global__ void k_kd_size(int lo, int hi, const int* __restrict__ kleft, const int* __restrict__ kright,
                          int* __restrict__ size) {
  const int v = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= hi) return;
  size[v] = kleft[v] < 0 ? 1 : 1 + size[kleft[v]] + size[kright[v]];
}

__global__ void k_kd_pre(int lo, int hi, const int* __restrict__ kleft, const int* __restrict__ kright,
                         const int* __restrict__ size, int* __restrict__ pre) {
  const int v = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= hi || kleft[v] < 0) return;
  pre[kleft[v]] = pre[v] + 1;
  pre[kright[v]] = pre[v] + 1 + size[kleft[v]];
}

__global__ void k_kd_layout(int nn, const int* __restrict__ pre, const int* __restrict__ kfirst,
                            const int* __restrict__ kcount, const int* __restrict__ kparent,
                            const int* __restrict__ kleft, const int* __restrict__ kright, int* __restrict__ nfirst,
                            int* __restrict__ ncount, int* __restrict__ nright, int* __restrict__ nparent,
                            uint32_t* __restrict__ isleaf) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nn) return;
  const int p = pre[v];
  nfirst[p] = kfirst[v];
  ncount[p] = kcount[v];
  nright[p] = kright[v] >= 0 ? pre[kright[v]] : -1;
  nparent[p] = kparent[v] >= 0 ? pre[kparent[v]] : -1;
  isleaf[p] = kleft[v] < 0 ? 1u : 0u;
}

__global__ void k_kd_leaves(int nn, const int* __restrict__ nright, const uint32_t* __restrict__ leafscan,
                            int* __restrict__ leaf_node) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nn && nright[p] < 0) leaf_node[leafscan[p]] = p;
}

__global__ void k_kd_gather(int n, const int* __restrict__ ord, const double* __restrict__ pos,
                            const double* __restrict__ mass, const double* __restrict__ h, double* __restrict__ px,
                            double* __restrict__ py, double* __restrict__ pz, double* __restrict__ pm,
                            double* __restrict__ ph, int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = ord[i];
  px[i] = pos[3 * j];
  py[i] = pos[3 * j + 1];
  pz[i] = pos[3 * j + 2];
  pm[i] = mass[j];
  ph[i] = h[j];
  perm[i] = (int)j;
}

__global__ void k_kd_root(int n, int* kfirst, int* kcount, int* kparent, int* kleft, int* kright, int* act,
                          int* pre) {
  kfirst[0] = 0;
  kcount[0] = n;
  kparent[0] = -1;
  kleft[0] = kright[0] = -1;
  act[0] = 0;
  pre[0] = 0;
}

__global__ void k_kd_iota(int n, int* ord) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ord[i] = i;
}

}  // namespace

int build_kd_topology(sfmm_ctx* c, const double* pos, const double* mass, const double* h) {
  const int n = (int)c->n;
  const int ls = c->leaf_size;
  cudaStream_t st = c->stream;
  const int cap = 2 * n + 1;  // a binary tree over n particles has at most 2n - 1 nodes
  int rc;
  if ((rc = c->kd_ord.ensure(sizeof(int) * 2 * (size_t)n)) || (rc = c->kd_node.ensure(sizeof(int) * 7 * (size_t)cap)) ||
      (rc = c->kd_act.ensure(sizeof(int) * (size_t)n + 64)) ||
      (rc = c->kd_work.ensure(sizeof(uint32_t) * (4 * (size_t)n + 64))))
    return rc;
  int* ord_a = c->kd_ord.as<int>();
  int* ord_b = ord_a + n;
  int* kfirst = c->kd_node.as<int>();
  int* kcount = kfirst + cap;
  int* kparent = kcount + cap;
  int* kleft = kparent + cap;
  int* kright = kleft + cap;
  int* ksize = kright + cap;
  int* kpre = ksize + cap;
  int* act = c->kd_act.as<int>();
  // per-level scratch (sized for the widest level): chunk offsets, chunk
  // records, partial sums, left counts, split results, child flags
  uint32_t* w = c->kd_work.as<uint32_t>();
  uint32_t* off = w;               // na + 1
  uint32_t* flag = w + n + 16;     // 2 na (children of the level)
  uint32_t* dtot = w + 3 * (size_t)n + 32;  // device totals: [0] chunks, [1] next active
  const int ch_cap = n / KD_CH + (n + 1) / 2 + 2;  // chunks of one level: at most n / KD_CH + na
  if ((rc = c->kd_chunk.ensure(sizeof(KdChunk) * (size_t)ch_cap)) ||
      (rc = c->kd_part.ensure(sizeof(double) * KD_NRED * (size_t)ch_cap + sizeof(uint32_t) * (size_t)ch_cap)) ||
      (rc = c->kd_split.ensure((sizeof(int) * 2 + sizeof(double)) * ((size_t)n / 2 + 2))))
    return rc;
  KdChunk* chunks = c->kd_chunk.as<KdChunk>();
  double* part = c->kd_part.as<double>();
  uint32_t* cl = reinterpret_cast<uint32_t*>(part + (size_t)KD_NRED * ch_cap);
  double* pivot = c->kd_split.as<double>();
  int* axis = reinterpret_cast<int*>(pivot + (n / 2 + 2));
  int* nl_enc = axis + (n / 2 + 2);

  k_kd_iota<<<nb(n, 256), 256, 0, st>>>(n, ord_a);
  k_kd_root<<<1, 1, 0, st>>>(n, kfirst, kcount, kparent, kleft, kright, act, kpre);
  c->nlaunch += 2;
  SFMM_CUDA_TRY(cudaGetLastError());
  std::vector<int> lev = {0, 1};  // breadth-first id range of every level
  int na = n > ls ? 1 : 0;
  int nn = 1;
  while (na > 0) {
    if ((int)lev.size() > SFMM_MAXDEPTH) return SFMM_ESTACK;
    // chunks of the active nodes
    k_kd_nchunks<<<nb(na, 256), 256, 0, st>>>(na, act, kcount, off);
    if ((rc = exclusive_scan_u32(c, off, na, dtot))) return rc;
    k_kd_fill<<<nb(na, 256), 256, 0, st>>>(na, act, kfirst, kcount, off, chunks);
    const int ub = n / KD_CH + na + 1;  // chunks of this level, at most
    k_kd_reduce<<<ub, KD_NT, 0, st>>>(dtot, chunks, ord_a, pos, mass, part);
    k_kd_pivot<<<nb(na, 128), 128, 0, st>>>(na, act, kcount, off, part, axis, pivot);
    k_kd_count<<<ub, KD_NT, 0, st>>>(dtot, chunks, ord_a, pos, axis, pivot, cl);
    k_kd_split<<<nb(na, 128), 128, 0, st>>>(na, act, kfirst, kcount, kparent, kleft, kright, off, cl, nl_enc, nn);
    SFMM_CUDA_TRY(cudaMemcpyAsync(ord_b, ord_a, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    k_kd_scatter<<<ub, KD_NT, 0, st>>>(dtot, chunks, act, kfirst, cl, nl_enc, axis, pivot, ord_a, pos, ord_b);
    std::swap(ord_a, ord_b);
    // next level
    const int nch2 = 2 * na;
    k_kd_flags<<<nb(nch2, 256), 256, 0, st>>>(nch2, nn, kcount, ls, flag);
    if ((rc = exclusive_scan_u32(c, flag, nch2, dtot + 1))) return rc;
    k_kd_next<<<nb(nch2, 256), 256, 0, st>>>(nch2, nn, kcount, ls, flag, act);
    c->nlaunch += 9;
    SFMM_CUDA_TRY(cudaGetLastError());
    uint32_t h_next = 0;
    SFMM_CUDA_TRY(cudaMemcpyAsync(&h_next, dtot + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    SFMM_CUDA_TRY(cudaStreamSynchronize(st));
    nn += nch2;
    lev.push_back(nn);
    na = (int)h_next;
  }
  // subtree sizes bottom-up, pre-order indices top-down, pre-order layout
  const int nlev = (int)lev.size() - 1;
  for (int L = nlev - 1; L >= 0; --L) {
    k_kd_size<<<nb(lev[L + 1] - lev[L], 256), 256, 0, st>>>(lev[L], lev[L + 1], kleft, kright, ksize);
    ++c->nlaunch;
  }
  for (int L = 0; L < nlev; ++L) {
    k_kd_pre<<<nb(lev[L + 1] - lev[L], 256), 256, 0, st>>>(lev[L], lev[L + 1], kleft, kright, ksize, kpre);
    ++c->nlaunch;
  }
  k_kd_layout<<<nb(nn, 256), 256, 0, st>>>(nn, kpre, kfirst, kcount, kparent, kleft, kright, c->nfirst.as<int>(),
                                          c->ncount.as<int>(), c->nright.as<int>(), c->nparent.as<int>(),
                                          c->isleaf.as<uint32_t>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  if ((rc = exclusive_scan_u32(c, c->isleaf.as<uint32_t>(), nn, dtot))) return rc;
  k_kd_leaves<<<nb(nn, 256), 256, 0, st>>>(nn, c->nright.as<int>(), c->isleaf.as<uint32_t>(), c->leaf_node.as<int>());
  k_kd_gather<<<nb(n, 256), 256, 0, st>>>(n, ord_a, pos, mass, h, c->px.as<double>(), c->py.as<double>(),
                                          c->pz.as<double>(), c->pm.as<double>(), c->ph.as<double>(),
                                          c->perm.as<int>());
  c->nlaunch += 2;
  SFMM_CUDA_TRY(cudaMemsetAsync(c->keys_a.p, 0, sizeof(uint64_t) * (size_t)n, st));  // a kd tree has no keys
  SFMM_CUDA_TRY(cudaGetLastError());
  c->nnodes = nn;
  c->nleaves = (nn + 1) / 2;
  return SFMM_OK;
}

}  // namespace sfmm
