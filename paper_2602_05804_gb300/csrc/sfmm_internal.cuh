// Internal declarations of the SFMM gravity library: the context and the
// stage launchers implemented in tree.cu, moments.cu, walk.cu, p2p.cu.
#pragma once
#include <string>
#include <vector>

#include "sfmm_common.cuh"

struct sfmm_tune_table;  // autotuner table (autotune.cu)

// Device buffer that only grows (freed on destroy).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t need);  // SFMM_OK / SFMM_ENOMEM
  void release();
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

struct sfmm_ctx {
  int device = 0;
  int precision = SFMM_FP64;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  std::string last_error;

  // options
  double G = 1.0;
  int self_potential = 0;
  int ring_capacity = 8192;
  int64_t list_capacity = 0;
  int64_t cf_capacity = 0;  // child-frontier arena entries per level parity (0 = automatic)
  int profile = 0;
  int tree_kind = 0;        // 0: Morton radix tree, 1: centre-of-mass-pivot kd tree

  // built state
  bool built = false;
  int64_t n = 0;
  int leaf_size = 0;
  // systems of a batch (nsys = 1 for a single particle set): particle offsets
  // and leaf sizes on host and device; the system of each particle; the root
  // node of each system; each node's parent for the walk (-1 at a system
  // root, -2 for nodes spanning several systems); per-system sums
  int nsys = 1;
  std::vector<int64_t> h_sys_off;
  std::vector<int> h_sys_lsz;
  DevBuf sys_off, sys_lsz, psys, sys_root, wparent, sys_sums;
  int32_t nnodes = 0, nleaves = 0;  // host copies, valid once a build has returned
  uint32_t* d_counts = nullptr;      // device: node count, leaf count of the current build, leaf-pair parents
  bool graph_mode = false;           // buffers sized for a captured step (bounds, device counts)
  // captured step (sfmm_solve_graph): one graph per shape class, with the
  // class it was captured for and the fingerprint of the buffers it uses;
  // a reallocated buffer, an option change or an ordinary build invalidates it
  cudaGraphExec_t graph_exec = nullptr;
  bool graph_valid = false;
  std::vector<int64_t> g_off;
  std::vector<int> g_lsz;
  double g_theta = -1.0;
  int g_order = -1;
  const void* g_ptr[5] = {};
  unsigned long long g_mark = 0;
  int64_t graph_replays = 0;
  int64_t g_launches = 0;  // kernels in the captured step
  bool g_auto_leaf = false;  // captured with autotuned (NULL) leaf sizes
  int moments_order = -1;  // order of the cached moments (-1: none)
  bool moments_fp64 = false;  // the cached moments include the FP64 rows (else FP32 only)
  int pref_order = 2;      // order the build computes moments for (the last gravity call's)
  int walk_mode = 1;        // 1: per-node shared pairs (default), 0: per-leaf replay (Algorithm 1),
                            // 2: per-node pairs, each evaluated once for both sides
  int schedule = 0;         // walk mode 1: 0 automatic, 1 one launch per depth, 2 readiness queue
  int p2p_chunk = SFMM_P2P_CHUNK_DEFAULT;  // neighbour-list entries per near-field work item
  int p2p_blocks = 0;       // near-field blocks per SM (0: as many as fit)
  int max_depth = 0;
  std::vector<int> h_level_off;  // host copy: internal nodes per depth, max_depth + 2 entries
  int* h_level_pin = nullptr;     // pinned landing buffer of the level offsets (and their total)
  bool levels_ready = false;      // per-depth lists built for the current tree
  int* h_sys_pin = nullptr;       // pinned staging of system offsets and leaf sizes
  size_t h_sys_pin_cap = 0;
  cudaEvent_t ev_stage = nullptr;  // after the last staged copies

  // inputs staged from host (sfmm_solve_host)
  DevBuf in_pos, in_mass, in_h;
  DevBuf out_acc, out_pot;

  // sort / build temporaries
  DevBuf keys_a, keys_b, idx_a, idx_b, sort_counts, scan_tmp, bbox_part;
  DevBuf sort_aux;  // radix sort: digit histograms of every pass, tile counters
  DevBuf k_left, k_right, k_first, k_last, par_int, par_leaf, chain, pre_int, pre_leaf;
  DevBuf misc;  // device-side scalars: bbox, counters

  // sorted particles
  DevBuf px, py, pz, pm, ph;    // float64 SoA
  DevBuf perm;                  // int32 sorted position -> input index
  DevBuf pnode;                 // int32 sorted position -> leaf node
  DevBuf prel;                  // float4 {x - s_leaf, y - s_leaf, z - s_leaf, m}
  DevBuf phh;                   // float4 {1/h, (2h)^2, 2h rounded up, 0}

  // nodes (pre-order)
  DevBuf nfirst, ncount, nright, nparent, ndepth;
  DevBuf ncx, ncy, ncz, nsize, nhmax, nmass;
  DevBuf l2bits, flags;
  DevBuf geo_hi, geo_lo;        // float4 walk records
  DevBuf leaf_node, isleaf;
  DevBuf nlu;                   // leaves under each node
  DevBuf n_extv, n_exti;        // axis-extreme particles (values, positions)
  DevBuf size_cand;             // per leaf: ancestors its particles may hold the size of
  DevBuf level_nodes, level_off, level_cur;  // internal nodes grouped by depth
  DevBuf leaf_order;            // leaves by depth, shallowest first
  DevBuf Qd, Qf;                // scaled moments float64 [nn x NQ], float32 [nn x NQS]

  // gravity
  DevBuf ring, far, arena, p2p_off, p2p_cnt, counters, red_part, dump;
  DevBuf cf_arena, cf_off, cf_cnt, Tnode;  // shared walk: child frontiers, node coefficients
  DevBuf sym_own, sym_recv;               // walk mode 2: own and received sums per node (FP64)
  DevBuf wqueue;                          // walk mode 3: nodes in order of readiness
  // near field: chunks of long neighbour lists (extra work items, per-leaf
  // slot base, split leaves, partial sums) and the list entries in use
  DevBuf p2p_extra, p2p_split, p2p_slist, p2p_part;
  // leapfrog: accelerations, per-tile momentum partials and their sum
  DevBuf lf_acc, lf_part;
  // kd-tree build: particle orders, breadth-first node records, level scratch
  DevBuf kd_ord, kd_node, kd_act, kd_work, kd_chunk, kd_part, kd_split;
  const double* red_acc = nullptr;  // outputs of the last near-field pass (caller order), read by the sums
  const double* red_pot = nullptr;
  int64_t arena_used = 0;
  int64_t split_chunks = 0, split_lists = 0;  // from the walk: chunks of split lists, split lists
  int64_t walk_arena_cap = 0, walk_cf_cap = 0;  // list and child-list capacities of the last walk

  // status word (device) + pinned host mirror
  int* d_status = nullptr;
  int* h_status = nullptr;
  double* h_scalars = nullptr;  // pinned host scratch

  // autotuner: table of tuned choices, and the theta / order that builds with
  // autotuned leaf sizes (sfmm_build_batch with leaf_size NULL) tune for
  sfmm_tune_table* tune = nullptr;
  double tune_theta = 0.5;
  int tune_order = 2;

  int64_t nlaunch = 0;  // kernels launched by this context (cumulative)
  cudaEvent_t ev[8] = {};
  sfmm_stats stats{};
};

namespace sfmm {

int set_error(sfmm_ctx* c, int code, const char* msg);

// tree.cu
int build_tree(sfmm_ctx* c, const double* pos, const double* mass, const double* h);
// per-depth node lists and their host offsets, on first use after a build
int ensure_levels(sfmm_ctx* c);
// kdtree.cu: kd-tree topology, sorted particles and pre-order node layout
int build_kd_topology(sfmm_ctx* c, const double* pos, const double* mass, const double* h);
int compute_depth(sfmm_ctx* c);
int build_levels(sfmm_ctx* c);  // depth, level lists, leaves under each node

// scan (tree.cu): exclusive scan of n uint32 values in place, returns total
// through `total_dev` (device uint32, may be null)
int exclusive_scan_u32(sfmm_ctx* c, uint32_t* data, int64_t n, uint32_t* total_dev);

// moments.cu
int compute_moments(sfmm_ctx* c, int order);

// walk_shared.cu: launches only (no host wait); the caller checks the status
// word and calls walk_shared_regrow on capacity bits
int run_walk_shared(sfmm_ctx* c, double theta, int order);
int walk_shared_regrow(sfmm_ctx* c, int bits, const unsigned long long* hs);

// walk.cu
int run_walk(sfmm_ctx* c, double theta, int order, bool dump, int64_t cap_m2l, int64_t cap_p2p);

// p2p.cu
int run_p2p(sfmm_ctx* c, double* acc, double* pot);
int run_reduce(sfmm_ctx* c, double** out_dev);  // device pointer of the 5 sums
int run_reduce_systems(sfmm_ctx* c);             // per-system sums (batches)

// autotune.cu
void tune_table_free(sfmm_ctx* c);
int tune_set_cache(sfmm_ctx* c, const char* path);
int tuned_leaf_sizes(sfmm_ctx* c, int nsys, const int64_t* offsets, const double* pos, const double* mass,
                     const double* h, double theta, int order, std::vector<int>& lsz);
int tuned_knobs(sfmm_ctx* c, double theta, int order, double* acc, bool run_trials);
int p2p_blocks_fit(sfmm_ctx* c);  // near-field blocks per SM that fit (p2p.cu)

std::vector<DevBuf*> ctx_buffers(sfmm_ctx* c);        // every device buffer of a context
unsigned long long buffers_fingerprint(sfmm_ctx* c);  // their addresses and sizes, folded

int check_status(sfmm_ctx* c);
int sync_status(sfmm_ctx* c, int* bits, bool counts = false);

inline int num_sms(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v > 0 ? v : 1;
}

}  // namespace sfmm
