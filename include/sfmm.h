/*
 * sfmm.h -- C ABI of the GB300 (sm_103a) symmetric fast multipole gravity
 * solver with adaptive kernel softening.
 *
 * The method is the momentum-conserving symmetric Cartesian fast multipole
 * method (SFMM) of Bernard, David-Cleris, Price & Lau, "Momentum-conserving
 * self-gravity in the Phantom SPH code" (arXiv 2602.05804):
 *   - the softened gravitational acceleration and potential of N particles
 *     (Sect. 2, Eqs. directsum and softdirectsum) are computed with
 *   - a binary tree whose nodes carry Cartesian mass moments (Eq. massmom,
 *     moments translated bottom-up with Eq. massmomtrans, App. A.1),
 *   - a dual-tree walk replayed per leaf on the leaf's branch of parents
 *     (Algorithms 1 and 2, Sect. 3) with the opening-angle criterion and the
 *     softening criterion of Sect. 3,
 *   - node-node expansions (Eq. dmkdeffmm, Sect. 2.2) translated down the
 *     branch (Eq. gravmtranslat, App. A.2) and evaluated at the particles,
 *   - pairwise kernel-softened gravity for every pair inside the kernel.
 *
 * Conventions for every entry point:
 *   - Return value: SFMM_OK (0) or one of the error codes below.  No entry
 *     point throws, aborts or prints; sfmm_last_error() gives a message.
 *   - Device pointers are CUDA device (or managed) memory on the context's
 *     device, owned by the caller; the library never frees them.  "host"
 *     pointers are ordinary or pinned host memory, owned by the caller.
 *   - All work is issued on the context's stream.  Calls return after the
 *     work they issued has completed (each call ends with one stream
 *     synchronisation to read the device status word), so outputs are ready
 *     on return.
 *   - Positions are row-major n x 3 (x, y, z per particle) float64.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef SFMM_H
#define SFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfmm_ctx sfmm_ctx;

/* Error codes. */
enum {
  SFMM_OK = 0,
  SFMM_EINVAL = 1,      /* bad argument (range, NULL, size) */
  SFMM_ENOMEM = 2,      /* device allocation failed */
  SFMM_ECUDA = 3,       /* a CUDA runtime call failed */
  SFMM_ESTATE = 4,      /* call out of order (e.g. gravity before build) */
  SFMM_ESTACK = 5,      /* a leaf's branch is deeper than the walk supports */
  SFMM_ECAPACITY = 6,   /* a work buffer was too small even after regrowing */
  SFMM_ENONFINITE = 7,  /* non-finite or non-positive input value */
  SFMM_ENOTIMPL = 8     /* not implemented in this build */
};

/* Arithmetic forms. */
enum {
  SFMM_FP64 = 0,  /* every step in float64 */
  SFMM_FP32 = 1   /* P2P and M2L in float32 on coordinates relative to node
                     centres; centres, sizes and the acceptance decisions in
                     float64; inherited expansion coefficients accumulated in
                     double-float; reductions in float64 */
};

/* Statistics of the last build / gravity call. */
typedef struct sfmm_stats {
  int64_t n;            /* particles */
  int64_t nnodes;       /* tree nodes (leaves included) */
  int64_t nleaves;      /* leaves */
  int64_t m2l;          /* node-node interactions evaluated, counted once per
                           leaf whose branch replays them (Algorithm 1) */
  int64_t m2l_unique;   /* distinct directed node pairs among them */
  int64_t p2p_leaves;   /* leaf-leaf entries of the neighbour lists */
  int64_t p2p_pairs;    /* particle-particle evaluations (i != j) */
  int64_t mac_fallbacks;/* acceptance tests settled by the exact float64 path */
  double momentum[3];   /* sum_i m_i a_i */
  double abs_momentum;  /* sum_i sum_d |m_i a_i,d| */
  double W;             /* 1/2 sum_i m_i Phi_i */
  double ms_build;      /* device time of the last sfmm_build (profiling on) */
  double ms_moments;    /* device time of the moment pass of the last gravity */
  double ms_walk;       /* device time of the walk + M2L + L2L + L2P kernel */
  double ms_p2p;        /* device time of the near-field kernel */
  double ms_reduce;     /* device time of the reductions */
  double ms_gravity;    /* device time of the whole last sfmm_gravity */
  int64_t kernel_launches; /* CUDA kernels this context has launched so far */
  int64_t graph_replays;   /* steps sfmm_solve_graph ran as a replayed graph */
} sfmm_stats;

/* Create a context on CUDA device `device` in arithmetic form `precision`
 * (SFMM_FP64 or SFMM_FP32).  `stream` is a cudaStream_t to issue all work on,
 * or NULL for a stream the context creates and owns.  *out receives the
 * context (NULL on failure).  Errors: EINVAL (bad device/precision), ECUDA. */
int sfmm_create(sfmm_ctx** out, int device, int precision, void* stream);

/* Destroy a context and free every buffer it owns.  NULL is a no-op. */
void sfmm_destroy(sfmm_ctx* ctx);

/* Replace the stream used by later calls (cudaStream_t, NULL = own stream). */
int sfmm_set_stream(sfmm_ctx* ctx, void* stream);

/* Set an option.  Keys:
 *   "G"              gravitational constant (default 1, code units as in Sect. 4.2)
 *   "self_potential" 1 adds each particle's own kernel term G m_i phi(0, h_i)
 *                    to its potential (the j = i term of Eq. softdirectsum);
 *                    default 0 (sum over j != i as in Eq. directsum)
 *   "ring_capacity"  walk frontier entries per warp (power of two, >= 256)
 *   "list_capacity"  P2P list arena entries (0 = automatic)
 *   "walk"           1 (default): each node's pairs are evaluated once and
 *                    shared by the leaves below it (the caching of shared
 *                    interactions proposed in Sect. 5); 0: each leaf replays
 *                    the walk of its branch (Algorithm 1 as printed); 2: as
 *                    1, with each accepted pair's derivative tensor evaluated
 *                    once for both nodes (the one-sided symmetric form of
 *                    Sect. 5, FP64 accumulation of the partner's side); same
 *                    interactions, same results up to summation order
 *   "schedule"       order of the nodes in walk 1 (a node needs its parent's
 *                    opened list and coefficients): 1 one launch per depth;
 *                    2 one launch in which a warp takes the next node whose
 *                    parent is done from a queue; 3 the same with both
 *                    children of a node taken by one warp (their common
 *                    inherited list read once); 0 (default) chooses 2 when
 *                    the walk's per-node records take at most twice the L2
 *                    cache, else 3; bitwise the same results
 *   "tree"           0 (default): binary radix tree over Morton keys (Sect. 3);
 *                    1: centre-of-mass-pivot kd tree (Sect. 3; single
 *                    systems only, sfmm_build_batch returns ENOTIMPL)
 *   "p2p_chunk"      neighbour-list entries per near-field work item: longer
 *                    lists are cut into chunks evaluated as separate items
 *                    and recombined in chunk order (default 256, 32..65536)
 *   "p2p_blocks"     near-field blocks per SM (0, default: as many as fit)
 *   "autotune_theta", "autotune_order"  theta and order that autotuned leaf
 *                    sizes are chosen for (sfmm_build_batch with NULL sizes)
 *   "profile"        1 records per-stage device times into the stats
 * Errors: EINVAL (unknown key or out-of-range value). */
int sfmm_set_option(sfmm_ctx* ctx, const char* key, double value);

/* Build the tree (Sect. 3) of n particles: bounding box, 63-bit Morton keys
 * (21 bits per axis on the cube of the box's largest extent), stable sort by
 * (key, input index), binary radix tree split at the highest differing bit
 * of (key, sorted position), leaves of at most leaf_size particles, node
 * centres of mass, sizes l = max |x_j - s| over the node's particles and
 * maximum smoothing lengths h_max.
 *   pos  device, n x 3 float64;  mass device, n float64 (> 0);
 *   h    device, n float64 smoothing lengths (> 0);  leaf_size in [1, 64].
 * The inputs are copied into the context and may be freed after the call.
 * Errors: EINVAL (n < 1, n > 2^31 - 2, leaf_size, NULL), ENONFINITE,
 * ENOMEM, ECUDA. */
int sfmm_build(sfmm_ctx* ctx, int64_t n, const double* pos, const double* mass, const double* h,
               int leaf_size);

/* Gravitational accelerations and potentials of the last built particle set
 * (Sect. 3, Algorithms 1 and 2): mass moments to order `order` (Eq. massmom,
 * App. A.1), the per-leaf walk with opening angle `theta`
 * ((l_t + l_s) / d < theta) and the softening criterion
 * (open if d < l_t + l_s + 2 max(h_max,t, h_max,s)), node-node expansions
 * (Eq. dmkdeffmm), their translation down each branch (Eq. gravmtranslat),
 * evaluation at the particles and pairwise M4-softened gravity over the
 * neighbour lists.
 *   theta in [0, 1) (0: every pair pairwise, i.e. the softened direct sum);
 *   order in [0, 4] (expansion order p; moments to p, coefficients to p + 1);
 *   acc  device, n x 3 float64, caller (input) order, written;
 *   pot  device, n float64, caller order, written; may be NULL.
 * Errors: ESTATE (no build), EINVAL, ESTACK, ECAPACITY, ENOMEM, ECUDA. */
int sfmm_gravity(sfmm_ctx* ctx, double theta, int order, double* acc, double* pot);

/* Build one tree over a batch of nsys independent particle systems packed
 * back to back (an ensemble service; the paper solves one particle set at a
 * time): system s owns particles
 * [offsets[s], offsets[s+1]).  Each system gets its own bounding box, Morton
 * keys and leaf size; the combined sort orders particles by (system, key,
 * input index) and nodes spanning several systems are always split and never
 * walked, so each system's subtree equals the tree sfmm_build would give it
 * and systems never interact.  All later calls then treat every system in
 * the same kernel launches.
 *   nsys in [1, 65536];  offsets HOST, nsys + 1 int64, offsets[0] = 0,
 *   strictly increasing, offsets[nsys] = total n <= 2^31 - 2;
 *   pos/mass/h device, packed as for sfmm_build;
 *   leaf_size HOST, nsys ints in [1, 64], or NULL: autotuned.  With NULL
 *             every system takes the leaf size the context's autotuner table
 *             holds for its (size bucket floor(log2 N), profile class, theta,
 *             order, form), theta and order being the options
 *             "autotune_theta" / "autotune_order" (default 0.5 / 2, set by
 *             sfmm_autotune_batch); groups of systems without an entry are
 *             timed first (see sfmm_autotune_batch), so a first NULL call
 *             takes longer.  The batch's cached launch knobs (walk schedule,
 *             near-field blocks per SM and list chunk) are applied too, when
 *             the table has them.
 * Errors: as sfmm_build. */
int sfmm_build_batch(sfmm_ctx* ctx, int nsys, const int64_t* offsets, const double* pos, const double* mass,
                     const double* h, const int* leaf_size);

/* Autotune a batch (an ensemble service; the paper has no counterpart) and
 * build it: every system's leaf size and the batch's launch knobs are picked
 * from timed trials on the caller's own systems at this theta and order, in
 * this context's arithmetic form.
 *   Leaf size in {8, 16, 32, 64} per (size bucket floor(log2 N), profile
 *   class, theta, order, form); the profile class is cut from the ratio of the
 *   rms to the mean distance from the system's centre of mass (<1.1: 0, e.g. a
 *   homogeneous sphere; <1.25: 1; <1.6: 2, e.g. a Plummer sphere; else 3).
 *   One trial per group without a table entry: the system nearest the group's
 *   median size, built and solved with each candidate in a scratch context
 *   (best of two timed runs after a warm-up run, CUDA events).
 *   Launch knobs per (total-size bucket, log2 nsys, theta, order, form): walk
 *   "schedule" {1, 2, 3} x "p2p_blocks" {all that fit, one fewer} x "p2p_chunk"
 *   {128, 256, 512}, each timed on a gravity call of the whole batch; the
 *   best are set as this context's options.
 * Arguments as sfmm_build_batch (leaf sizes are chosen, not given) plus
 * theta and order as sfmm_gravity; leaf_size_out HOST nsys ints or NULL
 * receives the chosen leaf sizes.  The batch is built on return (call
 * sfmm_gravity_batch next); "autotune_theta"/"autotune_order" are set to
 * theta/order.  Errors: as sfmm_build_batch and sfmm_gravity. */
int sfmm_autotune_batch(sfmm_ctx* ctx, int nsys, const int64_t* offsets, const double* pos, const double* mass,
                        const double* h, double theta, int order, int* leaf_size_out);

/* Build + gravity of one particle set or batch as ONE CUDA graph per shape
 * class (an ensemble service; the paper has no counterpart): the same
 * results as sfmm_build_batch + sfmm_gravity_batch (bitwise), issued as a
 * single graph launch followed by one synchronisation.
 *   Arguments as sfmm_build_batch (nsys = 1 for a single set; leaf_size
 *   HOST nsys ints, or NULL for autotuned sizes) and sfmm_gravity (theta,
 *   order, acc, pot).  The shape class is (offsets, leaf sizes, theta, order,
 *   the five array addresses); the particle values may change freely between
 *   calls (positions of a time step, say): the graph's kernels take the node
 *   and leaf counts of each replay's own build from the device.
 *   The first call of a shape class runs the ordinary calls (sizing every
 *   node- and leaf-indexed buffer for the bounds: 2n nodes, n leaves) and
 *   then captures the step on the context's stream; later calls replay it.
 *   A walk buffer that runs out during a replay (status bit) is grown and
 *   the step rerun the ordinary way, then captured again.  Changing an
 *   option, an ordinary build on the context, or any reallocation of the
 *   context's buffers invalidates the graph (the next call recaptures).
 *   sfmm_get_stats counts replays in graph_replays.
 * Needs the Morton tree (option "tree" 0), walk 1 and at least two
 * particles; the walk runs on a readiness queue (schedule 2 or 3, the
 * automatic choice otherwise).  Errors: as sfmm_build_batch and
 * sfmm_gravity; ENOTIMPL for another tree or walk. */
int sfmm_solve_graph(sfmm_ctx* ctx, int nsys, const int64_t* offsets, const double* pos, const double* mass,
                     const double* h, const int* leaf_size, double theta, int order, double* acc, double* pot);

/* Cache file of the context's autotuner table (JSON): entries in the file
 * are loaded now (a missing file is an empty table) and the file is
 * rewritten whenever a trial adds an entry.  NULL or "" stops caching.
 * Errors: EINVAL (file not writable when an entry is added). */
int sfmm_autotune_cache(sfmm_ctx* ctx, const char* path);

/* Gravity of every system of the last build (batch or single), same
 * arguments, layout (packed caller order) and errors as sfmm_gravity. */
int sfmm_gravity_batch(sfmm_ctx* ctx, double theta, int order, double* acc, double* pot);

/* Per-system sums of the last gravity call into HOST out[nsys x 5]:
 * sum m a (3), sum |m a| (componentwise), W = 1/2 sum m Phi.
 * Errors: ESTATE, EINVAL (nsys differs from the build). */
int sfmm_batch_sums(const sfmm_ctx* ctx, int nsys, double* out);

/* Whole solve from HOST buffers: copies the inputs to the device, builds,
 * runs the gravity and copies the results back, all on the context's stream.
 * Same arguments and errors as sfmm_build + sfmm_gravity, but every pointer
 * is a host pointer (pinned memory gives the fastest copies: the device
 * then reads and writes it directly, by a copy kernel).  With the
 * Morton tree and the shared walk (the defaults) and n >= 2, build and
 * gravity run as sfmm_solve_graph's captured step on the context's staging
 * buffers (bitwise the same results; repeated calls of one shape replay
 * one graph). */
int sfmm_solve_host(sfmm_ctx* ctx, int64_t n, const double* pos, const double* mass,
                    const double* h, int leaf_size, double theta, int order, double* acc,
                    double* pot);

/* Statistics of the last calls (counts, momentum and energy sums; stage
 * times when the "profile" option is on).  Errors: EINVAL (NULL). */
int sfmm_get_stats(const sfmm_ctx* ctx, sfmm_stats* out);

/* Sizes of the built tree.  Errors: ESTATE (no build). */
int sfmm_tree_size(const sfmm_ctx* ctx, int64_t* nnodes, int64_t* nleaves);

/* Copy the built tree to HOST arrays (any pointer may be NULL).  Nodes are in
 * pre-order (a node's left child is the next node); leaves in tree order.
 *   perm[n]    sorted position -> input index;   keys[n] Morton keys (sorted)
 *   first/count/right/parent/depth[nnodes]  (right = -1 and count <= leaf_size
 *              for leaves; parent = -1 for the root)
 *   centre[nnodes x 3], size[nnodes], hmax[nnodes], mass[nnodes]
 *   leaves[nleaves] node index of each leaf.
 * Errors: ESTATE, ECUDA. */
int sfmm_tree_export(const sfmm_ctx* ctx, int64_t* perm, uint64_t* keys, int32_t* first,
                     int32_t* count, int32_t* right, int32_t* parent, int32_t* depth,
                     double* centre, double* size, double* hmax, double* mass, int32_t* leaves);

/* Compute the scaled mass moments Q_alpha / alpha! of every node to order
 * `order` (Eq. massmom, translated with Eq. massmomtrans) and copy them to
 * HOST array Q[nnodes x C(order+3,3)].  mi (may be NULL) receives the
 * multi-index (a,b,c) of each column, C(order+3,3) x 3 int32.
 * Errors: ESTATE, EINVAL, ECUDA. */
int sfmm_moments_export(sfmm_ctx* ctx, int order, double* Q, int32_t* mi);

/* Interaction lists of every leaf for opening angle theta (decisions of
 * Algorithm 2 only, no arithmetic), into HOST arrays:
 *   m2l_off[nleaves + 1], p2p_off[nleaves + 1] offsets (always written);
 *   m2l_level[cap_m2l], m2l_src[cap_m2l]: level k of the branch node and the
 *     source node of each accepted pair; p2p_src[cap_p2p]: neighbour leaves.
 * With NULL entry arrays only the offsets are written (sizes query).  Order
 * of entries within a leaf is unspecified.
 * Errors: ESTATE, EINVAL (theta), ECAPACITY (caps too small), ECUDA. */
int sfmm_lists(sfmm_ctx* ctx, double theta, int64_t* m2l_off, int32_t* m2l_level, int32_t* m2l_src,
               int64_t cap_m2l, int64_t* p2p_off, int32_t* p2p_src, int64_t cap_p2p);

/* Gravity-only leapfrog of one particle set with the SFMM forces (the
 * gravity part of the binary-polytrope test of Sect. 4: every pair force is
 * antisymmetric, so the total linear momentum is conserved to rounding).
 * Kick-drift-kick steps: v += a dt/2, x += v dt, rebuild the tree at the new
 * positions, a = SFMM acceleration, v += a dt/2.
 *   n            number of particles, as in sfmm_build
 *   pos, vel     device, n x 3 row-major FP64, caller order; advanced in
 *                place by nsteps steps
 *   mass, h      device, n; h stays fixed
 *   leaf_size, theta, order   as in sfmm_build / sfmm_gravity
 *   dt           step length (finite, may be negative: steps run backwards)
 *   nsteps       >= 0
 *   record_every >= 1; a record is taken before the first step and after
 *                every record_every-th step
 *   record       host, (nsteps / record_every + 1) x 8 doubles, or NULL:
 *                t, P = sum m v (3), L = sum m x cross v (3), sum |m v_d|
 *                (over particles and components); FP64 sums in a fixed order
 *   acc          device n x 3 or NULL: the accelerations of the final state
 * The context holds the tree of the final positions afterwards.  Errors: as
 * sfmm_build and sfmm_gravity, EINVAL for bad arguments; after an error pos
 * and vel are left part-way through the failed step. */
int sfmm_leapfrog(sfmm_ctx* ctx, int64_t n, double* pos, double* vel, const double* mass, const double* h,
                  int leaf_size, double theta, int order, double dt, int64_t nsteps, int64_t record_every,
                  double* record, double* acc);

/* Largest n accepted by sfmm_reduce_noalloc. */
#define SFMM_NOALLOC_MAX_N 67108864

/* Momentum and energy sums of a particle set WITHOUT ANY DEVICE ALLOCATION:
 * out[0..2] = sum_i m_i a_i, out[3] = sum_i sum_d |m_i a_i,d|,
 * out[4] = 1/2 sum_i m_i Phi_i (0 when pot is NULL) -- the same sums that
 * sfmm_get_stats reports after sfmm_gravity (momentum components as
 * Neumaier-compensated FP64 sums), here over caller arrays.  The paper has no counterpart: this is a service for callers
 * that cannot call cudaMalloc, such as code that must draw all device memory
 * from its own pre-reserved pool or must not change the device's memory
 * footprint once it is running.  No context is needed and nothing is
 * allocated, freed or taken from a library allocator.
 *   n     number of particles, 1 <= n <= SFMM_NOALLOC_MAX_N (larger n is
 *         rejected with SFMM_EINVAL);
 *   mass  device, n float64;  acc device, n x 3 float64;  pot device, n
 *         float64 or NULL;  out device, 5 float64, written;
 *   stream  cudaStream_t to run on (NULL: the default stream), on the
 *         current device.
 * Scratch: per-tile partial sums (one per 4096 particles) in a fixed 1.25 MB
 * array of device memory inside this library, which every GPU that loads the
 * library holds until the process exits.  Every call shares that array, which
 * keeps the last call's contents; each call writes every partial it reads, so
 * nothing needs clearing.  Each GPU has its own copy of the array; calls that
 * overlap on the same GPU (for example on two streams) race on the partials,
 * so serialise them.  The first call in a CUDA context looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The address is cached per device
 * and context: after cudaDeviceReset (a new context) the next call looks it
 * up again.  Unlike the other entry points this call does not synchronise:
 * out is ready when the stream reaches it.
 * Errors: EINVAL (n out of range, NULL pointer), ECUDA. */
int sfmm_reduce_noalloc(int64_t n, const double* mass, const double* acc, const double* pot, double* out,
                        void* stream);

/* Measured fused-multiply-add throughput of device `device` (a measurement
 * aid for the arithmetic rooflines of the near-field and M2L kernels; the
 * paper has no counterpart).  A kernel of eight independent FMA chains per
 * thread, 32 warps on every SM, in form
 *   0: FP64 fma,  1: FP32 fma,  2: packed FP32 (two fmas per instruction),
 * calibrated to last about target_ms (0 < target_ms <= 1000) per launch and
 * timed with CUDA events on `stream` (cudaStream_t, NULL: default stream);
 * the best of `reps` launches (1..1000) gives *tflops (2 flops per fma) and
 * *ms (its duration; may be NULL).  Allocates a small scratch buffer for the
 * duration of the call.  Errors: EINVAL (bad argument or device), ECUDA. */
int sfmm_fma_peak(int device, int form, void* stream, double target_ms, int reps, double* tflops, double* ms);

/* Message describing an error code. */
const char* sfmm_strerror(int code);

/* Last error message recorded by this context (never NULL). */
const char* sfmm_last_error(const sfmm_ctx* ctx);

/* Library version string. */
const char* sfmm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SFMM_H */
