// Shared-interaction walk: the pairs of Algorithm 2 evaluated once per node
// instead of once per leaf below it.
//
// In the per-leaf replay (Algorithm 1) the pairs whose target is a branch
// node c_k depend only on c_k, not on the leaf: a pair (c_k, s) opened at an
// internal c_k is pushed as (c_{k+1}, .) whichever child c_{k+1} is, so both
// children of a node receive the same opened list.  Processing the tree
// level by level, one warp per node, therefore visits every pair exactly once
// -- the caching of shared long-range interactions suggested in Sect. 5 --
// and yields the same interactions, hence the same result up to the order of
// summation.  The inherited coefficients are translated once per node
// (T(A) = shift(T(parent)) + C(A), Eq. gravmtranslat) and evaluated at the
// leaves (L2P).  Leaves run the lowering of Algorithm 2 and emit their
// neighbour lists exactly as in the per-leaf replay.
#include "walk_common.cuh"

namespace sfmm {

struct LevelArgs {
  WalkArgs w;
  int level;
  const int* level_nodes;
  int level_begin, level_count;
  const int* nparent;
  const int* nlu;
  const uint32_t* leaf_index;  // exclusive scan of leaf flags: leaf number of a leaf node
  const int* cf_in;            // opened lists of the internal nodes
  const long long* cf_off;
  const int* cf_cnt;
  int* cf_out;
  long long* cf_off_out;
  int* cf_cnt_out;
  unsigned long long* cf_counter;
  long long cf_cap;
  float* T32;                  // node coefficients: hi/lo pairs (FP32 form)
  double* T64;                 // node coefficients (FP64 form)
  int tstride;                 // coefficients per node (padded)
  // mode 2 (one-sided symmetric pairs): node depths, each node's own sums and
  // the sums its partners sent it (FP64, tstride per node)
  const int* ndepth;
  double* Cown;
  double* Erecv;
  // queue walks (schedules 2 and 3): items in order of readiness (-1: not
  // yet filled), slots handed out by q_head, filled through q_tail; q_total
  // items in all (an upper bound on the host: the kernels count them from
  // the build's counts)
  int* queue;          // pair queue: one int per item
  long long* queue64;  // node queue: (walk parent + 1) << 32 | node
  int* q_head;
  int* q_tail;
  int q_total;
  // the build's node and leaf counts on the device (the queue walks size
  // their work from them, so a captured graph follows every rebuild)
  const uint32_t* counts;
  int nsys;
};

// Data a parent's warp wrote earlier in the same launch (the queue walk) is
// read through L2; written by an earlier launch, a plain load may use L1.
template <typename T>
__device__ __forceinline__ T ld_parent(const T* p, bool l2) {
  return l2 ? __ldcg(p) : *p;
}

// Bounded wait of the queue walk for a slot to be filled: about a second,
// then the walk reports an internal error instead of waiting on.
#define SFMM_QUEUE_SPIN (1 << 24)


// T(A) = shift(T(parent)) + own: the parent's coefficients translated to A's
// centre (Eq. gravmtranslat, lane-parallel through the shift table) plus A's
// own sums (own_lo: low parts of a double-float own sum, or zeros).  Stored
// for an internal node; returned in Tn (+ Tl) for a leaf.
template <int P, bool F32, bool LO, bool L2 = false>
__device__ __forceinline__ void node_coefficients(const LevelArgs& la, int A, int par, bool leafA, const float4& hiA,
                                                  const float4& loA, double cAx, double cAy, double cAz,
                                                  const typename std::conditional<F32, float, double>::type* lev,
                                                  const float* lev_lo,
                                                  typename std::conditional<F32, float, double>::type* Tn,
                                                  float* Tl, typename std::conditional<F32, float, double>::type* sT,
                                                  typename std::conditional<F32, float, double>::type* sH,
                                                  const signed char* s_tab, int lane) {
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int NC = E::NC;
  constexpr int NCS = (NC + 31) / 32;
  const WalkArgs& a = la.w;
#pragma unroll
  for (int b = 0; b < NCS; ++b) {
    Tn[b] = R(0);
    Tl[b] = 0.0f;
  }
  if (par >= 0) {
    const float4 hiP = a.geo_hi[par], loP = a.geo_lo[par];
#pragma unroll
    for (int b = 0; b < NCS; ++b) {
      const int j = lane + 32 * b;
      if constexpr (F32) {
        Tn[b] = ld_parent(&la.T32[2 * ((size_t)par * la.tstride + j)], L2);
        Tl[b] = ld_parent(&la.T32[2 * ((size_t)par * la.tstride + j) + 1], L2);
      } else {
        Tn[b] = ld_parent(&la.T64[(size_t)par * la.tstride + j], L2);
      }
      sT[j] = Tn[b];
    }
    if (lane == 0) {
      R hx, hy, hz;
      if constexpr (F32) {
        hx = df_diff(hiA.x, loA.x, hiP.x, loP.x);
        hy = df_diff(hiA.y, loA.y, hiP.y, loP.y);
        hz = df_diff(hiA.z, loA.z, hiP.z, loP.z);
      } else {
        hx = cAx - a.ncx[par];
        hy = cAy - a.ncy[par];
        hz = cAz - a.ncz[par];
      }
      R hm[E::NMONO1];
      E::mono1(hx, hy, hz, hm);
#pragma unroll
      for (int t = 0; t < E::NMONO1; ++t) sH[t] = hm[t];
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < NCS; ++b) {
      const int j = lane + 32 * b;
      if (j < NC) {
        R corr = R(0);
        const signed char* row = s_tab + j * NC;
        for (int i = 0; i < NC; ++i) {
          const int t = row[i];
          if (t > 0) corr = fma(sH[t], sT[i], corr);
        }
        if constexpr (F32) {
          dfloat r = df_add_f(dfloat{Tn[b], Tl[b]}, corr);
          Tn[b] = r.hi;
          Tl[b] = r.lo;
        } else {
          Tn[b] += corr;
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int b = 0; b < NCS; ++b) {
    const int j = lane + 32 * b;
    if constexpr (F32) {
      dfloat r = df_add_f(dfloat{Tn[b], Tl[b]}, lev[b]);
      if constexpr (LO) r = df_add_f(r, lev_lo[b]);
      Tn[b] = r.hi;
      Tl[b] = r.lo;
      if (!leafA) {
        la.T32[2 * ((size_t)A * la.tstride + j)] = Tn[b];
        la.T32[2 * ((size_t)A * la.tstride + j) + 1] = Tl[b];
      }
    } else {
      Tn[b] += lev[b];
      if (!leafA) la.T64[(size_t)A * la.tstride + j] = Tn[b];
    }
  }
}

// Evaluation of a leaf's coefficients at its particles (L2P, Eq. 16 / 28).
template <int P, bool F32>
__device__ __forceinline__ void leaf_l2p(const LevelArgs& la, int A, double cAx, double cAy, double cAz,
                                         const typename std::conditional<F32, float, double>::type* Tn,
                                         const float* Tl, typename std::conditional<F32, float, double>::type* sT,
                                         int lane) {
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int NCS = (E::NC + 31) / 32;
  const WalkArgs& a = la.w;
  const int fL = a.nfirst[A], nL = a.ncount[A];
#pragma unroll
  for (int b = 0; b < NCS; ++b) {
    if constexpr (F32) sT[lane + 32 * b] = Tn[b] + Tl[b];
    else sT[lane + 32 * b] = Tn[b];
  }
  __syncwarp();
  for (int t = lane; t < nL; t += 32) {
    const int i = fL + t;
    R ax, ay, az;
    if constexpr (F32) {
      const float4 p = a.prel[i];
      ax = p.x;
      ay = p.y;
      az = p.z;
    } else {
      ax = a.px[i] - cAx;
      ay = a.py[i] - cAy;
      az = a.pz[i] - cAz;
    }
    R am[E::NQ], o4[4];
    E::mono(ax, ay, az, am);
    E::l2p(am, &sT[0], o4);
    if constexpr (F32) a.far32[i] = make_float4(o4[1], o4[2], o4[3], -o4[0]);
    else {
      a.far64[4 * (size_t)i] = o4[1];
      a.far64[4 * (size_t)i + 1] = o4[2];
      a.far64[4 * (size_t)i + 2] = o4[3];
      a.far64[4 * (size_t)i + 3] = -o4[0];
    }
  }
}

#include "walk_pair.cuh"

// Blocks per SM (FP32, p <= 2): 5 for the queue walk, 4 per depth -- measured:
// the queue walk gains from the fifth block despite a few spilled registers,
// the per-depth walk loses.
template <int P, bool F32, bool SYM, bool QUEUE>
__global__ void __launch_bounds__(WALK_NT, (P <= 2 && F32) ? (QUEUE ? 5 : 4) : 1) k_walk_level(const LevelArgs la) {
  static_assert(!(SYM && QUEUE), "the queue walk runs walk mode 1 only");
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int NC = E::NC;
  constexpr int NCS = (NC + 31) / 32;
  const WalkArgs& a = la.w;

  __shared__ int s_queue[WALK_WARPS][WALK_MQ];
  __shared__ float4 s_qr[WALK_WARPS][F32 ? WALK_MQ : 1];  // accepted pairs' separation s_B - s_A
  __shared__ R s_T[WALK_WARPS][NCS * 32];
  __shared__ R s_h[WALK_WARPS][E::NMONO1];
  __shared__ signed char s_tab[NC * NC];
  {
    const signed char* tab = E::table();
    for (int t = threadIdx.x; t < NC * NC; t += WALK_NT) s_tab[t] = tab[t];
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int gw = blockIdx.x * WALK_WARPS + warp;
  const int cap = a.ring_cap;
  int* const stk = a.ring + (size_t)gw * 2 * cap;  // lowering stack (leaves)
  int* const out = stk + cap;                      // child frontier / neighbour list

  unsigned long long st_m2l = 0, st_uniq = 0, st_pl = 0;
  unsigned long long st_m2l_p = 0;  // mode 2: replicated count of the partner sides, per lane
  int st_fb = 0;

  // queue walk: an internal node hands its right child on through the queue
  // once everything the child reads (coefficients, opened list) is written,
  // and goes on with its left child itself (no queue round trip, no wait:
  // the warp wrote what the child reads); when both children are leaves it
  // takes both and queues neither
  constexpr bool queue = QUEUE;
  int next = -1, next2 = -1, next_par = -1;  // queue walk: the children this warp takes next
  auto push_children = [&](int node, int right, bool two_leaves) {
    if constexpr (queue) {
      if (!two_leaves) {
        __threadfence();
        __syncwarp();
        if (lane == 0) {
          // the entry carries the parent, so that the child reads the
          // parent's list without first looking the parent up
          const int t = atomicAdd(la.q_tail, 1);
          la.queue64[t] = ((long long)(node + 1) << 32) | (unsigned)right;
        }
      }
      next = node + 1;
      next2 = two_leaves ? right : -1;
      next_par = node;
    }
  };
  // queue walk: the system roots and the right child of every walkable
  // internal node whose children are not both leaves (walkable: all but the
  // nsys - 1 nodes spanning systems; a full binary tree per system):
  // counts[0] + 1 - counts[1] - counts[2] items
  const int q_total = queue ? (int)la.counts[0] + 1 - (int)la.counts[1] - (int)la.counts[2] : 0;
  while (true) {
    int A, par;
    if (queue && next >= 0) {
      par = next_par;
      A = next;
      next = next2;
      next2 = -1;
    } else if constexpr (queue) {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(la.q_head, 1);
      slot = __shfl_sync(SFMM_FULL, slot, 0);
      if (slot >= q_total) break;
      long long got = -1;
      if (lane == 0) {
        for (int it = 0; it < SFMM_QUEUE_SPIN; ++it) {
          got = *reinterpret_cast<volatile long long*>(la.queue64 + slot);
          if (got >= 0) break;
          __nanosleep(64);
        }
      }
      got = __shfl_sync(SFMM_FULL, got, 0);
      if (got < 0) {
        if (lane == 0) set_status(a.status, SFMM_ST_INTERNAL);
        break;
      }
      __threadfence();
      A = (int)(got & 0xffffffffLL);
      par = (int)(got >> 32) - 1;
    } else {
      int idx = 0;
      if (lane == 0) idx = atomicAdd(a.leaf_counter, 1);
      idx = __shfl_sync(SFMM_FULL, idx, 0);
      if (idx >= la.level_count) break;
      A = la.level_nodes[la.level_begin + idx];
      par = la.nparent[A];
    }
    const int rA = a.nright[A];
    const bool leafA = rA < 0;
    // (queue walk) whether both children are leaves: loaded now, used at the end
    bool two_leaves = false;
    if (queue && !leafA) two_leaves = a.nright[A + 1] < 0 && a.nright[rA] < 0;
    const float4 hiA = a.geo_hi[A], loA = a.geo_lo[A];
    double cAx = 0.0, cAy = 0.0, cAz = 0.0;
    if (!F32) {
      cAx = a.ncx[A];
      cAy = a.ncy[A];
      cAz = a.ncz[A];
    }
    // the opened list inherited from the parent (a system's root starts from
    // itself), read in order; a leaf's lowering pushes the pairs it opens on
    // the warp's stack and pops them after the inherited list
    const int* fin = nullptr;
    int nF = 1;
    if (par >= 0) {
      // written by the parent's warp: read through L2 (the queue walk runs
      // parent and child in the same launch)
      fin = la.cf_in + ld_parent(&la.cf_off[par], queue);
      nF = ld_parent(&la.cf_cnt[par], queue);
    }
    int head = 0, sp = 0, nn = 0;
    bool bad = false;
    // an internal node writes the list its children inherit straight into the
    // arena: every opened pair yields at most two entries
    int* cfw = nullptr;
    unsigned long long cfbase = 0;
    if (!leafA) {
      if (lane == 0) cfbase = atomicAdd(la.cf_counter, 2ull * (unsigned long long)nF);
      cfbase = __shfl_sync(SFMM_FULL, cfbase, 0);
      if ((long long)(cfbase + 2ull * nF) > la.cf_cap) {
        if (lane == 0) {
          set_status(a.status, SFMM_ST_CHILDLIST);
          la.cf_cnt_out[A] = 0;
        }
        push_children(A, rA, two_leaves);
        continue;
      }
      cfw = la.cf_out + cfbase;
    }
    R C[NCS * 32];
#pragma unroll
    for (int t = 0; t < NCS * 32; ++t) C[t] = R(0);
    int nq = 0, nacc_tot = 0;
    int rankA = 0;
    R QA[SYM ? (F32 ? ((E::NQ + 3) / 4) * 4 : E::NQ) : 1];
    if constexpr (SYM) {
      rankA = leafA ? INT_MAX : la.ndepth[A];
      if constexpr (F32) {
        const float4* q4 = reinterpret_cast<const float4*>(a.Qf + (size_t)A * a.nqs);
#pragma unroll
        for (int t = 0; t < (E::NQ + 3) / 4; ++t) {
          const float4 v = __ldg(q4 + t);
          QA[4 * t] = v.x;
          QA[4 * t + 1] = v.y;
          QA[4 * t + 2] = v.z;
          QA[4 * t + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < E::NQ; ++t) QA[t] = __ldg(a.Qd + (size_t)A * E::NQ + t);
      }
    }
    // the inherited list is read through a two-stage pipeline: ids one chunk
    // ahead of the node records, records one chunk ahead of their use, so the
    // loads of a chunk overlap the work on the previous one
    auto fin_id = [&](int at) -> int { return (at + lane < nF) ? (fin ? ld_parent(fin + at + lane, queue) : A) : -1; };
    int pf_s = fin_id(0), pf_s2 = fin_id(32), pf_r = -1;
    float4 pf_hi = make_float4(0.f, 0.f, 0.f, 0.f), pf_lo = pf_hi;
    if (pf_s >= 0) {
      pf_hi = a.geo_hi[pf_s];
      pf_lo = a.geo_lo[pf_s];
      pf_r = a.nright[pf_s];
    }
    while (!bad) {
      const bool from_fin = head < nF;
      const bool more = from_fin || sp > 0;
      if (more) {
        int s, rB = -1;
        float4 hiB = make_float4(0.f, 0.f, 0.f, 0.f), loB = hiB;
        if (from_fin) {
          s = pf_s;
          hiB = pf_hi;
          loB = pf_lo;
          rB = pf_r;
          head += min(32, nF - head);
          pf_s = pf_s2;
          if (pf_s >= 0) {
            pf_hi = a.geo_hi[pf_s];
            pf_lo = a.geo_lo[pf_s];
            pf_r = a.nright[pf_s];
          }
          pf_s2 = fin_id(head + 32);
        } else {
          const int cnt = min(32, sp);
          s = (lane < cnt) ? stk[sp - cnt + lane] : -1;
          sp -= cnt;
          if (s >= 0) {
            hiB = a.geo_hi[s];
            loB = a.geo_lo[s];
            rB = a.nright[s];
          }
        }
        bool acc = false, open = false;
        float rx = 0.f, ry = 0.f, rz = 0.f;
        if (s >= 0) {
          if (s == A) open = true;
          else {
            acc = decide(hiA, loA, hiB, loB, A, s, a, st_fb, rx, ry, rz);
            open = !acc;
          }
        }
        if constexpr (SYM) {
          // the node processed first evaluates the pair for both sides
          // (leaves run last; ties within a launch go to the smaller id)
          if (acc) {
            const int rankB = rB < 0 ? INT_MAX : la.ndepth[s];
            acc = rankA < rankB || (rankA == rankB && A < s);
          }
        }
        const unsigned bacc = __ballot_sync(SFMM_FULL, acc);
        const int nacc = __popc(bacc);
        nacc_tot += nacc;
        if (acc) {
          const int q = nq + __popc(bacc & lt);
          s_queue[warp][q] = s;
          if constexpr (F32) s_qr[warp][q] = make_float4(rx, ry, rz, 0.f);
        }
        nq += nacc;
        const bool sleaf = open && rB < 0;
        const bool sint = open && rB >= 0;
        if (!leafA) {
          const unsigned b1 = __ballot_sync(SFMM_FULL, open), b2 = __ballot_sync(SFMM_FULL, sint);
          const int add = __popc(b1) + __popc(b2);
          if (open) {
            const int pos = nn + __popc(b1 & lt) + __popc(b2 & lt);
            if (sleaf) cfw[pos] = s;
            else {
              cfw[pos] = s + 1;
              cfw[pos + 1] = rB;
            }
          }
          nn += add;
        } else {
          const unsigned bl = __ballot_sync(SFMM_FULL, sleaf), bi = __ballot_sync(SFMM_FULL, sint);
          const int addl = __popc(bl), addi = 2 * __popc(bi);
          if (nn + addl > cap || sp + addi > cap) {
            bad = true;
          } else {
            if (sleaf) out[nn + __popc(bl & lt)] = s;
            if (sint) {
              const int cp = sp + 2 * __popc(bi & lt);
              stk[cp] = s + 1;
              stk[cp + 1] = rB;
            }
          }
          nn += addl;
          sp += addi;
        }
        __syncwarp();
        if (bad) break;
      }
      while (nq >= 32 || (!more && nq > 0)) {
        const int take = min(nq, 32);
        const int src = (lane < take) ? s_queue[warp][nq - take + lane] : -1;
        float4 rq = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (F32) {
          if (lane < take) rq = s_qr[warp][nq - take + lane];
        }
        __syncwarp();
        if constexpr (SYM) {
          if (src >= 0) {
            m2l_eval_sym<P, F32>(src, cAx, cAy, cAz, a, C, rq, QA, la.Erecv + (size_t)src * la.tstride);
            st_m2l_p += (unsigned long long)la.nlu[src];
          }
        } else {
          m2l_eval<P, F32>(src, hiA, loA, cAx, cAy, cAz, a, C, rq);
        }
        nq -= take;
      }
      if (!more) break;
    }
    if (bad) {
      // leave empty lists behind so that nothing downstream reads stale offsets
      if (lane == 0) {
        set_status(a.status, SFMM_ST_RING);
        if (leafA) a.p2p_cnt[la.leaf_index[A]] = 0;
        else la.cf_cnt_out[A] = 0;
      }
      if (!leafA) push_children(A, rA, two_leaves);
      continue;
    }
    if (lane == 0) {
      st_uniq += (SYM ? 2ull : 1ull) * nacc_tot;
      st_m2l += (unsigned long long)nacc_tot * la.nlu[A];
    }

    // coefficients of A: own level sum plus the parent's, translated
    R lev[NCS];
#pragma unroll
    for (int b = 0; b < NCS; ++b) {
      R v[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) v[t] = C[32 * b + t];
      lev[b] = reduce_scatter32(v, lane);
    }
    R Tn[NCS];
    float Tl[NCS];
    if constexpr (SYM) {
      // own sums to the node's slot; the finalize pass adds the parent's
      // translated coefficients and the sums received from partners
#pragma unroll
      for (int b = 0; b < NCS; ++b) la.Cown[(size_t)A * la.tstride + lane + 32 * b] = (double)lev[b];
    } else {
      node_coefficients<P, F32, false, QUEUE>(la, A, par, leafA, hiA, loA, cAx, cAy, cAz, lev, nullptr, Tn, Tl, s_T[warp],
                                       s_h[warp], s_tab, lane);
    }

    if (!leafA) {
      // the opened list both children inherit, already in the arena
      if (lane == 0) {
        la.cf_off_out[A] = (long long)cfbase;
        la.cf_cnt_out[A] = nn;
      }
      __syncwarp();
      push_children(A, rA, two_leaves);
      continue;
    }

    // leaf: L2P (mode 2: in the finalize pass), then its neighbour list
    const int leaf = (int)la.leaf_index[A];
    if constexpr (!SYM) leaf_l2p<P, F32>(la, A, cAx, cAy, cAz, Tn, Tl, s_T[warp], lane);
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.arena_counter, (unsigned long long)nn);
    base = __shfl_sync(SFMM_FULL, base, 0);
    if ((long long)(base + nn) > a.arena_cap) {
      if (lane == 0) {
        set_status(a.status, SFMM_ST_ARENA);
        a.p2p_cnt[leaf] = 0;
      }
    } else {
      // (the pair count is taken by the near-field pass, which loads the counts anyway)
      for (int t = lane; t < nn; t += 32) a.arena[base + t] = out[t];
      if (lane == 0) {
        a.p2p_off[leaf] = (long long)base;
        a.p2p_cnt[leaf] = nn;
        st_pl += nn;
        if (nn > a.chunk) {
          atomicAdd(a.split_counter, (unsigned long long)((nn + a.chunk - 1) / a.chunk));
          atomicAdd(a.split_counter + 1, 1ull);
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) st_fb += __shfl_xor_sync(SFMM_FULL, st_fb, o);
  if constexpr (SYM) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) st_m2l_p += __shfl_xor_sync(SFMM_FULL, st_m2l_p, o);
    st_m2l += st_m2l_p;
  }
  if (lane == 0) {
    atomicAdd(&a.stat[0], st_m2l);
    atomicAdd(&a.stat[1], st_uniq);
    atomicAdd(&a.stat[2], st_pl);
    atomicAdd(&a.stat[4], (unsigned long long)st_fb);
  }
}

// Mode 2, per level after its walk launch: every node's coefficients are
// the parent's translated ones plus its own sums plus the sums its partners
// sent it (all partners of a node are processed no later than its own
// launch); internal nodes store them, leaves evaluate them (L2P).
template <int P, bool F32>
__global__ void __launch_bounds__(WALK_NT) k_walk_finalize(const LevelArgs la, int* __restrict__ counter) {
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int NC = E::NC;
  constexpr int NCS = (NC + 31) / 32;
  const WalkArgs& a = la.w;
  __shared__ R s_T[WALK_WARPS][NCS * 32];
  __shared__ R s_h[WALK_WARPS][E::NMONO1];
  __shared__ signed char s_tab[NC * NC];
  {
    const signed char* tab = E::table();
    for (int t = threadIdx.x; t < NC * NC; t += WALK_NT) s_tab[t] = tab[t];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(counter, 1);
    idx = __shfl_sync(SFMM_FULL, idx, 0);
    if (idx >= la.level_count) break;
    const int A = la.level_nodes[la.level_begin + idx];
    const bool leafA = a.nright[A] < 0;
    const int par = la.nparent[A];
    const float4 hiA = a.geo_hi[A], loA = a.geo_lo[A];
    double cAx = 0.0, cAy = 0.0, cAz = 0.0;
    if (!F32) {
      cAx = a.ncx[A];
      cAy = a.ncy[A];
      cAz = a.ncz[A];
    }
    R lev[NCS];
    float lev_lo[NCS];
#pragma unroll
    for (int b = 0; b < NCS; ++b) {
      const size_t j = (size_t)A * la.tstride + lane + 32 * b;
      const double v = la.Cown[j] + la.Erecv[j];
      if constexpr (F32) {
        float hi, lo;
        split_double(v, hi, lo);
        lev[b] = hi;
        lev_lo[b] = lo;
      } else {
        lev[b] = v;
        lev_lo[b] = 0.0f;
      }
    }
    R Tn[NCS];
    float Tl[NCS];
    node_coefficients<P, F32, F32>(la, A, par, leafA, hiA, loA, cAx, cAy, cAz, lev, lev_lo, Tn, Tl, s_T[warp],
                                   s_h[warp], s_tab, lane);
    if (leafA) leaf_l2p<P, F32>(la, A, cAx, cAy, cAz, Tn, Tl, s_T[warp], lane);
    __syncwarp();
  }
}

// Queue walk: the system roots (no walk parent) fill the first slots.
__global__ void k_queue_seed(int nsys, const int* __restrict__ sys_root, long long* __restrict__ queue,
                             int* __restrict__ tail) {
  for (int i = threadIdx.x; i < nsys; i += blockDim.x) queue[i] = (long long)(unsigned)sys_root[i];
  if (threadIdx.x == 0) *tail = nsys;
}

template <int P, bool F32, bool SYM>
static int run_levels(sfmm_ctx* c, double theta, int order) {
  using E = Exp<P>;
  constexpr int NCS = (E::NC + 31) / 32;
  const int nn = c->nnodes, nl = c->nleaves;
  int per_sm = 0, q_per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_level<P, F32, SYM, false>, WALK_NT, 0);
  int p_per_sm = 0;
  if (!SYM) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q_per_sm, k_walk_level<P, F32, false, true>, WALK_NT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p_per_sm, k_walk_pair<P, F32>, WALK_NT, 0);
  }
  if (per_sm < 1) per_sm = 1;
  if (q_per_sm < 1) q_per_sm = 1;
  if (p_per_sm < 1) p_per_sm = 1;
  const int max_blocks = per_sm * num_sms(c->device);
  const int tstride = NCS * 32;
  // schedule (walk mode 1; bitwise the same results): 1 one launch per
  // depth; 2 readiness queue of nodes; 3 readiness queue of sibling pairs
  // (each record load serves both children's decisions, at fewer warps per
  // SM); 0 chooses 2 while the walk's records (geometry, moments,
  // coefficients, list offsets) take at most twice the L2, else 3
  // (measured on GB300: 2 is faster on the 10^6 Plummer sphere, 1.21 against
  // 1.32 ms, records 64 MB, and on the 2x10^6 binary, 2.11 against 2.17 ms,
  // records 127 MB; 3 on the 1.6x10^7 cloud, 16.3 against 17.4 ms, 1 GB)
  int sched = SYM ? 1 : c->schedule;
  if (sched == 0) {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess) l2 = 0;
    // geometry and right child (36 B), list offset and count (12 B),
    // moments, coefficients
    const size_t mom = F32 ? 4 * (size_t)((ncoef(order) + 3) & ~3) : 24 + 8 * (size_t)E::NQ;
    const size_t per_node = 48 + mom + 8 * (size_t)tstride;
    sched = ((double)per_node * nn <= 2.0 * (double)l2) ? 2 : 3;
  }
  // a captured step runs on the counts of each replay's own build: node- and
  // leaf-indexed buffers are sized for the bounds (2n nodes, n leaves), and
  // only the queue schedules (which need no host-side level lists) run
  if (c->graph_mode && sched == 1) sched = 2;
  const int nn_b = c->graph_mode ? (int)std::min<int64_t>(2 * c->n, INT32_MAX) : nn;
  const int nl_b = c->graph_mode ? (int)c->n : nl;
  const bool queue = sched >= 2, pairs = sched == 3;
  const int q_blocks = (pairs ? p_per_sm : q_per_sm) * num_sms(c->device);
  int rc;
  // per-depth launches (and the symmetric walk) run over the per-depth lists
  if (!queue && (rc = ensure_levels(c)))
    return set_error(c, rc, rc == SFMM_ESTACK ? "tree deeper than supported" : "per-depth node lists failed");
  {
    // one ring per resident warp (the pair walk keeps both children's stacks
    // and lists and the second child's set-aside batches)
    const size_t ring_ints = pairs ? (size_t)q_blocks * WALK_WARPS * WALK_PAIR_RING * c->ring_capacity
                                   : (size_t)(queue ? q_blocks : max_blocks) * WALK_WARPS * 2 * c->ring_capacity;
    if ((rc = c->ring.ensure(sizeof(int) * ring_ints))) return rc;
    long long arena_cap = c->list_capacity > 0 ? c->list_capacity : (long long)nl * 96 + 1024;
    if ((rc = c->arena.ensure(sizeof(int) * (size_t)arena_cap))) return rc;
    arena_cap = (long long)(c->arena.bytes / sizeof(int));
    // the opened lists of every internal node are kept until the leaves run
    long long cf_cap = c->cf_capacity > 0 ? c->cf_capacity : (long long)nn * 256 + 4096;
    if ((rc = c->cf_arena.ensure(sizeof(int) * (size_t)cf_cap))) return rc;
    cf_cap = (long long)(c->cf_arena.bytes / sizeof(int));
    if ((rc = c->cf_off.ensure(sizeof(long long) * (size_t)nn_b))) return rc;
    if ((rc = c->cf_cnt.ensure(sizeof(int) * (size_t)nn_b))) return rc;
    if ((rc = c->Tnode.ensure((F32 ? 2 * sizeof(float) : sizeof(double)) * (size_t)nn_b * tstride))) return rc;
    if (SYM) {
      if ((rc = c->sym_own.ensure(sizeof(double) * (size_t)nn * tstride)) ||
          (rc = c->sym_recv.ensure(sizeof(double) * (size_t)nn * tstride)))
        return rc;
      SFMM_CUDA_TRY(cudaMemsetAsync(c->sym_recv.p, 0, sizeof(double) * (size_t)nn * tstride, c->stream));
    }
    if ((rc = c->p2p_off.ensure(sizeof(long long) * (size_t)nl_b))) return rc;
    if ((rc = c->p2p_cnt.ensure(sizeof(int) * (size_t)nl_b))) return rc;
    // empty lists until a leaf writes its own: the near field runs before the
    // status is read, and a walk cut short must leave no stale list behind
    SFMM_CUDA_TRY(cudaMemsetAsync(c->p2p_cnt.p, 0, sizeof(int) * (size_t)nl_b, c->stream));
    const int nlev = queue ? 0 : c->max_depth + 1;  // levels holding internal nodes
    if ((rc = c->counters.ensure(sizeof(unsigned long long) * (20 + 2 * (size_t)nlev)))) return rc;
    if ((rc = c->far.ensure((F32 ? sizeof(float4) : 4 * sizeof(double)) * (size_t)c->n))) return rc;
    unsigned long long* ctr = c->counters.as<unsigned long long>();
    SFMM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * (20 + 2 * (size_t)nlev), c->stream));

    LevelArgs la{};
    WalkArgs& a = la.w;
    a.nleaves = nl;
    a.leaf_node = c->leaf_node.as<int>();
    a.nfirst = c->nfirst.as<int>();
    a.ncount = c->ncount.as<int>();
    a.nright = c->nright.as<int>();
    a.geo_hi = c->geo_hi.as<float4>();
    a.geo_lo = c->geo_lo.as<float4>();
    a.ncx = c->ncx.as<double>();
    a.ncy = c->ncy.as<double>();
    a.ncz = c->ncz.as<double>();
    a.nsize = c->nsize.as<double>();
    a.nhmax = c->nhmax.as<double>();
    a.Qf = c->Qf.as<float>();
    a.Qd = c->Qd.as<double>();
    a.nqs = (ncoef(order) + 3) & ~3;
    a.prel = c->prel.as<float4>();
    a.px = c->px.as<double>();
    a.py = c->py.as<double>();
    a.pz = c->pz.as<double>();
    a.ring = c->ring.as<int>();
    a.ring_cap = c->ring_capacity;
    a.arena = c->arena.as<int>();
    a.arena_counter = ctr + 9;
    a.split_counter = ctr + 5;
    a.chunk = c->p2p_chunk;
    a.arena_cap = arena_cap;
    a.p2p_off = c->p2p_off.as<long long>();
    a.p2p_cnt = c->p2p_cnt.as<int>();
    a.far32 = c->far.as<float4>();
    a.far64 = c->far.as<double>();
    a.status = c->d_status;
    a.stat = ctr;
    a.theta = theta;
    a.theta_f = (float)theta;
    a.theta2_f = (float)(theta * theta);
    la.nparent = c->wparent.as<int>();  // -1 at system roots
    la.nlu = c->nlu.as<int>();
    la.leaf_index = c->isleaf.as<uint32_t>();
    la.cf_cap = cf_cap;
    la.T32 = c->Tnode.as<float>();
    la.T64 = c->Tnode.as<double>();
    la.tstride = tstride;
    la.cf_in = c->cf_arena.as<int>();
    la.cf_off = c->cf_off.as<long long>();
    la.cf_cnt = c->cf_cnt.as<int>();
    la.cf_out = c->cf_arena.as<int>();
    la.cf_off_out = c->cf_off.as<long long>();
    la.cf_cnt_out = c->cf_cnt.as<int>();
    la.cf_counter = ctr + 16;
    la.ndepth = c->ndepth.as<int>();
    la.Cown = SYM ? c->sym_own.as<double>() : nullptr;
    la.Erecv = SYM ? c->sym_recv.as<double>() : nullptr;
    la.queue = nullptr;
    if (queue) {
      // one launch: a warp takes the next slot of the queue and waits until
      // the item there has been pushed.  Node queue: the system roots first,
      // then the right child of every walkable internal node (its left child
      // goes on in the parent's warp).  Pair queue: the system roots and the
      // children of every walkable internal node.  Both: nsys + (nn - nsys +
      // 1 - nl) = nn + 1 - nl items
      la.q_total = nn + 1 - nl;  // (the kernels take it from the counts)
      const int q_bound = c->graph_mode ? nn_b : la.q_total;
      if ((rc = c->wqueue.ensure(sizeof(long long) * (size_t)(q_bound + 1)))) return rc;
      la.queue = c->wqueue.as<int>();
      la.queue64 = c->wqueue.as<long long>();
      la.q_head = reinterpret_cast<int*>(ctr + 14);
      la.q_tail = reinterpret_cast<int*>(ctr + 15);
      la.counts = c->d_counts;
      la.nsys = c->nsys;
      SFMM_CUDA_TRY(cudaMemsetAsync(la.queue, 0xff, (pairs ? sizeof(int) : sizeof(long long)) * (size_t)q_bound,
                                    c->stream));
      if (pairs) k_queue_seed_pairs<<<1, 32, 0, c->stream>>>(c->nsys, c->sys_root.as<int>(), la.queue, la.q_tail);
      else k_queue_seed<<<1, 32, 0, c->stream>>>(c->nsys, c->sys_root.as<int>(), la.queue64, la.q_tail);
      la.level = 0;
      la.level_nodes = nullptr;
      la.level_begin = 0;
      la.level_count = la.q_total;
      if (la.q_total > 0 || c->graph_mode) {
        // one block per resident slot (the queue needs none resident: a warp
        // only takes a slot while it runs, and a node's parent always holds
        // an earlier slot)
        if (pairs) k_walk_pair<P, F32><<<q_blocks, WALK_NT, 0, c->stream>>>(la);
        else k_walk_level<P, F32, false, true><<<q_blocks, WALK_NT, 0, c->stream>>>(la);
        ++c->nlaunch;
      }
      ++c->nlaunch;
      SFMM_CUDA_TRY(cudaGetLastError());
    }
    // internal nodes level by level (each needs its parent's opened list and
    // coefficients), then every leaf in one launch, shallowest first
    for (int k = 0; k <= nlev && !queue; ++k) {
      const bool leaves = (k == nlev);
      la.level = k;
      if (leaves) {
        la.level_nodes = c->leaf_order.as<int>();
        la.level_begin = 0;
        la.level_count = nl;
      } else {
        la.level_nodes = c->level_nodes.as<int>();
        la.level_begin = c->h_level_off[k];
        la.level_count = c->h_level_off[k + 1] - c->h_level_off[k];
      }
      if (la.level_count <= 0) continue;
      a.leaf_counter = reinterpret_cast<int*>(ctr + 18 + 2 * k);
      const int blocks = min(max_blocks, (la.level_count + WALK_WARPS - 1) / WALK_WARPS);
      k_walk_level<P, F32, SYM, false><<<blocks, WALK_NT, 0, c->stream>>>(la);
      ++c->nlaunch;
      if (SYM) {
        k_walk_finalize<P, F32><<<blocks, WALK_NT, 0, c->stream>>>(la, reinterpret_cast<int*>(ctr + 19 + 2 * k));
        ++c->nlaunch;
      }
      SFMM_CUDA_TRY(cudaGetLastError());
    }
    // no host wait here: the gravity call checks the status word once, after
    // the near field and the sums, and regrows and reruns on overflow
    c->walk_arena_cap = arena_cap;
    c->walk_cf_cap = cf_cap;
  }
  return SFMM_OK;
}

// Capacity overflow of the shared walk (status bits of the last run, its
// counters in hs): grow what ran out before the rerun.
int walk_shared_regrow(sfmm_ctx* c, int bits, const unsigned long long* hs) {
  if (bits & SFMM_ST_RING) c->ring_capacity = c->ring_capacity < (1 << 20) ? c->ring_capacity * 16 : (1 << 24);
  if (bits & SFMM_ST_ARENA) {
    const unsigned long long need = hs[9];
    const int64_t grown = 2 * c->walk_arena_cap, want = (int64_t)(need + need / 4 + 1024);
    c->list_capacity = want > grown ? want : grown;
  }
  if (bits & SFMM_ST_CHILDLIST) {
    // the count undercounts: a node that could not reserve skipped its
    // children's lists, so their descendants reserved less
    const unsigned long long need = hs[16];
    const int64_t grown = 4 * c->walk_cf_cap, want = 2 * (int64_t)need + 4096;
    c->cf_capacity = want > grown ? want : grown;
  }
  return SFMM_OK;
}

int run_walk_shared(sfmm_ctx* c, double theta, int order) {
  const bool f32 = c->precision == SFMM_FP32;
  const bool sym = c->walk_mode == 2;  // one-sided symmetric pairs
  switch (order) {
    case 0: return f32 ? (sym ? run_levels<0, true, true>(c, theta, order) : run_levels<0, true, false>(c, theta, order))
                : (sym ? run_levels<0, false, true>(c, theta, order) : run_levels<0, false, false>(c, theta, order));
    case 1: return f32 ? (sym ? run_levels<1, true, true>(c, theta, order) : run_levels<1, true, false>(c, theta, order))
                : (sym ? run_levels<1, false, true>(c, theta, order) : run_levels<1, false, false>(c, theta, order));
    case 2: return f32 ? (sym ? run_levels<2, true, true>(c, theta, order) : run_levels<2, true, false>(c, theta, order))
                : (sym ? run_levels<2, false, true>(c, theta, order) : run_levels<2, false, false>(c, theta, order));
    case 3: return f32 ? (sym ? run_levels<3, true, true>(c, theta, order) : run_levels<3, true, false>(c, theta, order))
                : (sym ? run_levels<3, false, true>(c, theta, order) : run_levels<3, false, false>(c, theta, order));
    case 4: return f32 ? (sym ? run_levels<4, true, true>(c, theta, order) : run_levels<4, true, false>(c, theta, order))
                : (sym ? run_levels<4, false, true>(c, theta, order) : run_levels<4, false, false>(c, theta, order));
    default: return SFMM_EINVAL;
  }
}

}  // namespace sfmm
