// Shared-interaction walk on a readiness queue of sibling pairs (walk mode 1,
// schedule 2; included by walk_shared.cu after its node helpers).
//
// Every queue item is a system root (value 2 root + 1) or the two children of
// an internal node P (value 2 P).  Both children of P inherit the same list,
// P's opened list (Algorithm 2 pushes an opened pair (c_k, s) as (c_{k+1}, .)
// whichever child c_{k+1} is), so one warp takes both: the inherited list is
// read once and every entry's node record serves the decisions of both
// children.  Each child keeps its own queue of accepted pairs with the
// per-node flush order (after each chunk, batches of the last 32); the
// batches are appended to the child's buffer in that order and evaluated
// when the child is finished, so both children's sums equal, bit for bit,
// those of the per-node walk.  Then each child runs its own lowering
// (leaves), gets its coefficients and, if internal, hands its own children on
// as one item.  The children are finished one after the other by the same
// code (a loop, not unrolled): the kernel stays small enough for the
// instruction cache, which an inlined copy per child overflowed (measured:
// instruction-fetch stalls led, and the walk took 2.09 ms instead of 1.30).
// (Included inside namespace sfmm.)
#pragma once

// Ring entries per warp of the pair walk, in units of ring_capacity: lowering
// stack and neighbour list of each child (4), each child's batches of
// accepted sources (2).
#define WALK_PAIR_RING 6

// One child of a pair: its node, geometry and running counts.
struct PairKid {
  int A;       // node (-1: absent, the second slot of a root item)
  int r;       // right child (-1: leaf)
  float4 hi, lo;
  double cx, cy, cz;  // centre (FP64 form)
  int* cfw;    // internal: where its children's inherited list goes
  long long cfbase;
  int nn;      // entries of that list / of the neighbour list (leaf)
  int sp;      // lowering stack depth (leaf)
  int nq;      // accepted pairs waiting in its queue
  int nacc;    // accepted pairs in all
  int nb;      // entries of its batches of accepted sources (32 per batch)
  bool bad;
};

// Decisions of one child for one chunk of 32 entries (one per lane): the
// acceptance test of Sect. 3; accepted pairs join the child's queue, opened
// ones its children's list (internal child) or its neighbour list and
// lowering stack (leaf child), exactly as in the per-node walk.  (The
// separation the test forms is formed again, identically, when the pair is
// evaluated.)
__device__ __forceinline__ void pair_decide(PairKid& k, int s, const float4& hiB, const float4& loB, int rB,
                                            const WalkArgs& a, int* s_queue, int* stk, int* out, int cap, unsigned lt,
                                            int& nfb) {
  bool acc = false, open = false;
  float rx = 0.f, ry = 0.f, rz = 0.f;
  if (k.A >= 0 && s >= 0) {
    if (s == k.A) open = true;
    else {
      acc = decide(k.hi, k.lo, hiB, loB, k.A, s, a, nfb, rx, ry, rz);
      open = !acc;
    }
  }
  const unsigned bacc = __ballot_sync(SFMM_FULL, acc);
  const int nacc = __popc(bacc);
  if (acc) s_queue[k.nq + __popc(bacc & lt)] = s;
  k.nq += nacc;
  k.nacc += nacc;
  const bool sleaf = open && rB < 0;
  const bool sint = open && rB >= 0;
  if (k.r >= 0) {
    const unsigned b1 = __ballot_sync(SFMM_FULL, open), b2 = __ballot_sync(SFMM_FULL, sint);
    if (open) {
      const int pos = k.nn + __popc(b1 & lt) + __popc(b2 & lt);
      if (sleaf) k.cfw[pos] = s;
      else {
        k.cfw[pos] = s + 1;
        k.cfw[pos + 1] = rB;
      }
    }
    k.nn += __popc(b1) + __popc(b2);
  } else {
    const unsigned bl = __ballot_sync(SFMM_FULL, sleaf), bi = __ballot_sync(SFMM_FULL, sint);
    const int addl = __popc(bl), addi = 2 * __popc(bi);
    if (k.nn + addl > cap || k.sp + addi > cap) {
      k.bad = true;
    } else {
      if (sleaf) out[k.nn + __popc(bl & lt)] = s;
      if (sint) {
        const int cp = k.sp + 2 * __popc(bi & lt);
        stk[cp] = s + 1;
        stk[cp + 1] = rB;
      }
    }
    k.nn += addl;
    k.sp += addi;
  }
}



template <int P, bool F32>
__global__ void __launch_bounds__(WALK_NT, (P <= 2 && F32) ? 4 : 1) k_walk_pair(const LevelArgs la) {
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int NC = E::NC;
  constexpr int NCS = (NC + 31) / 32;
  const WalkArgs& a = la.w;

  __shared__ int s_queue[WALK_WARPS][2][WALK_MQ];
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
  // per child q: lowering stack, neighbour list, batches of accepted sources
  int* const ring = a.ring + (size_t)gw * WALK_PAIR_RING * cap;
  auto stk_of = [&](int q) { return ring + (size_t)(2 * q) * cap; };
  auto out_of = [&](int q) { return ring + (size_t)(2 * q + 1) * cap; };
  auto bat_of = [&](int q) { return ring + (size_t)(4 + q) * cap; };

  unsigned long long st_m2l = 0, st_uniq = 0, st_pl = 0;
  int st_fb = 0;

  // an internal node hands its children on as one item once everything they
  // read (coefficients, opened list) is written
  auto push_item = [&](int node) {
    __threadfence();
    __syncwarp();
    if (lane == 0) {
      const int t = atomicAdd(la.q_tail, 1);
      la.queue[t] = 2 * node;
    }
  };
  auto init_kid = [&](PairKid& k) {
    k.r = -1;
    k.hi = k.lo = make_float4(0.f, 0.f, 0.f, 0.f);
    k.cx = k.cy = k.cz = 0.0;
    k.cfw = nullptr;
    k.cfbase = 0;
    k.nn = k.sp = k.nq = k.nacc = k.nb = 0;
    k.bad = false;
    if (k.A >= 0) {
      k.r = a.nright[k.A];
      k.hi = a.geo_hi[k.A];
      k.lo = a.geo_lo[k.A];
      if (!F32) {
        k.cx = a.ncx[k.A];
        k.cy = a.ncy[k.A];
        k.cz = a.ncz[k.A];
      }
    }
  };
  // a child whose buffers ran out: empty list behind, children handed on
  // (the walk is redone after regrowing)
  auto drop_kid = [&](const PairKid& k, int bits) {
    if (k.A < 0) return;
    if (lane == 0) {
      set_status(a.status, bits);
      if (k.r < 0) a.p2p_cnt[la.leaf_index[k.A]] = 0;
      else la.cf_cnt_out[k.A] = 0;
    }
    if (k.r >= 0) push_item(k.A);
  };
  // the last `take` queued pairs of child q as one batch of 32 (lane l holds
  // entry l, as in the per-node flush); false when the buffer is full
  auto append = [&](PairKid& k, int q, int take) -> bool {
    if (k.nb + 32 > cap) return false;
    bat_of(q)[k.nb + lane] = (lane < take) ? s_queue[warp][q][k.nq - take + lane] : -1;
    __syncwarp();
    k.nb += 32;
    k.nq -= take;
    return true;
  };

  // items: the system roots and the children of every walkable internal node
  const int q_total = (int)la.counts[0] + 1 - (int)la.counts[1];
  while (true) {
    // next item: a warp only takes a slot while it runs, and an item's slot
    // comes after its parent's, so the wait ends (bounded all the same)
    int slot = 0;
    if (lane == 0) slot = atomicAdd(la.q_head, 1);
    slot = __shfl_sync(SFMM_FULL, slot, 0);
    if (slot >= q_total) break;
    int got = -1;
    if (lane == 0) {
      for (int it = 0; it < SFMM_QUEUE_SPIN; ++it) {
        got = *reinterpret_cast<volatile int*>(la.queue + slot);
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
    const bool root = (got & 1) != 0;
    const int par = root ? -1 : (got >> 1);
    PairKid k0, k1;
    k0.A = root ? (got >> 1) : par + 1;
    k1.A = root ? -1 : a.nright[par];
    init_kid(k0);
    init_kid(k1);
    // the inherited list: the parent's opened list, written by the parent's
    // warp in this launch (read through L2); a root starts from itself
    const int* fin = nullptr;
    int nF = 1;
    if (!root) {
      fin = la.cf_in + __ldcg(&la.cf_off[par]);
      nF = __ldcg(&la.cf_cnt[par]);
    }
    // internal children write their children's lists straight into the
    // arena: every opened pair yields at most two entries
    const int need0 = (k0.A >= 0 && k0.r >= 0) ? 2 * nF : 0;
    const int need1 = (k1.A >= 0 && k1.r >= 0) ? 2 * nF : 0;
    if (need0 + need1 > 0) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(la.cf_counter, (unsigned long long)(need0 + need1));
      base = __shfl_sync(SFMM_FULL, base, 0);
      if ((long long)(base + need0 + need1) > la.cf_cap) {
        drop_kid(k0, SFMM_ST_CHILDLIST);
        drop_kid(k1, SFMM_ST_CHILDLIST);
        continue;
      }
      k0.cfbase = (long long)base;
      k1.cfbase = (long long)base + need0;
      k0.cfw = la.cf_out + k0.cfbase;
      k1.cfw = la.cf_out + k1.cfbase;
    }

    // the inherited list through a two-stage pipeline (ids one chunk ahead
    // of the node records, records one chunk ahead of their use); every
    // entry is decided for both children
    auto fin_id = [&](int at) -> int { return (at + lane < nF) ? (fin ? __ldcg(fin + at + lane) : k0.A) : -1; };
    int pf_s = fin_id(0), pf_s2 = fin_id(32), pf_r = -1;
    float4 pf_hi = make_float4(0.f, 0.f, 0.f, 0.f), pf_lo = pf_hi;
    if (pf_s >= 0) {
      pf_hi = a.geo_hi[pf_s];
      pf_lo = a.geo_lo[pf_s];
      pf_r = a.nright[pf_s];
    }
    bool bad = false;
    for (int head = 0; head < nF;) {
      const int s = pf_s, rB = pf_r;
      const float4 hiB = pf_hi, loB = pf_lo;
      head += min(32, nF - head);
      pf_s = pf_s2;
      if (pf_s >= 0) {
        pf_hi = a.geo_hi[pf_s];
        pf_lo = a.geo_lo[pf_s];
        pf_r = a.nright[pf_s];
      }
      pf_s2 = fin_id(head + 32);
      pair_decide(k0, s, hiB, loB, rB, a, s_queue[warp][0], stk_of(0), out_of(0), cap, lt, st_fb);
      if (k1.A >= 0) pair_decide(k1, s, hiB, loB, rB, a, s_queue[warp][1], stk_of(1), out_of(1), cap, lt, st_fb);
      __syncwarp();
      if (k0.bad || k1.bad) {
        bad = true;
        break;
      }
      while (!bad && k0.nq >= 32) bad = !append(k0, 0, 32);
      while (!bad && k1.nq >= 32) bad = !append(k1, 1, 32);
      if (bad) break;
    }
    if (bad) {
      drop_kid(k0, SFMM_ST_RING);
      drop_kid(k1, SFMM_ST_RING);
      continue;
    }

    // each child in turn, by the same code
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
      PairKid k = q ? k1 : k0;
      if (k.A < 0) break;
      // its own lowering (leaves pop the pairs they opened), then its
      // remaining accepted pairs, batched as in the per-node walk
      int* const stk = stk_of(q);
      int* const out = out_of(q);
      bool ok = true;
      while (true) {
        const bool more = k.sp > 0;
        if (more) {
          const int cnt = min(32, k.sp);
          const int s = (lane < cnt) ? stk[k.sp - cnt + lane] : -1;
          k.sp -= cnt;
          float4 hiB = make_float4(0.f, 0.f, 0.f, 0.f), loB = hiB;
          int rB = -1;
          if (s >= 0) {
            hiB = a.geo_hi[s];
            loB = a.geo_lo[s];
            rB = a.nright[s];
          }
          pair_decide(k, s, hiB, loB, rB, a, s_queue[warp][q], stk, out, cap, lt, st_fb);
          __syncwarp();
          if (k.bad) {
            ok = false;
            break;
          }
        }
        while (ok && (k.nq >= 32 || (!more && k.nq > 0))) ok = append(k, q, min(k.nq, 32));
        if (!ok || !more) break;
      }
      if (!ok) {
        drop_kid(k, SFMM_ST_RING);
        continue;
      }
      if (lane == 0) {
        st_uniq += k.nacc;
        st_m2l += (unsigned long long)k.nacc * la.nlu[k.A];
      }
      // its batches, in the order they filled
      R C[NCS * 32];
#pragma unroll
      for (int t = 0; t < NCS * 32; ++t) C[t] = R(0);
      const int* const bat = bat_of(q);
      for (int b = 0; b < k.nb; b += 32) m2l_eval<P, F32>(bat[b + lane], k.hi, k.lo, k.cx, k.cy, k.cz, a, C);
      // coefficients: own sums plus the parent's, translated; an internal
      // child stores them and hands its children on, a leaf evaluates them
      // (L2P) and writes its neighbour list
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
      const bool leafA = k.r < 0;
      node_coefficients<P, F32, false, true>(la, k.A, par, leafA, k.hi, k.lo, k.cx, k.cy, k.cz, lev, nullptr, Tn, Tl,
                                             s_T[warp], s_h[warp], s_tab, lane);
      if (!leafA) {
        if (lane == 0) {
          la.cf_off_out[k.A] = k.cfbase;
          la.cf_cnt_out[k.A] = k.nn;
        }
        __syncwarp();
        push_item(k.A);
        continue;
      }
      const int leaf = (int)la.leaf_index[k.A];
      leaf_l2p<P, F32>(la, k.A, k.cx, k.cy, k.cz, Tn, Tl, s_T[warp], lane);
      __syncwarp();
      const int nn = k.nn;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(a.arena_counter, (unsigned long long)nn);
      base = __shfl_sync(SFMM_FULL, base, 0);
      if ((long long)(base + nn) > a.arena_cap) {
        if (lane == 0) {
          set_status(a.status, SFMM_ST_ARENA);
          a.p2p_cnt[leaf] = 0;
        }
      } else {
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
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) st_fb += __shfl_xor_sync(SFMM_FULL, st_fb, o);
  if (lane == 0) {
    atomicAdd(&a.stat[0], st_m2l);
    atomicAdd(&a.stat[1], st_uniq);
    atomicAdd(&a.stat[2], st_pl);
    atomicAdd(&a.stat[4], (unsigned long long)st_fb);
  }
}

// Queue of the pair walk: the system roots fill the first slots.
__global__ void k_queue_seed_pairs(int nsys, const int* __restrict__ sys_root, int* __restrict__ queue,
                                   int* __restrict__ tail) {
  for (int i = threadIdx.x; i < nsys; i += blockDim.x) queue[i] = 2 * sys_root[i] + 1;
  if (threadIdx.x == 0) *tail = nsys;
}
