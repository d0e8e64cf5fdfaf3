// Per-leaf dual-tree walk (Algorithms 1 and 2, Sect. 3) fused with the
// node-node expansions (M2L, Eq. dmkdeffmm), their translation down the
// leaf's branch (Eq. gravmtranslat, App. A.2) and the evaluation at the
// leaf's particles (L2P).
//
// One warp replays the walk of one leaf.  The pairs (p_i, n_s) of
// Algorithm 2 are processed level by level of the branch: all pairs whose
// target is the branch node c_k form the frontier of level k, 32 at a time
// (one per lane).  Accepted pairs are queued and evaluated 32 at a time, one
// per lane, into per-lane partial coefficients of level k; at the end of the
// level a shuffle reduce-scatter leaves coefficient j on lane j, the
// coefficients inherited from c_{k-1} are translated to c_k and the level's
// sum is added (the branch loop of Algorithm 1, fused).  Opened pairs go to
// the frontier of level k+1 (or, at the leaf, back into the same level, or
// into the leaf's neighbour list).  The order of pairs differs from the
// paper's stack order; only the summation order depends on it.
//
// Acceptance is decided in float32 from the double-float node centres with
// a certified error bound; within 1e-5 relative of a tie the decision is
// taken again in float64 with the exact expression of the acceptance test,
// so the interaction lists equal those of a plain float64 evaluation.
#include "walk_common.cuh"

namespace sfmm {
template <int P, bool F32, int MODE>
__global__ void __launch_bounds__(WALK_NT) k_walk(const WalkArgs a) {
  using E = Exp<P>;
  using R = typename std::conditional<F32, float, double>::type;
  constexpr int NC = E::NC;
  constexpr int NCS = (NC + 31) / 32;
  constexpr bool COMPUTE = (MODE == MODE_COMPUTE);

  __shared__ int s_queue[WALK_WARPS][WALK_MQ];
  __shared__ R s_T[WALK_WARPS][NCS * 32];
  __shared__ R s_h[WALK_WARPS][E::NMONO1];
  __shared__ signed char s_tab[NC * NC];

  if (COMPUTE) {
    const signed char* tab = E::table();
    for (int t = threadIdx.x; t < NC * NC; t += WALK_NT) s_tab[t] = tab[t];
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = lanemask_lt();
  const int gw = blockIdx.x * WALK_WARPS + warp;
  const int cap = a.ring_cap;
  int* const bufA = a.ring + (size_t)gw * 2 * cap;
  int* const bufB = bufA + cap;

  unsigned long long st_m2l = 0, st_uniq = 0, st_pl = 0;
  int st_fb = 0;

  while (true) {
    int leaf = 0;
    if (lane == 0) leaf = atomicAdd(a.leaf_counter, 1);
    leaf = __shfl_sync(SFMM_FULL, leaf, 0);
    if (leaf >= a.nleaves) break;
    const int L = a.leaf_node[leaf];
    const int fL = a.nfirst[L], nL = a.ncount[L];

    // inherited coefficients of the current branch node: lane j holds j + 32 b
    R Tn[NCS];
    float Tl[NCS];  // low parts (double-float) in the FP32 form
#pragma unroll
    for (int b = 0; b < NCS; ++b) {
      Tn[b] = R(0);
      Tl[b] = 0.0f;
    }
    int Aid = a.sys_root[a.psys ? a.psys[fL] : 0], prevA = 0;  // the walk starts at the system's root
    float4 hiP = make_float4(0.f, 0.f, 0.f, 0.f), loP = hiP;
    double cPx = 0.0, cPy = 0.0, cPz = 0.0;
    int* cur = bufA;
    int* nxt = bufB;
    if (lane == 0) cur[0] = Aid;
    __syncwarp();
    int head = 0, tail = 1, nn = 0, k = 0;
    bool bad = false;
    long long dump_pos = 0;
    int m2l_here = 0;
    if (MODE == MODE_WRITE) dump_pos = a.m2l_off[leaf];

    while (true) {
      const bool leafA = (Aid == L);
      const float4 hiA = a.geo_hi[Aid], loA = a.geo_lo[Aid];
      double cAx = 0.0, cAy = 0.0, cAz = 0.0;
      if (!F32) {
        cAx = a.ncx[Aid];
        cAy = a.ncy[Aid];
        cAz = a.ncz[Aid];
      }
      const bool uniqueA = (a.nfirst[Aid] == fL);
      R C[NCS * 32];
#pragma unroll
      for (int t = 0; t < NCS * 32; ++t) C[t] = R(0);
      int nq = 0;
      nn = 0;
      while (true) {
        const bool more = head < tail;
        if (more) {
          // FIFO over the fixed frontier of an internal branch node; LIFO at the
          // leaf, where lowering pushes children (keeps the live list short)
          const int cnt = min(32, tail - head);
          int s;
          if (!leafA) {
            s = (lane < cnt) ? cur[head + lane] : -1;
            head += cnt;
          } else {
            s = (lane < cnt) ? cur[tail - cnt + lane] : -1;
            tail -= cnt;
          }
          bool acc = false, open = false;
          int rB = -1;
          if (s >= 0) {
            const float4 hiB = a.geo_hi[s], loB = a.geo_lo[s];
            rB = a.nright[s];
            if (s == Aid) open = true;
            else {
              acc = decide(hiA, loA, hiB, loB, Aid, s, a, st_fb);
              open = !acc;
            }
          }
          const unsigned bacc = __ballot_sync(SFMM_FULL, acc);
          const int nacc = __popc(bacc);
          if (lane == 0) {
            st_m2l += nacc;
            if (uniqueA) st_uniq += nacc;
          }
          m2l_here += nacc;
          if (COMPUTE) {
            if (acc) s_queue[warp][nq + __popc(bacc & lt)] = s;
            nq += nacc;
          } else if (MODE == MODE_WRITE) {
            if (acc) {
              long long o = dump_pos + __popc(bacc & lt);
              a.dump_level[o] = k;
              a.dump_src[o] = s;
            }
            dump_pos += nacc;
          }
          const bool sleaf = open && rB < 0;
          const bool sint = open && rB >= 0;
          if (!leafA) {
            const unsigned b1 = __ballot_sync(SFMM_FULL, open), b2 = __ballot_sync(SFMM_FULL, sint);
            const int add = __popc(b1) + __popc(b2);
            if (nn + add > cap) {
              bad = true;
            } else if (open) {
              const int pos = nn + __popc(b1 & lt) + __popc(b2 & lt);
              if (sleaf) nxt[pos] = s;
              else {
                nxt[pos] = s + 1;
                nxt[pos + 1] = rB;
              }
            }
            nn += add;
          } else {
            const unsigned bl = __ballot_sync(SFMM_FULL, sleaf), bi = __ballot_sync(SFMM_FULL, sint);
            const int addl = __popc(bl), addi = 2 * __popc(bi);
            if (nn + addl > cap || tail + addi > cap) {
              bad = true;
            } else {
              if (sleaf) nxt[nn + __popc(bl & lt)] = s;
              if (sint) {
                const int cp = tail + 2 * __popc(bi & lt);
                cur[cp] = s + 1;
                cur[cp + 1] = rB;
              }
            }
            nn += addl;
            tail += addi;
          }
          __syncwarp();
          if (bad) break;
        }
        if (COMPUTE) {
          while (nq >= 32 || (!more && nq > 0)) {
            const int take = min(nq, 32);
            const int src = (lane < take) ? s_queue[warp][nq - take + lane] : -1;
            __syncwarp();
            m2l_eval<P, F32>(src, hiA, loA, cAx, cAy, cAz, a, C);
            nq -= take;
          }
        }
        if (!more) break;
      }
      if (bad) break;

      if (COMPUTE) {
        // coefficients of level k about c_k: coefficient j on lane j (+32 b)
        R lev[NCS];
#pragma unroll
        for (int b = 0; b < NCS; ++b) {
          R v[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) v[t] = C[32 * b + t];
          lev[b] = reduce_scatter32(v, lane);
        }
        if (k > 0) {
          // translate the inherited coefficients from c_{k-1} to c_k
          if (lane == 0) {
            R hx, hy, hz;
            if constexpr (F32) {
              hx = df_diff(hiA.x, loA.x, hiP.x, loP.x);
              hy = df_diff(hiA.y, loA.y, hiP.y, loP.y);
              hz = df_diff(hiA.z, loA.z, hiP.z, loP.z);
            } else {
              hx = cAx - cPx;
              hy = cAy - cPy;
              hz = cAz - cPz;
            }
            R hm[E::NMONO1];
            E::mono1(hx, hy, hz, hm);
#pragma unroll
            for (int t = 0; t < E::NMONO1; ++t) s_h[warp][t] = hm[t];
          }
#pragma unroll
          for (int b = 0; b < NCS; ++b) s_T[warp][lane + 32 * b] = Tn[b];
          __syncwarp();
#pragma unroll
          for (int b = 0; b < NCS; ++b) {
            const int j = lane + 32 * b;
            if (j < NC) {
              R corr = R(0);
              const signed char* row = s_tab + j * NC;
              for (int i = 0; i < NC; ++i) {
                const int t = row[i];
                if (t > 0) corr = fma(s_h[warp][t], s_T[warp][i], corr);
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
          if constexpr (F32) {
            dfloat r = df_add_f(dfloat{Tn[b], Tl[b]}, lev[b]);
            Tn[b] = r.hi;
            Tl[b] = r.lo;
          } else {
            Tn[b] += lev[b];
          }
        }
      }
      if (leafA) break;
      // next node of the branch: the child containing the leaf
      const int Rc = a.nright[Aid];
      prevA = Aid;
      hiP = hiA;
      loP = loA;
      cPx = cAx;
      cPy = cAy;
      cPz = cAz;
      Aid = (fL >= a.nfirst[Rc]) ? Rc : Aid + 1;
      int* tmp = cur;
      cur = nxt;
      nxt = tmp;
      head = 0;
      tail = nn;
      ++k;
      if (k >= SFMM_MAXDEPTH) {
        bad = true;
        if (lane == 0) set_status(a.status, SFMM_ST_DEPTH);
        break;
      }
    }
    (void)prevA;
    if (bad) {
      if (lane == 0) set_status(a.status, SFMM_ST_RING);
      if (lane == 0) a.p2p_cnt[leaf] = 0;
      continue;
    }

    if (COMPUTE) {
      // L2P: evaluate the leaf's expansion at its particles
#pragma unroll
      for (int b = 0; b < NCS; ++b) {
        if constexpr (F32) s_T[warp][lane + 32 * b] = Tn[b] + Tl[b];
        else s_T[warp][lane + 32 * b] = Tn[b];
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
          ax = a.px[i] - a.ncx[L];
          ay = a.py[i] - a.ncy[L];
          az = a.pz[i] - a.ncz[L];
        }
        R am[E::NQ], out[4];
        E::mono(ax, ay, az, am);
        E::l2p(am, &s_T[warp][0], out);
        if constexpr (F32) a.far32[i] = make_float4(out[1], out[2], out[3], -out[0]);
        else {
          a.far64[4 * (size_t)i] = out[1];
          a.far64[4 * (size_t)i + 1] = out[2];
          a.far64[4 * (size_t)i + 2] = out[3];
          a.far64[4 * (size_t)i + 3] = -out[0];
        }
      }
      __syncwarp();
    }
    if (MODE == MODE_COUNT && lane == 0) a.m2l_cnt[leaf] = m2l_here;

    // neighbour list of the leaf (nxt[0..nn)) into the arena
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
      for (int t = lane; t < nn; t += 32) a.arena[base + t] = nxt[t];
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
  // statistics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) st_fb += __shfl_xor_sync(SFMM_FULL, st_fb, o);
  if (lane == 0) {
    atomicAdd(&a.stat[0], st_m2l);
    atomicAdd(&a.stat[1], st_uniq);
    atomicAdd(&a.stat[2], st_pl);
    atomicAdd(&a.stat[4], (unsigned long long)st_fb);
  }
}

template <int P, bool F32, int MODE>
static int launch_walk(sfmm_ctx* c, WalkArgs& a, int nblocks) {
  k_walk<P, F32, MODE><<<nblocks, WALK_NT, 0, c->stream>>>(a);
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

template <int P, bool F32, int MODE>
static int walk_blocks(sfmm_ctx* c) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<P, F32, MODE>, WALK_NT, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms(c->device);
}

typedef int (*launch_fn)(sfmm_ctx*, WalkArgs&, int);
typedef int (*blocks_fn)(sfmm_ctx*);

template <int MODE>
static void pick(int order, bool f32, launch_fn& L, blocks_fn& B) {
#define SFMM_PICK(PP)                                           \
  if (order == PP) {                                            \
    if (f32) { L = launch_walk<PP, true, MODE>; B = walk_blocks<PP, true, MODE>; } \
    else { L = launch_walk<PP, false, MODE>; B = walk_blocks<PP, false, MODE>; }  \
  }
  SFMM_PICK(0) SFMM_PICK(1) SFMM_PICK(2) SFMM_PICK(3) SFMM_PICK(4)
#undef SFMM_PICK
}

// Runs the walk.  dump = false: full computation (far field + neighbour
// lists).  dump = true: decisions only, into c->dump (tests).
int run_walk(sfmm_ctx* c, double theta, int order, bool dump, int64_t cap_m2l, int64_t /*cap_p2p*/) {
  const bool f32 = (c->precision == SFMM_FP32) && !dump;
  const int nl = c->nleaves;
  int rc;
  launch_fn L = nullptr;
  blocks_fn B = nullptr;
  if (!dump) pick<MODE_COMPUTE>(order, f32, L, B);
  else L = launch_walk<0, true, MODE_COUNT>, B = walk_blocks<0, true, MODE_COUNT>;
  if (!L) return SFMM_EINVAL;
  const int nblocks = B(c);
  const int nwarps = nblocks * WALK_WARPS;

  for (int attempt = 0; attempt < SFMM_WALK_ATTEMPTS; ++attempt) {
    if ((rc = c->ring.ensure(sizeof(int) * (size_t)nwarps * 2 * c->ring_capacity))) return rc;
    long long arena_cap = c->list_capacity > 0 ? c->list_capacity : (long long)nl * 96 + 1024;
    if ((rc = c->arena.ensure(sizeof(int) * (size_t)arena_cap))) return rc;
    arena_cap = (long long)(c->arena.bytes / sizeof(int));
    if ((rc = c->p2p_off.ensure(sizeof(long long) * (size_t)nl))) return rc;
    if ((rc = c->p2p_cnt.ensure(sizeof(int) * (size_t)nl))) return rc;
    if ((rc = c->counters.ensure(sizeof(unsigned long long) * 20))) return rc;
    if ((rc = c->far.ensure((f32 ? sizeof(float4) : 4 * sizeof(double)) * (size_t)c->n))) return rc;
    unsigned long long* ctr = c->counters.as<unsigned long long>();
    SFMM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 16, c->stream));

    WalkArgs a{};
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
    a.leaf_counter = reinterpret_cast<int*>(ctr + 8);
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
    a.psys = c->nsys > 1 ? c->psys.as<int>() : nullptr;
    a.sys_root = c->sys_root.as<int>();
    if (dump) {
      // counting pass, then the writing pass at the scanned offsets
      if ((rc = c->dump.ensure(sizeof(int) * (size_t)(nl + 1) + sizeof(long long) * (size_t)(nl + 1)))) return rc;
      a.m2l_cnt = c->dump.as<int>();
      if ((rc = L(c, a, nblocks))) return rc;
    } else {
      if ((rc = L(c, a, nblocks))) return rc;
    }
    int bits = 0;
    if ((rc = sync_status(c, &bits))) return rc;
    if (bits & SFMM_ST_DEPTH) return set_error(c, SFMM_ESTACK, "a leaf's branch is deeper than the walk supports");
    if (bits & (SFMM_ST_RING | SFMM_ST_ARENA)) {
      if (attempt == SFMM_WALK_ATTEMPTS - 1)
        return set_error(c, SFMM_ECAPACITY, "walk buffers too small after the last regrow");
      // the arena counter counts every list that reached it, so it is a lower
      // bound when frontier rings also overflowed
      unsigned long long need = 0;
      SFMM_CUDA_TRY(cudaMemcpy(&need, ctr + 9, sizeof(need), cudaMemcpyDeviceToHost));
      if (bits & SFMM_ST_RING) c->ring_capacity = c->ring_capacity < (1 << 20) ? c->ring_capacity * 16 : (1 << 24);
      if (bits & SFMM_ST_ARENA) {
        int64_t grown = 2 * (int64_t)arena_cap;
        int64_t want = (int64_t)(need + need / 4 + 1024);
        c->list_capacity = want > grown ? want : grown;
      }
      SFMM_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
      continue;
    }
    SFMM_CUDA_TRY(cudaMemcpy(c->h_scalars, ctr, sizeof(unsigned long long) * 10, cudaMemcpyDeviceToHost));
    const unsigned long long* hs = reinterpret_cast<const unsigned long long*>(c->h_scalars);
    c->arena_used = (int64_t)hs[9];
    c->split_chunks = (int64_t)hs[5];
    c->split_lists = (int64_t)hs[6];
    c->stats.m2l = (int64_t)hs[0];
    c->stats.m2l_unique = (int64_t)hs[1];
    c->stats.p2p_leaves = (int64_t)hs[2];
    c->stats.p2p_pairs = (int64_t)hs[3];
    c->stats.mac_fallbacks = (int64_t)hs[4];
    return SFMM_OK;
  }
  (void)cap_m2l;
  return SFMM_ECAPACITY;
}

// Second pass of the list dump: write entries at the scanned offsets.
int run_walk_dump_write(sfmm_ctx* c, double theta, const long long* d_off, int* d_level, int* d_src) {
  const int nl = c->nleaves;
  int rc;
  const int nblocks = walk_blocks<0, true, MODE_WRITE>(c);
  unsigned long long* ctr = c->counters.as<unsigned long long>();
  SFMM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 16, c->stream));
  WalkArgs a{};
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
  a.ring = c->ring.as<int>();
  a.ring_cap = c->ring_capacity;
  a.leaf_counter = reinterpret_cast<int*>(ctr + 8);
  a.arena = c->arena.as<int>();
  a.arena_counter = ctr + 9;
  a.split_counter = ctr + 5;
    a.chunk = c->p2p_chunk;
  a.arena_cap = (long long)(c->arena.bytes / sizeof(int));
  a.p2p_off = c->p2p_off.as<long long>();
  a.p2p_cnt = c->p2p_cnt.as<int>();
  a.status = c->d_status;
  a.stat = ctr;
  a.theta = theta;
  a.theta_f = (float)theta;
  a.theta2_f = (float)(theta * theta);
  a.psys = c->nsys > 1 ? c->psys.as<int>() : nullptr;
  a.sys_root = c->sys_root.as<int>();
  a.m2l_off = d_off;
  a.dump_level = d_level;
  a.dump_src = d_src;
  if ((rc = launch_walk<0, true, MODE_WRITE>(c, a, nblocks))) return rc;
  int bits = 0;
  if ((rc = sync_status(c, &bits))) return rc;
  if (bits) return set_error(c, SFMM_ECAPACITY, "list dump: walk buffers overflowed");
  return SFMM_OK;
}

}  // namespace sfmm
