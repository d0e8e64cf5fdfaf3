// Mass moments of the tree nodes (Eq. massmom, Sect. 2.1): scaled moments
// Q_alpha / alpha! about each node's centre of mass, computed from the
// particles at the leaves (P2M) and translated bottom-up to the parents
// (Eq. massmomtrans, App. A.1: Q'_alpha/alpha! = sum_{beta<=alpha}
// g^(alpha-beta)/(alpha-beta)! Q_beta/beta!, g = child - parent centre).
#include "mom_ops.cuh"
#include "sfmm_internal.cuh"

namespace sfmm {


// P2M: one thread per leaf (short FP64 sums; no cross-lane reduction).
template <int P>
__global__ void k_p2m(int nleaves, const int* __restrict__ leaf_node, const int* __restrict__ nfirst,
                      const int* __restrict__ ncount, const double* __restrict__ px, const double* __restrict__ py,
                      const double* __restrict__ pz, const double* __restrict__ pm, const double* __restrict__ ncx,
                      const double* __restrict__ ncy, const double* __restrict__ ncz, double* __restrict__ Qd) {
  constexpr int NQ = MomOps<P>::NQ;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaves) return;
  const int v = leaf_node[q];
  const int f = nfirst[v], cnt = ncount[v];
  const double sx = ncx[v], sy = ncy[v], sz = ncz[v];
  double acc[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) acc[k] = 0.0;
  for (int i = f; i < f + cnt; ++i) {
    double mono[NQ];
    MomOps<P>::mono(px[i] - sx, py[i] - sy, pz[i] - sz, mono);
    const double m = pm[i];
#pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = fma(m, mono[k], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < NQ; ++k) Qd[(int64_t)v * NQ + k] = acc[k];
}

// M2M bottom-up: the second child to finish translates both children.
template <int P>
__global__ void k_m2m(int nleaves, const int* __restrict__ leaf_node, const int* __restrict__ nparent,
                      const int* __restrict__ nright, const double* __restrict__ ncx, const double* __restrict__ ncy,
                      const double* __restrict__ ncz, double* Qd, int* flags) {
  constexpr int NQ = MomOps<P>::NQ;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaves) return;
  int v = nparent[leaf_node[q]];
  while (v >= 0) {
    __threadfence();
    if (atomicAdd(&flags[v], 1) == 0) return;
    __threadfence();
    double qp[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) qp[k] = 0.0;
    const int kids[2] = {v + 1, nright[v]};
    for (int c = 0; c < 2; ++c) {
      int u = kids[c];
      double g[NQ], qc[NQ];
      MomOps<P>::mono(ncx[u] - ncx[v], ncy[u] - ncy[v], ncz[u] - ncz[v], g);
#pragma unroll
      for (int k = 0; k < NQ; ++k) qc[k] = __ldcg(&Qd[(int64_t)u * NQ + k]);
      MomOps<P>::m2m(g, qc, qp);
    }
#pragma unroll
    for (int k = 0; k < NQ; ++k) Qd[(int64_t)v * NQ + k] = qp[k];
    v = nparent[v];
  }
}

// float32 copies for the FP32 form, rows padded to a multiple of 4.
__global__ void k_moments_f32(int64_t total, int nq, int nqs, const double* __restrict__ Qd, float* __restrict__ Qf) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int64_t v = t / nqs;
  int k = (int)(t - v * nqs);
  Qf[t] = (k < nq) ? __double2float_rn(Qd[v * nq + k]) : 0.0f;
}

template <int P>
static int moments_p(sfmm_ctx* c) {
  constexpr int NQ = MomOps<P>::NQ;
  const int nn = c->nnodes, nl = c->nleaves;
  int rc;
  if ((rc = c->Qd.ensure(sizeof(double) * (size_t)nn * NQ))) return rc;
  const int nqs = (NQ + 3) & ~3;
  if ((rc = c->Qf.ensure(sizeof(float) * (size_t)nn * nqs))) return rc;
  cudaStream_t st = c->stream;
  k_p2m<P><<<(unsigned)((nl + 127) / 128), 128, 0, st>>>(
      nl, c->leaf_node.as<int>(), c->nfirst.as<int>(), c->ncount.as<int>(), c->px.as<double>(), c->py.as<double>(),
      c->pz.as<double>(), c->pm.as<double>(), c->ncx.as<double>(), c->ncy.as<double>(), c->ncz.as<double>(),
      c->Qd.as<double>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaMemsetAsync(c->flags.p, 0, sizeof(int) * nn, st));
  k_m2m<P><<<(nl + 127) / 128, 128, 0, st>>>(nl, c->leaf_node.as<int>(), c->nparent.as<int>(), c->nright.as<int>(),
                                             c->ncx.as<double>(), c->ncy.as<double>(), c->ncz.as<double>(),
                                             c->Qd.as<double>(), c->flags.as<int>());
  ++c->nlaunch;
  int64_t tot = (int64_t)nn * nqs;
  k_moments_f32<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, NQ, nqs, c->Qd.as<double>(), c->Qf.as<float>());
  ++c->nlaunch;
  SFMM_CUDA_TRY(cudaGetLastError());
  return SFMM_OK;
}

int compute_moments(sfmm_ctx* c, int order) {
  int rc;
  switch (order) {
    case 0: rc = moments_p<0>(c); break;
    case 1: rc = moments_p<1>(c); break;
    case 2: rc = moments_p<2>(c); break;
    case 3: rc = moments_p<3>(c); break;
    case 4: rc = moments_p<4>(c); break;
    default: return SFMM_EINVAL;
  }
  if (rc == SFMM_OK) {
    c->moments_order = order;
    c->moments_fp64 = true;
  }
  return rc;
}

}  // namespace sfmm
