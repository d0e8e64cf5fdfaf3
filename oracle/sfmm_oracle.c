/*
 * sfmm_oracle.c -- plain, slow, FP64 CPU oracle of the symmetric fast
 * multipole method (SFMM) with adaptive kernel softening.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant with the CUDA solver; the two meet only on the seeded
 * inputs drawn by the `workloads` module.
 *
 * Everything is written the obvious way, in the paper's notation:
 *   - tensors are FULL Cartesian tensors (3^n components, row-major index
 *     i1 i2 ... in), contracted index by index, exactly as the paper writes
 *     T . b^(n) (no symmetric compression, no fused evaluation);
 *   - node moments are computed directly from the particles of each node
 *     (Eq. massmom, Sect. 2.1; computed per node as in Sect. 3);
 *   - the tree walk is Algorithms 1 and 2 (Sect. 3) with an explicit stack and
 *     one buffer of gravitational moments per parent on the leaf's branch,
 *     followed by the top-down propagation (Eq. gravmtranslat, App. A.2),
 *     the evaluation at the particles and the pairwise softened pass.
 * Compile with -ffp-contract=off so that every expression rounds as written.
 *
 * Function catalogue (each cites its passage):
 *   orc_kernel        M4 softening kernel phi(r,h), g(r,h) (Eq. softdirectsum, Sect. 2)
 *   orc_direct        O(N^2) softened direct sum (Eqs. directsum, softdirectsum)
 *   orc_derivs        D_gamma = d^gamma (1/|r|) (the D_n of Sect. 2.1)
 *   orc_p2m           Q_n = sum_j m_j b_j^(n) (Eq. massmom)
 *   orc_m2m           moment translation (Eq. massmomtrans, App. A.1)
 *   orc_m2l_eval      dM_k / M_k expansion about two centres (Eq. dmkdeffmm, Sect. 2.2)
 *   orc_l2l           translation of gravitational moments (Eq. gravmtranslat, App. A.2)
 *   orc_build         tree, node centres/sizes/h_max/moments (Sect. 3)
 *   orc_build_kd      the same over a centre-of-mass-pivot kd tree (Sect. 3)
 *   orc_sfmm          Algorithms 1 and 2, propagation, evaluation, P2P (Sect. 3)
 *
 * Readings where the paper is silent or garbled (each is stated in the
 * design notes):
 *   - softening kernel: cubic-spline (M4) kernel of compact support 2h, the
 *     kernel cited for Eq. softdirectsum; pair value = mean of the two
 *     particles' kernels;
 *   - Eqs. 25-28 omit the factor -G; the potential is -G sum ..., the
 *     acceleration -G sum_k a^(k)/k! . dM_k (Eqs. 12 and 16);
 *   - node size l = max_j |x_j - s| about the centre of mass s;
 *   - the secondary criterion (Eq. after the MAC) is an OPENING condition:
 *     a pair is accepted only if l_t + l_s < theta d AND NOT
 *     d < l_t + l_s + R_kern max(h_t, h_s), with R_kern = 2;
 *   - tree: binary radix tree over 63-bit Morton keys (21 bits per axis),
 *     ties broken by sorted position, leaves hold <= leaf_size particles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_RKERN 2.0
#define ORC_PMAX 4             /* highest expansion order p supported */
#define ORC_MAXRANK (ORC_PMAX + 1)
#define ORC_MAXDEPTH 256

/* ------------------------------------------------------------------------ */
/* Small helpers                                                             */
/* ------------------------------------------------------------------------ */

static int ipow3(int n) { int r = 1; while (n-- > 0) r *= 3; return r; }

static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= (double)i; return f; }

/* ------------------------------------------------------------------------ */
/* M4 softening kernel (Eq. softdirectsum, Sect. 2; kernel of Price 2007)    */
/*   phi(r,h): potential kernel, -> -1/r for r >= 2h                         */
/*   g(r,h)  : (d phi / d r) / r, -> 1/r^3 for r >= 2h                       */
/* ------------------------------------------------------------------------ */

static double kernel_phi(double r, double h)
{
    double q = r / h;
    if (q < 1.0) {
        double q2 = q * q;
        return (2.0 / 3.0 * q2 - 3.0 / 10.0 * q2 * q2 + 1.0 / 10.0 * q2 * q2 * q - 7.0 / 5.0) / h;
    } else if (q < 2.0) {
        double q2 = q * q;
        return (4.0 / 3.0 * q2 - q2 * q + 3.0 / 10.0 * q2 * q2 - 1.0 / 30.0 * q2 * q2 * q
                - 8.0 / 5.0 + 1.0 / (15.0 * q)) / h;
    }
    return -1.0 / r;
}

static double kernel_g(double r, double h)
{
    double q = r / h;
    if (q < 1.0) {
        double q2 = q * q;
        return (4.0 / 3.0 - 6.0 / 5.0 * q2 + 1.0 / 2.0 * q2 * q) / (h * h * h);
    } else if (q < 2.0) {
        double q2 = q * q;
        return (8.0 / 3.0 - 3.0 * q + 6.0 / 5.0 * q2 - 1.0 / 6.0 * q2 * q - 1.0 / (15.0 * q2 * q))
               / (h * h * h);
    }
    return 1.0 / (r * r * r);
}

void orc_kernel(int64_t n, const double* r, const double* h, double* phi, double* g)
{
    for (int64_t i = 0; i < n; ++i) {
        phi[i] = kernel_phi(r[i], h[i]);
        g[i] = kernel_g(r[i], h[i]);
    }
}

/* Softened pair: contribution of source j (mass mj, smoothing hj) to target
 * i (smoothing hi), with d = x_i - x_j.  The pair kernel is the mean of the
 * two particles' kernels, so the pair force is equal and opposite.         */
static void pair_softened(const double d[3], double hi, double mj, double hj,
                          double G, double acc[3], double* pot)
{
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double gbar = 0.5 * (kernel_g(r, hi) + kernel_g(r, hj));
    double pbar = 0.5 * (kernel_phi(r, hi) + kernel_phi(r, hj));
    for (int c = 0; c < 3; ++c) acc[c] += -G * mj * gbar * d[c];
    *pot += G * mj * pbar;
}

/* ------------------------------------------------------------------------ */
/* O(N^2) direct sum (Eqs. directsum and softdirectsum, Sect. 2)             */
/* targets: NULL for all particles, else nt indices.                         */
/* ------------------------------------------------------------------------ */

void orc_direct(int64_t n, const double* pos, const double* m, const double* h,
                double G, int self_pot, int64_t nt, const int64_t* targets,
                double* acc, double* pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = targets ? targets[t] : t;
        double a[3] = {0.0, 0.0, 0.0}, p = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                           pos[3 * i + 2] - pos[3 * j + 2]};
            pair_softened(d, h[i], m[j], h[j], G, a, &p);
        }
        if (self_pot) p += G * m[i] * kernel_phi(0.0, h[i]);
        acc[3 * t] = a[0]; acc[3 * t + 1] = a[1]; acc[3 * t + 2] = a[2];
        pot[t] = p;
    }
}

/* ------------------------------------------------------------------------ */
/* Derivatives of the Green's function (the D_n of Sect. 2.1)                */
/*                                                                           */
/* D_gamma(r) = d^gamma (1/|r|) for a multi-index gamma, computed with the   */
/* McMurchie-Davidson (1978) recurrence                                      */
/*   R^(m)_0 = (-1)^m (2m-1)!! |r|^-(2m+1)                                   */
/*   R^(m)_gamma = (g_t - 1) R^(m+1)_{gamma - 2e_t} + r_t R^(m+1)_{gamma-e_t} */
/* (t the first axis with g_t > 0), D_gamma = R^(0)_gamma.  The full rank-n  */
/* tensor D_n is then filled index by index: D_{i1..in} = D_gamma, gamma    */
/* the axis counts of (i1..in).                                              */
/* ------------------------------------------------------------------------ */

/* multi-index table: for |gamma| <= ORC_MAXRANK, dense index by (a,b,c) */
#define MI_DIM (ORC_MAXRANK + 1)

static double R_rec(int m, int a, int b, int c, const double r[3], double rinv2, double rinv,
                    double memo[][MI_DIM][MI_DIM][MI_DIM], unsigned char done[][MI_DIM][MI_DIM][MI_DIM])
{
    if (done[m][a][b][c]) return memo[m][a][b][c];
    double v;
    if (a == 0 && b == 0 && c == 0) {
        double df = 1.0;               /* (2m-1)!! */
        for (int k = 2 * m - 1; k > 1; k -= 2) df *= (double)k;
        double pw = rinv;               /* |r|^-(2m+1) */
        for (int k = 0; k < m; ++k) pw *= rinv2;
        v = ((m % 2) ? -1.0 : 1.0) * df * pw;
    } else if (a > 0) {
        v = r[0] * R_rec(m + 1, a - 1, b, c, r, rinv2, rinv, memo, done);
        if (a > 1) v += (double)(a - 1) * R_rec(m + 1, a - 2, b, c, r, rinv2, rinv, memo, done);
    } else if (b > 0) {
        v = r[1] * R_rec(m + 1, a, b - 1, c, r, rinv2, rinv, memo, done);
        if (b > 1) v += (double)(b - 1) * R_rec(m + 1, a, b - 2, c, r, rinv2, rinv, memo, done);
    } else {
        v = r[2] * R_rec(m + 1, a, b, c - 1, r, rinv2, rinv, memo, done);
        if (c > 1) v += (double)(c - 1) * R_rec(m + 1, a, b, c - 2, r, rinv2, rinv, memo, done);
    }
    memo[m][a][b][c] = v;
    done[m][a][b][c] = 1;
    return v;
}

/* D_gamma for all |gamma| <= P (P <= ORC_MAXRANK); out[a][b][c]. */
static void derivs_mi(int P, const double r[3], double out[MI_DIM][MI_DIM][MI_DIM])
{
    static const int M = ORC_MAXRANK + 2;
    double memo[ORC_MAXRANK + 2][MI_DIM][MI_DIM][MI_DIM];
    unsigned char done[ORC_MAXRANK + 2][MI_DIM][MI_DIM][MI_DIM];
    (void)M;
    memset(done, 0, sizeof(done));
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rinv = 1.0 / sqrt(r2);
    double rinv2 = 1.0 / r2;
    for (int a = 0; a <= P; ++a)
        for (int b = 0; a + b <= P; ++b)
            for (int c = 0; a + b + c <= P; ++c)
                out[a][b][c] = R_rec(0, a, b, c, r, rinv2, rinv, memo, done);
}

/* Fill the full rank-n tensor D_n from the multi-index values. */
static void derivs_full(int n, double mi[MI_DIM][MI_DIM][MI_DIM], double* T)
{
    int sz = ipow3(n);
    for (int idx = 0; idx < sz; ++idx) {
        int cnt[3] = {0, 0, 0}, t = idx;
        for (int k = 0; k < n; ++k) { cnt[t % 3]++; t /= 3; }
        T[idx] = mi[cnt[0]][cnt[1]][cnt[2]];
    }
}

/* Exported: D_gamma for |gamma| <= P in a caller table of multi-indices. */
void orc_derivs(int P, const double r[3], int ngam, const int* gam /* ngam x 3 */, double* out)
{
    double mi[MI_DIM][MI_DIM][MI_DIM];
    derivs_mi(P, r, mi);
    for (int k = 0; k < ngam; ++k) out[k] = mi[gam[3 * k]][gam[3 * k + 1]][gam[3 * k + 2]];
}

/* ------------------------------------------------------------------------ */
/* Full-tensor contraction helpers                                           */
/* ------------------------------------------------------------------------ */

/* out (rank rA - rB) = A (rank rA) . B (rank rB): contract the FIRST rB
 * indices of A with all indices of B (A symmetric, so which ones is moot). */
static void contract(const double* A, int rA, const double* B, int rB, double* out)
{
    int sB = ipow3(rB), sO = ipow3(rA - rB);
    for (int o = 0; o < sO; ++o) {
        double s = 0.0;
        for (int b = 0; b < sB; ++b) s += A[b * sO + o] * B[b];
        out[o] = s;
    }
}

/* v^(n): n-fold tensor product of a 3-vector, full tensor of 3^n entries. */
static void outer_power(const double v[3], int n, double* out)
{
    int sz = ipow3(n);
    for (int idx = 0; idx < sz; ++idx) {
        double p = 1.0;
        int t = idx;
        /* row-major: i1 is the most significant digit */
        int digits[ORC_MAXRANK + 4];
        for (int k = n - 1; k >= 0; --k) { digits[k] = t % 3; t /= 3; }
        for (int k = 0; k < n; ++k) p *= v[digits[k]];
        out[idx] = p;
    }
}

/* offsets of rank-n blocks in a packed array of ranks 0..R */
static int rank_off(int n) { int o = 0; for (int k = 0; k < n; ++k) o += ipow3(k); return o; }
static int packed_size(int R) { return rank_off(R + 1); }

/* ------------------------------------------------------------------------ */
/* Mass moments Q_n = sum_j m_j b_j^(n), b_j = x_j - s (Eq. massmom)         */
/* packed: ranks 0..p, full tensors                                          */
/* ------------------------------------------------------------------------ */

static void p2m_direct(int p, int64_t n, const double* pos, const double* m,
                       const int64_t* idx, const double s[3], double* Q)
{
    memset(Q, 0, sizeof(double) * packed_size(p));
    double tmp[243];
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = idx ? idx[k] : k;
        double b[3] = {pos[3 * j] - s[0], pos[3 * j + 1] - s[1], pos[3 * j + 2] - s[2]};
        for (int r = 0; r <= p; ++r) {
            outer_power(b, r, tmp);
            double* Qr = Q + rank_off(r);
            for (int e = 0; e < ipow3(r); ++e) Qr[e] += m[j] * tmp[e];
        }
    }
}

void orc_p2m(int p, int64_t n, const double* pos, const double* m, const double s[3], double* Q)
{
    p2m_direct(p, n, pos, m, NULL, s, Q);
}

/* Moment translation (Eq. massmomtrans, App. A.1):
 * Q'_n = sum_j m_j (g + b_j)^(n), expanded with the binomial identity of
 * Sect. 2.2 (Eq. after 20): (g + b)^(n) symmetrised = sum_k C(n,k) g^(n-k) b^(k).
 * Written out on full tensors: component (i1..in) of (g+b)^(n) is
 * prod_k (g_{ik} + b_{ik}) = sum over subsets S of {1..n} of
 * prod_{k in S} b_{ik} prod_{k not in S} g_{ik}; summing m_j over the child
 * gives sum_S Q_{|S|}[indices in S] * prod_{k not in S} g_{ik}.             */
void orc_m2m(int p, const double* Qc, const double g[3], double* Qp)
{
    for (int n = 0; n <= p; ++n) {
        int sz = ipow3(n);
        double* out = Qp + rank_off(n);
        for (int idx = 0; idx < sz; ++idx) {
            int digits[ORC_MAXRANK + 4], t = idx;
            for (int k = n - 1; k >= 0; --k) { digits[k] = t % 3; t /= 3; }
            double s = 0.0;
            for (int S = 0; S < (1 << n); ++S) {
                int nb = 0, bidx = 0;
                double gp = 1.0;
                for (int k = 0; k < n; ++k) {
                    if (S & (1 << k)) { bidx = bidx * 3 + digits[k]; nb++; }
                    else gp *= g[digits[k]];
                }
                s += Qc[rank_off(nb) + bidx] * gp;
            }
            out[idx] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Expansion about two centres (Eq. dmkdeffmm and the M_k of Sect. 2.2)      */
/*   M_k  = (-1)^k sum_{n=0}^{p-k} 1/n! D_{n+k}   . Q_n   (rank k)           */
/*   dM_k = (-1)^k sum_{n=0}^{p-k} 1/n! D_{n+k+1} . Q_n   (rank k+1)         */
/* r = s_B - s_A.  Layout: M packed ranks 0..p; dM packed ranks 1..p+1 (the  */
/* rank k+1 block of dM_k stored at rank_off(k+1) - 1).                      */
/* ------------------------------------------------------------------------ */

static int dm_off(int k) { return rank_off(k + 1) - 1; }
static int dm_size(int p) { return dm_off(p + 1); }

static void m2l_add(int p, const double r[3], const double* QB, double* M, double* dM)
{
    double mi[MI_DIM][MI_DIM][MI_DIM];
    derivs_mi(p + 1, r, mi);
    double D[ORC_MAXRANK + 1][243];
    for (int n = 0; n <= p + 1; ++n) derivs_full(n, mi, D[n]);
    double tmp[243];
    for (int k = 0; k <= p; ++k) {
        double sg = (k % 2) ? -1.0 : 1.0;
        for (int n = 0; n <= p - k; ++n) {
            double c = sg / factorial(n);
            contract(D[n + k], n + k, QB + rank_off(n), n, tmp);
            for (int e = 0; e < ipow3(k); ++e) M[rank_off(k) + e] += c * tmp[e];
            contract(D[n + k + 1], n + k + 1, QB + rank_off(n), n, tmp);
            for (int e = 0; e < ipow3(k + 1); ++e) dM[dm_off(k) + e] += c * tmp[e];
        }
    }
}

/* Translation of gravitational moments (Eq. gravmtranslat, App. A.2):
 * dM_k(new) = sum_{l=k}^{p} 1/(l-k)! h^(l-k) . dM_l, same for M_k,
 * h = new centre - old centre.  Accumulates into Mo/dMo.                   */
static void l2l_add(int p, const double h[3], const double* Mi, const double* dMi,
                    double* Mo, double* dMo)
{
    double hp[243], tmp[243];
    for (int k = 0; k <= p; ++k) {
        for (int l = k; l <= p; ++l) {
            double c = 1.0 / factorial(l - k);
            outer_power(h, l - k, hp);
            contract(Mi + rank_off(l), l, hp, l - k, tmp);
            for (int e = 0; e < ipow3(k); ++e) Mo[rank_off(k) + e] += c * tmp[e];
            contract(dMi + dm_off(l), l + 1, hp, l - k, tmp);
            for (int e = 0; e < ipow3(k + 1); ++e) dMo[dm_off(k) + e] += c * tmp[e];
        }
    }
}

/* Evaluation at a particle (Eqs. 27-28 with the -G of Eqs. 12, 16):
 * Phi = -G sum_k a^(k)/k! . M_k ;  acc = -G sum_k a^(k)/k! . dM_k.        */
static void l2p(int p, const double a[3], const double* M, const double* dM, double G,
                double acc[3], double* pot)
{
    double ap[243], tmp[243];
    for (int k = 0; k <= p; ++k) {
        double c = 1.0 / factorial(k);
        outer_power(a, k, ap);
        contract(M + rank_off(k), k, ap, k, tmp);
        *pot += -G * c * tmp[0];
        contract(dM + dm_off(k), k + 1, ap, k, tmp);
        for (int d = 0; d < 3; ++d) acc[d] += -G * c * tmp[d];
    }
}

/* Exported pin helpers ---------------------------------------------------- */

int orc_packed_size(int p) { return packed_size(p); }
int orc_dm_size(int p) { return dm_size(p); }

/* M2L from the particles of B (moments about sB) to the centre sA, then
 * evaluation at the particles of A. */
void orc_m2l_eval(int p, const double sA[3], const double sB[3],
                  int64_t nB, const double* xB, const double* mB,
                  int64_t nA, const double* xA, double G, double* acc, double* pot)
{
    double Q[400], M[400], dM[1200];
    p2m_direct(p, nB, xB, mB, NULL, sB, Q);
    memset(M, 0, sizeof(M));
    memset(dM, 0, sizeof(dM));
    double r[3] = {sB[0] - sA[0], sB[1] - sA[1], sB[2] - sA[2]};
    m2l_add(p, r, Q, M, dM);
    for (int64_t i = 0; i < nA; ++i) {
        double a[3] = {xA[3 * i] - sA[0], xA[3 * i + 1] - sA[1], xA[3 * i + 2] - sA[2]};
        double f[3] = {0, 0, 0}, ph = 0.0;
        l2p(p, a, M, dM, G, f, &ph);
        acc[3 * i] = f[0]; acc[3 * i + 1] = f[1]; acc[3 * i + 2] = f[2];
        pot[i] = ph;
    }
}

/* Same as orc_m2l_eval but the coefficients are first translated from sA to
 * sA2 (Eq. gravmtranslat) and evaluated about sA2. */
void orc_m2l_l2l_eval(int p, const double sA[3], const double sA2[3], const double sB[3],
                      int64_t nB, const double* xB, const double* mB,
                      int64_t nA, const double* xA, double G, double* acc, double* pot)
{
    double Q[400], M[400], dM[1200], M2[400], dM2[1200];
    p2m_direct(p, nB, xB, mB, NULL, sB, Q);
    memset(M, 0, sizeof(M)); memset(dM, 0, sizeof(dM));
    memset(M2, 0, sizeof(M2)); memset(dM2, 0, sizeof(dM2));
    double r[3] = {sB[0] - sA[0], sB[1] - sA[1], sB[2] - sA[2]};
    m2l_add(p, r, Q, M, dM);
    double h[3] = {sA2[0] - sA[0], sA2[1] - sA[1], sA2[2] - sA[2]};
    l2l_add(p, h, M, dM, M2, dM2);
    for (int64_t i = 0; i < nA; ++i) {
        double a[3] = {xA[3 * i] - sA2[0], xA[3 * i + 1] - sA2[1], xA[3 * i + 2] - sA2[2]};
        double f[3] = {0, 0, 0}, ph = 0.0;
        l2p(p, a, M2, dM2, G, f, &ph);
        acc[3 * i] = f[0]; acc[3 * i + 1] = f[1]; acc[3 * i + 2] = f[2];
        pot[i] = ph;
    }
}

/* Raw coefficients of one M2L: M (packed ranks 0..p) and dM (packed). */
void orc_m2l_coeffs(int p, const double r[3], const double* QB, double* M, double* dM)
{
    memset(M, 0, sizeof(double) * packed_size(p));
    memset(dM, 0, sizeof(double) * dm_size(p));
    m2l_add(p, r, QB, M, dM);
}

/* ------------------------------------------------------------------------ */
/* Tree (Sect. 3): binary radix tree over Morton keys                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int leaf_size, p;
    double *x, *m, *h;         /* sorted copies: x is n x 3 */
    int64_t* perm;             /* sorted position -> caller index */
    uint64_t* key;             /* sorted keys */
    int64_t nnodes, nleaves;
    int32_t *first, *count, *left, *right, *parent, *depth;
    double *centre, *size, *hmax, *mass;   /* centre is nnodes x 3 */
    double* Q;                 /* nnodes x packed_size(p) */
    int32_t* leaves;           /* leaf node ids, in tree (Morton) order */
    double bbmin[3], extent, scale;
} orc_tree;

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void* a, const void* b)
{
    const keyidx* x = (const keyidx*)a;
    const keyidx* y = (const keyidx*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Morton key: 21 bits per axis, x highest: bit 3b+2 = x_b, 3b+1 = y_b, 3b = z_b */
static uint64_t morton(uint64_t kx, uint64_t ky, uint64_t kz)
{
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b) {
        key |= ((kx >> b) & 1ull) << (3 * b + 2);
        key |= ((ky >> b) & 1ull) << (3 * b + 1);
        key |= ((kz >> b) & 1ull) << (3 * b);
    }
    return key;
}

static int highest_bit64(uint64_t v) { int b = -1; while (v) { v >>= 1; ++b; } return b; }

typedef struct { int64_t cap; } tree_cap;

static int64_t build_rec(orc_tree* t, int64_t first, int64_t count, int depth, int32_t parent)
{
    int64_t id = t->nnodes++;
    t->first[id] = (int32_t)first;
    t->count[id] = (int32_t)count;
    t->parent[id] = parent;
    t->depth[id] = depth;
    t->left[id] = -1;
    t->right[id] = -1;
    if (count <= t->leaf_size) return id;
    int64_t last = first + count - 1;
    int64_t split;
    if (t->key[first] != t->key[last]) {
        int b = highest_bit64(t->key[first] ^ t->key[last]);
        split = first + 1;
        while (!((t->key[split] >> b) & 1ull)) ++split;
    } else {
        /* equal keys: the augmented key's low part is the sorted position */
        int b = highest_bit64((uint64_t)(first ^ last));
        split = (last >> b) << b;
    }
    int64_t l = build_rec(t, first, split - first, depth + 1, (int32_t)id);
    int64_t r = build_rec(t, split, last + 1 - split, depth + 1, (int32_t)id);
    t->left[id] = (int32_t)l;
    t->right[id] = (int32_t)r;
    return id;
}

/* Node centre (centre of mass), size, h_max, mass and moments, each computed
 * directly from the node's particles (Sect. 3: moments per node during the
 * build; Eq. massmom). */
static void node_props(orc_tree* t, int64_t id)
{
    int64_t f = t->first[id], c = t->count[id];
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, hm = 0.0;
    for (int64_t j = f; j < f + c; ++j) {
        M += t->m[j];
        sx += t->m[j] * t->x[3 * j];
        sy += t->m[j] * t->x[3 * j + 1];
        sz += t->m[j] * t->x[3 * j + 2];
        if (t->h[j] > hm) hm = t->h[j];
    }
    double s[3] = {sx / M, sy / M, sz / M};
    double l = 0.0;
    for (int64_t j = f; j < f + c; ++j) {
        double dx = t->x[3 * j] - s[0], dy = t->x[3 * j + 1] - s[1], dz = t->x[3 * j + 2] - s[2];
        double d = sqrt(dx * dx + dy * dy + dz * dz);
        if (d > l) l = d;
    }
    t->centre[3 * id] = s[0]; t->centre[3 * id + 1] = s[1]; t->centre[3 * id + 2] = s[2];
    t->size[id] = l;
    t->hmax[id] = hm;
    t->mass[id] = M;
    p2m_direct(t->p, c, t->x + 3 * f, t->m + f, NULL, s, t->Q + id * packed_size(t->p));
}

void orc_free(orc_tree* t)
{
    if (!t) return;
    free(t->x); free(t->m); free(t->h); free(t->perm); free(t->key);
    free(t->first); free(t->count); free(t->left); free(t->right); free(t->parent); free(t->depth);
    free(t->centre); free(t->size); free(t->hmax); free(t->mass); free(t->Q); free(t->leaves);
    free(t);
}

orc_tree* orc_build(int64_t n, const double* pos, const double* m, const double* h,
                    int leaf_size, int p, int nthreads)
{
    if (n < 1 || leaf_size < 1 || p < 0 || p > ORC_PMAX) return NULL;
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->n = n; t->leaf_size = leaf_size; t->p = p;
    /* bounding box and cube extent */
    double mn[3] = {pos[0], pos[1], pos[2]}, mx[3] = {pos[0], pos[1], pos[2]};
    for (int64_t i = 1; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            if (pos[3 * i + c] < mn[c]) mn[c] = pos[3 * i + c];
            if (pos[3 * i + c] > mx[c]) mx[c] = pos[3 * i + c];
        }
    double E = 0.0;
    for (int c = 0; c < 3; ++c) if (mx[c] - mn[c] > E) E = mx[c] - mn[c];
    double scale = (E > 0.0) ? 2097152.0 / E : 0.0;
    t->bbmin[0] = mn[0]; t->bbmin[1] = mn[1]; t->bbmin[2] = mn[2];
    t->extent = E; t->scale = scale;
    keyidx* ki = (keyidx*)malloc(sizeof(keyidx) * n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k3[3];
        for (int c = 0; c < 3; ++c) {
            double v = floor((pos[3 * i + c] - mn[c]) * scale);
            uint64_t kv = (uint64_t)v;
            if (kv > 2097151ull) kv = 2097151ull;
            k3[c] = kv;
        }
        ki[i].key = morton(k3[0], k3[1], k3[2]);
        ki[i].idx = i;
    }
    qsort(ki, n, sizeof(keyidx), cmp_keyidx);
    t->x = (double*)malloc(sizeof(double) * 3 * n);
    t->m = (double*)malloc(sizeof(double) * n);
    t->h = (double*)malloc(sizeof(double) * n);
    t->perm = (int64_t*)malloc(sizeof(int64_t) * n);
    t->key = (uint64_t*)malloc(sizeof(uint64_t) * n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = ki[i].idx;
        t->perm[i] = j;
        t->key[i] = ki[i].key;
        t->x[3 * i] = pos[3 * j]; t->x[3 * i + 1] = pos[3 * j + 1]; t->x[3 * i + 2] = pos[3 * j + 2];
        t->m[i] = m[j];
        t->h[i] = h[j];
    }
    free(ki);
    int64_t cap = 2 * n + 1;
    t->first = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->count = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->left = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->right = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->parent = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->depth = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->nnodes = 0;
    build_rec(t, 0, n, 0, -1);
    int64_t nn = t->nnodes;
    t->centre = (double*)malloc(sizeof(double) * 3 * nn);
    t->size = (double*)malloc(sizeof(double) * nn);
    t->hmax = (double*)malloc(sizeof(double) * nn);
    t->mass = (double*)malloc(sizeof(double) * nn);
    t->Q = (double*)malloc(sizeof(double) * nn * packed_size(p));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t id = 0; id < nn; ++id) node_props(t, id);
    t->nleaves = 0;
    for (int64_t id = 0; id < nn; ++id) if (t->left[id] < 0) t->nleaves++;
    t->leaves = (int32_t*)malloc(sizeof(int32_t) * t->nleaves);
    int64_t k = 0;
    for (int64_t id = 0; id < nn; ++id) if (t->left[id] < 0) t->leaves[k++] = (int32_t)id;
    return t;
}

/* ------------------------------------------------------------------------ */
/* Centre-of-mass-pivot kd tree (Sect. 3: "the centre of mass ... as the     */
/* pivot position to build the kd-tree"; the axis rule is not printed).      */
/* Reading: split along the axis of largest extent of the node's particles   */
/* (ties: lowest axis) at the node's centre of mass on that axis; particles  */
/* below the pivot go left, the others right, both keeping their order.  If  */
/* one side would be empty the node is split at the middle of its order.     */
/* ------------------------------------------------------------------------ */

static int64_t build_kd_rec(orc_tree* t, int64_t first, int64_t count, int depth, int32_t parent,
                            double* tx, double* tm, double* th, int64_t* tp)
{
    int64_t id = t->nnodes++;
    t->first[id] = (int32_t)first;
    t->count[id] = (int32_t)count;
    t->parent[id] = parent;
    t->depth[id] = depth;
    t->left[id] = -1;
    t->right[id] = -1;
    if (count <= t->leaf_size) return id;
    double mn[3], mx[3], M = 0.0, sm[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3; ++c) { mn[c] = t->x[3 * first + c]; mx[c] = mn[c]; }
    for (int64_t j = first; j < first + count; ++j) {
        M += t->m[j];
        for (int c = 0; c < 3; ++c) {
            double v = t->x[3 * j + c];
            sm[c] += t->m[j] * v;
            if (v < mn[c]) mn[c] = v;
            if (v > mx[c]) mx[c] = v;
        }
    }
    int axis = 0;
    for (int c = 1; c < 3; ++c) if (mx[c] - mn[c] > mx[axis] - mn[axis]) axis = c;
    double pivot = sm[axis] / M;
    int64_t nl = 0;
    for (int64_t j = first; j < first + count; ++j) if (t->x[3 * j + axis] < pivot) ++nl;
    if (nl == 0 || nl == count) {
        nl = count / 2;  /* degenerate pivot: keep the order, split in the middle */
    } else {
        int64_t a = 0, b = nl;
        for (int64_t j = first; j < first + count; ++j) {
            int64_t d = (t->x[3 * j + axis] < pivot) ? a++ : b++;
            tx[3 * d] = t->x[3 * j]; tx[3 * d + 1] = t->x[3 * j + 1]; tx[3 * d + 2] = t->x[3 * j + 2];
            tm[d] = t->m[j]; th[d] = t->h[j]; tp[d] = t->perm[j];
        }
        memcpy(t->x + 3 * first, tx, sizeof(double) * 3 * count);
        memcpy(t->m + first, tm, sizeof(double) * count);
        memcpy(t->h + first, th, sizeof(double) * count);
        memcpy(t->perm + first, tp, sizeof(int64_t) * count);
    }
    int64_t l = build_kd_rec(t, first, nl, depth + 1, (int32_t)id, tx, tm, th, tp);
    int64_t r = build_kd_rec(t, first + nl, count - nl, depth + 1, (int32_t)id, tx, tm, th, tp);
    t->left[id] = (int32_t)l;
    t->right[id] = (int32_t)r;
    return id;
}

orc_tree* orc_build_kd(int64_t n, const double* pos, const double* m, const double* h,
                       int leaf_size, int p, int nthreads)
{
    if (n < 1 || leaf_size < 1 || p < 0 || p > ORC_PMAX) return NULL;
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->n = n; t->leaf_size = leaf_size; t->p = p;
    t->x = (double*)malloc(sizeof(double) * 3 * n);
    t->m = (double*)malloc(sizeof(double) * n);
    t->h = (double*)malloc(sizeof(double) * n);
    t->perm = (int64_t*)malloc(sizeof(int64_t) * n);
    t->key = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));  /* no keys in a kd tree */
    memcpy(t->x, pos, sizeof(double) * 3 * n);
    memcpy(t->m, m, sizeof(double) * n);
    memcpy(t->h, h, sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
    int64_t cap = 2 * n + 1;
    t->first = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->count = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->left = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->right = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->parent = (int32_t*)malloc(sizeof(int32_t) * cap);
    t->depth = (int32_t*)malloc(sizeof(int32_t) * cap);
    double* tx = (double*)malloc(sizeof(double) * 3 * n);
    double* tm = (double*)malloc(sizeof(double) * n);
    double* th = (double*)malloc(sizeof(double) * n);
    int64_t* tp = (int64_t*)malloc(sizeof(int64_t) * n);
    t->nnodes = 0;
    build_kd_rec(t, 0, n, 0, -1, tx, tm, th, tp);
    free(tx); free(tm); free(th); free(tp);
    int64_t nn = t->nnodes;
    t->centre = (double*)malloc(sizeof(double) * 3 * nn);
    t->size = (double*)malloc(sizeof(double) * nn);
    t->hmax = (double*)malloc(sizeof(double) * nn);
    t->mass = (double*)malloc(sizeof(double) * nn);
    t->Q = (double*)malloc(sizeof(double) * nn * packed_size(p));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t id = 0; id < nn; ++id) node_props(t, id);
    t->nleaves = 0;
    for (int64_t id = 0; id < nn; ++id) if (t->left[id] < 0) t->nleaves++;
    t->leaves = (int32_t*)malloc(sizeof(int32_t) * t->nleaves);
    int64_t k = 0;
    for (int64_t id = 0; id < nn; ++id) if (t->left[id] < 0) t->leaves[k++] = (int32_t)id;
    return t;
}

int64_t orc_tree_nnodes(const orc_tree* t) { return t->nnodes; }
int64_t orc_tree_nleaves(const orc_tree* t) { return t->nleaves; }

void orc_tree_export(const orc_tree* t, int64_t* perm, uint64_t* keys, int32_t* first, int32_t* count,
                     int32_t* left, int32_t* right, int32_t* parent, int32_t* depth,
                     double* centre, double* size, double* hmax, double* mass, double* Q,
                     int32_t* leaves, double* bbox /* min[3], extent, scale */)
{
    int64_t n = t->n, nn = t->nnodes;
    if (perm) memcpy(perm, t->perm, sizeof(int64_t) * n);
    if (keys) memcpy(keys, t->key, sizeof(uint64_t) * n);
    if (first) memcpy(first, t->first, sizeof(int32_t) * nn);
    if (count) memcpy(count, t->count, sizeof(int32_t) * nn);
    if (left) memcpy(left, t->left, sizeof(int32_t) * nn);
    if (right) memcpy(right, t->right, sizeof(int32_t) * nn);
    if (parent) memcpy(parent, t->parent, sizeof(int32_t) * nn);
    if (depth) memcpy(depth, t->depth, sizeof(int32_t) * nn);
    if (centre) memcpy(centre, t->centre, sizeof(double) * 3 * nn);
    if (size) memcpy(size, t->size, sizeof(double) * nn);
    if (hmax) memcpy(hmax, t->hmax, sizeof(double) * nn);
    if (mass) memcpy(mass, t->mass, sizeof(double) * nn);
    if (Q) memcpy(Q, t->Q, sizeof(double) * nn * packed_size(t->p));
    if (leaves) memcpy(leaves, t->leaves, sizeof(int32_t) * t->nleaves);
    if (bbox) { bbox[0] = t->bbmin[0]; bbox[1] = t->bbmin[1]; bbox[2] = t->bbmin[2];
                bbox[3] = t->extent; bbox[4] = t->scale; }
}

/* ------------------------------------------------------------------------ */
/* Acceptance (Sect. 3): MAC (l_t + l_s) / d < theta_crit, and the softening */
/* criterion: open when d < l_t + l_s + R_kern max(h_t, h_s).               */
/* ------------------------------------------------------------------------ */

static double node_distance(const orc_tree* t, int32_t A, int32_t B)
{
    double dx = t->centre[3 * B] - t->centre[3 * A];
    double dy = t->centre[3 * B + 1] - t->centre[3 * A + 1];
    double dz = t->centre[3 * B + 2] - t->centre[3 * A + 2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

static int mac_accept(const orc_tree* t, int32_t A, int32_t B, double theta)
{
    double d = node_distance(t, A, B);
    double lsum = t->size[A] + t->size[B];
    double hm = t->hmax[A] > t->hmax[B] ? t->hmax[A] : t->hmax[B];
    int mac = lsum < theta * d;
    int soft_open = d < lsum + ORC_RKERN * hm;
    return mac && !soft_open;
}

/* Exported for tests: the acceptance decision and its inputs. */
int orc_accept(const orc_tree* t, int32_t A, int32_t B, double theta) { return mac_accept(t, A, B, theta); }

/* ------------------------------------------------------------------------ */
/* Algorithms 1 and 2 (Sect. 3) for one leaf                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t m2l, m2l_unique, p2p_leaves, p2p_pairs, max_stack;
} orc_stats;

typedef struct {
    /* optional list recording for one leaf */
    int32_t* m2l_level; int32_t* m2l_src; int64_t m2l_n, m2l_cap;
    int32_t* p2p_src; int64_t p2p_n, p2p_cap;
} orc_lists;

typedef struct { int32_t k; int32_t s; } stack_item;

/* Walk one leaf.  parents[0..D] = root .. leaf.  M, dM: (D+1) packed
 * buffers (one per parent).  nbr: cached neighbour leaves. Returns 0 on
 * success, -1 on stack overflow.                                           */
static int walk_leaf(const orc_tree* t, const int32_t* parents, int D, double theta, int compute,
                     double* M, double* dM, int32_t* nbr, int64_t* nnbr, orc_stats* st,
                     orc_lists* lists, stack_item* stack, int64_t stack_cap)
{
    int p = t->p;
    int psz = packed_size(p), dsz = dm_size(p);
    int64_t sp = 0;
    /* push (parents(1), root): parents(1) is the root (Algorithm 1) */
    stack[sp].k = 0; stack[sp].s = 0; sp++;
    *nnbr = 0;
    while (sp > 0) {
        stack_item it = stack[--sp];
        int32_t pi = parents[it.k], ns = it.s;
        int stackit = 0;
        if (pi == ns) {
            stackit = 1;
        } else if (mac_accept(t, pi, ns, theta)) {
            st->m2l++;
            if (t->first[pi] == t->first[parents[D]]) st->m2l_unique++;
            if (lists && lists->m2l_n < lists->m2l_cap) {
                lists->m2l_level[lists->m2l_n] = it.k;
                lists->m2l_src[lists->m2l_n] = ns;
            }
            if (lists) lists->m2l_n++;
            if (compute) {
                double r[3] = {t->centre[3 * ns] - t->centre[3 * pi],
                               t->centre[3 * ns + 1] - t->centre[3 * pi + 1],
                               t->centre[3 * ns + 2] - t->centre[3 * pi + 2]};
                m2l_add(p, r, t->Q + (int64_t)ns * psz, M + (int64_t)it.k * psz, dM + (int64_t)it.k * dsz);
            }
        } else {
            stackit = 1;
        }
        if (!stackit) continue;
        int ns_leaf = t->left[ns] < 0;
        int pi_leaf = (it.k == D);
        if (ns_leaf) {
            if (pi_leaf) {
                nbr[(*nnbr)++] = ns;          /* cache_neighbours */
            } else {
                if (sp + 1 > stack_cap) return -1;
                stack[sp].k = it.k + 1; stack[sp].s = ns; sp++;
            }
        } else {
            if (sp + 2 > stack_cap) return -1;
            int kk = pi_leaf ? it.k : it.k + 1;
            stack[sp].k = kk; stack[sp].s = t->left[ns]; sp++;
            stack[sp].k = kk; stack[sp].s = t->right[ns]; sp++;
        }
        if (sp > st->max_stack) st->max_stack = sp;
    }
    return 0;
}

/* Full per-leaf pipeline: walk, propagate down the branch, evaluate at the
 * particles (far field), then the pairwise softened pass over the cached
 * neighbours (near field).  Writes acc/pot for the leaf's particles in
 * sorted order. */
static int leaf_pipeline(const orc_tree* t, int32_t leaf, double theta, double G, int self_pot,
                         double* acc_sorted, double* pot_sorted, orc_stats* st, orc_lists* lists,
                         int compute)
{
    int p = t->p;
    int psz = packed_size(p), dsz = dm_size(p);
    int32_t parents[ORC_MAXDEPTH];
    int D = t->depth[leaf];
    if (D >= ORC_MAXDEPTH) return -2;
    /* get_leaf_branch: parents from the root (index 0) to the leaf (index D) */
    int32_t v = leaf;
    for (int k = D; k >= 0; --k) { parents[k] = v; v = t->parent[v]; }
    double* M = (double*)calloc((size_t)(D + 1) * psz, sizeof(double));
    double* dM = (double*)calloc((size_t)(D + 1) * dsz, sizeof(double));
    int64_t nbr_cap = t->nleaves;
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * nbr_cap);
    int64_t stack_cap = 4 * (int64_t)t->nleaves + 64;
    stack_item* stack = (stack_item*)malloc(sizeof(stack_item) * stack_cap);
    int64_t nnbr = 0;
    int rc = walk_leaf(t, parents, D, theta, compute, M, dM, nbr, &nnbr, st, lists, stack, stack_cap);
    if (rc == 0 && lists) {
        for (int64_t q = 0; q < nnbr; ++q) {
            if (lists->p2p_n < lists->p2p_cap) lists->p2p_src[lists->p2p_n] = nbr[q];
            lists->p2p_n++;
        }
    }
    st->p2p_leaves += nnbr;
    for (int64_t q = 0; q < nnbr; ++q) {
        int64_t cl = t->count[leaf], cs = t->count[nbr[q]];
        st->p2p_pairs += cl * cs - (nbr[q] == leaf ? cl : 0);
    }
    if (rc == 0 && compute) {
        /* propagate_to_next_parent, top to bottom (Algorithm 1) */
        for (int k = 0; k < D; ++k) {
            int32_t a = parents[k], b = parents[k + 1];
            double hv[3] = {t->centre[3 * b] - t->centre[3 * a],
                            t->centre[3 * b + 1] - t->centre[3 * a + 1],
                            t->centre[3 * b + 2] - t->centre[3 * a + 2]};
            l2l_add(p, hv, M + (int64_t)k * psz, dM + (int64_t)k * dsz,
                    M + (int64_t)(k + 1) * psz, dM + (int64_t)(k + 1) * dsz);
        }
        const double* ML = M + (int64_t)D * psz;
        const double* dML = dM + (int64_t)D * dsz;
        int64_t f = t->first[leaf], c = t->count[leaf];
        for (int64_t i = f; i < f + c; ++i) {
            double a[3] = {t->x[3 * i] - t->centre[3 * leaf], t->x[3 * i + 1] - t->centre[3 * leaf + 1],
                           t->x[3 * i + 2] - t->centre[3 * leaf + 2]};
            double fa[3] = {0, 0, 0}, ph = 0.0;
            l2p(p, a, ML, dML, G, fa, &ph);
            /* short-range interactions over the cached neighbours */
            for (int64_t q = 0; q < nnbr; ++q) {
                int32_t S = nbr[q];
                for (int64_t j = t->first[S]; j < t->first[S] + t->count[S]; ++j) {
                    if (j == i) continue;
                    double d[3] = {t->x[3 * i] - t->x[3 * j], t->x[3 * i + 1] - t->x[3 * j + 1],
                                   t->x[3 * i + 2] - t->x[3 * j + 2]};
                    pair_softened(d, t->h[i], t->m[j], t->h[j], G, fa, &ph);
                }
            }
            if (self_pot) ph += G * t->m[i] * kernel_phi(0.0, t->h[i]);
            acc_sorted[3 * i] = fa[0]; acc_sorted[3 * i + 1] = fa[1]; acc_sorted[3 * i + 2] = fa[2];
            pot_sorted[i] = ph;
        }
    }
    free(M); free(dM); free(nbr); free(stack);
    return rc;
}

/* SFMM over all leaves (or a subset: leaf_ids != NULL, nsel of them).
 * acc/pot are returned in CALLER order (particles outside the selected
 * leaves are left untouched).  stats: [m2l, m2l_unique, p2p_leaves,
 * p2p_pairs, max_stack].  Returns 0, or -1 on a stack overflow.           */
int orc_sfmm(const orc_tree* t, double theta, double G, int self_pot,
             int64_t nsel, const int32_t* leaf_ids, double* acc, double* pot,
             int64_t* stats, int nthreads)
{
    int64_t n = t->n;
    double* as = (double*)calloc((size_t)3 * n, sizeof(double));
    double* ps = (double*)calloc((size_t)n, sizeof(double));
    int64_t nl = leaf_ids ? nsel : t->nleaves;
    int64_t s_m2l = 0, s_u = 0, s_pl = 0, s_pp = 0, s_ms = 0;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : s_m2l, s_u, s_pl, s_pp) reduction(max : s_ms) reduction(| : err)
#endif
    for (int64_t q = 0; q < nl; ++q) {
        int32_t leaf = leaf_ids ? t->leaves[leaf_ids[q]] : t->leaves[q];
        orc_stats st = {0, 0, 0, 0, 0};
        int rc = leaf_pipeline(t, leaf, theta, G, self_pot, as, ps, &st, NULL, 1);
        if (rc) err |= 1;
        s_m2l += st.m2l; s_u += st.m2l_unique; s_pl += st.p2p_leaves; s_pp += st.p2p_pairs;
        if (st.max_stack > s_ms) s_ms = st.max_stack;
    }
    for (int64_t q = 0; q < nl; ++q) {
        int32_t leaf = leaf_ids ? t->leaves[leaf_ids[q]] : t->leaves[q];
        for (int64_t i = t->first[leaf]; i < t->first[leaf] + t->count[leaf]; ++i) {
            int64_t j = t->perm[i];
            acc[3 * j] = as[3 * i]; acc[3 * j + 1] = as[3 * i + 1]; acc[3 * j + 2] = as[3 * i + 2];
            pot[j] = ps[i];
        }
    }
    free(as); free(ps);
    if (stats) { stats[0] = s_m2l; stats[1] = s_u; stats[2] = s_pl; stats[3] = s_pp; stats[4] = s_ms; }
    return err ? -1 : 0;
}

/* Interaction lists of every leaf (decisions only, no arithmetic).
 * Pass NULL arrays to obtain the sizes first (m2l_off/p2p_off are always
 * filled, nleaves + 1 entries).  Entries are in walk order.                */
int orc_lists_dump(const orc_tree* t, double theta, int64_t* m2l_off, int32_t* m2l_level,
                   int32_t* m2l_src, int64_t* p2p_off, int32_t* p2p_src)
{
    int64_t mo = 0, po = 0;
    int err = 0;
    for (int64_t q = 0; q < t->nleaves; ++q) {
        orc_stats st = {0, 0, 0, 0, 0};
        orc_lists L;
        L.m2l_level = m2l_level ? m2l_level + mo : NULL;
        L.m2l_src = m2l_src ? m2l_src + mo : NULL;
        L.m2l_n = 0;
        L.m2l_cap = m2l_level ? (int64_t)1 << 62 : 0;
        L.p2p_src = p2p_src ? p2p_src + po : NULL;
        L.p2p_n = 0;
        L.p2p_cap = p2p_src ? (int64_t)1 << 62 : 0;
        m2l_off[q] = mo;
        p2p_off[q] = po;
        if (leaf_pipeline(t, t->leaves[q], theta, 1.0, 0, NULL, NULL, &st, &L, 0)) err = 1;
        mo += L.m2l_n;
        po += L.p2p_n;
    }
    m2l_off[t->nleaves] = mo;
    p2p_off[t->nleaves] = po;
    return err ? -1 : 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
