"""Generate straight-line Cartesian expansion code for the CUDA kernels.

Writes ``expansion_gen.cuh``: for every order p = 0..4 a set of
``__device__`` functions, templated on the arithmetic type T, over
*scaled* symmetric coefficients (multi-index alpha = (a,b,c); scaled means
divided by alpha! = a! b! c!):

  sfmm_mono_K(v, out)     out[alpha] = v^alpha / alpha!        |alpha| <= K
  sfmm_derivs_K(u, rinv, D)  D[gamma] = d^gamma (1/|r|)        |gamma| <= K
                          from the unit vector u = r/|r| and rinv = 1/|r|
                          (McMurchie-Davidson recurrence in u, then the
                          factor rinv^(|gamma|+1): no overflow in FP32)
  sfmm_m2l_p(D, Q, C)     C[0..NM) += M_beta, C[NM..NM+NF) += F_gamma
                          (Sect. 2.2; Q scaled moments, dipole optional)
  sfmm_l2p_p(am, C, out)  potential and acceleration polynomials at a
  sfmm_m2m_p(gm, Qc, Qp)  Qp[alpha] += sum_{beta<=alpha} gm[alpha-beta] Qc[beta]
  constant tables for the lane-parallel L2L translation (App. A.2)

The layout of a coefficient vector C of order p is [M_beta for |beta| <= p]
followed by [F_gamma for 1 <= |gamma| <= p+1]; multi-indices are ordered by
degree, then a descending, then b descending.

Run: python gen_expansion.py  (build() runs it before compiling).
"""
import os
from math import factorial

PMAX = 4


def mis(K, lo=0):
    return [(a, b, n - a - b) for n in range(lo, K + 1) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


def idx_of(K, lo=0):
    return {g: i for i, g in enumerate(mis(K, lo))}


def deg(g):
    return sum(g)


def sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def geq(a, b):
    return all(x >= y for x, y in zip(a, b))


def lit(v):
    """A literal of type T (cast from a double literal)."""
    return "T(%r)" % float(v)


def gen_mono(K):
    I = idx_of(K)
    lines = ["template <typename T> __device__ __forceinline__ void sfmm_mono_%d(T vx, T vy, T vz, T* o) {" % K]
    lines.append("  o[0] = T(1);")
    comp = ["vx", "vy", "vz"]
    for g in mis(K, 1):
        t = next(i for i in range(3) if g[i] > 0)
        prev = list(g)
        prev[t] -= 1
        f = g[t]
        if f == 1:
            lines.append("  o[%d] = o[%d] * %s;" % (I[g], I[tuple(prev)], comp[t]))
        else:
            lines.append("  o[%d] = o[%d] * (%s * %s);" % (I[g], I[tuple(prev)], comp[t], lit(1.0 / f)))
    lines.append("}")
    return "\n".join(lines)


def gen_derivs(K):
    """D_gamma for |gamma| <= K via R^(m)_gamma in the unit vector u."""
    I = idx_of(K)
    stmts = []
    have = {}

    def R(m, g):
        key = (m, g)
        if key in have:
            return have[key]
        if deg(g) == 0:
            df = 1
            for k in range(2 * m - 1, 1, -2):
                df *= k
            val = lit(((-1) ** m) * df)
            have[key] = val
            return val
        t = next(i for i in range(3) if g[i] > 0)
        g1 = list(g)
        g1[t] -= 1
        a = R(m + 1, tuple(g1))
        name = "R%d_%d%d%d" % (m, g[0], g[1], g[2])
        expr = "u%s * %s" % ("xyz"[t], a)
        if g[t] > 1:
            g2 = list(g)
            g2[t] -= 2
            b = R(m + 1, tuple(g2))
            expr = "fma(u%s, %s, %s * %s)" % ("xyz"[t], a, lit(g[t] - 1), b)
        stmts.append("  const T %s = %s;" % (name, expr))
        have[key] = name
        return name

    body = []
    for g in mis(K):
        R(0, g)
    lines = ["template <typename T> __device__ __forceinline__ void sfmm_derivs_%d(T ux, T uy, T uz, T rinv, T* D) {" % K]
    lines += stmts
    # powers of rinv
    lines.append("  T s = rinv;")
    for n in range(K + 1):
        for g in mis(n, n):
            lines.append("  D[%d] = %s * s;" % (I[g], have[(0, g)]))
        if n < K:
            lines.append("  s = s * rinv;")
    lines.append("}")
    return "\n".join(lines)


def gen_m2l(p, skip_dipole):
    """C[M_beta] += (-1)^|b| sum_{|a|<=p-|b|} D[a+b] Q[a];
    C[NM + F_gamma] += (-1)^|g| sum_{|a|<=p+1-|g|} D[a+g] Q[a]."""
    ID = idx_of(p + 1)
    IQ = idx_of(p)
    NM = len(mis(p))
    IF = idx_of(p + 1, 1)
    lines = ["template <typename T> __device__ __forceinline__ void sfmm_m2l_%d%s(const T* D, const T* Q, T* C) {"
             % (p, "_nodip" if skip_dipole else "")]
    for b in mis(p):
        terms = [(a, ID[add(a, b)]) for a in mis(p - deg(b)) if not (skip_dipole and deg(a) == 1)]
        lines.append("  { T s = D[%d] * Q[0];" % terms[0][1])
        for a, d in terms[1:]:
            lines.append("    s = fma(D[%d], Q[%d], s);" % (d, IQ[a]))
        op = "+=" if deg(b) % 2 == 0 else "-="
        lines.append("    C[%d] %s s; }" % (IQ[b], op))
    for g in mis(p + 1, 1):
        terms = [(a, ID[add(a, g)]) for a in mis(p + 1 - deg(g)) if not (skip_dipole and deg(a) == 1)]
        lines.append("  { T s = D[%d] * Q[0];" % terms[0][1])
        for a, d in terms[1:]:
            lines.append("    s = fma(D[%d], Q[%d], s);" % (d, IQ[a]))
        op = "+=" if deg(g) % 2 == 0 else "-="
        lines.append("    C[%d] %s s; }" % (NM + IF[g], op))
    lines.append("}")
    return "\n".join(lines)


def gen_l2p(p):
    """phi = sum_b am[b] M_b ; acc_d = sum_b am[b] F_{b+e_d} (signs and G
    applied by the caller: Phi = -G phi, a = +G acc)."""
    IQ = idx_of(p)
    NM = len(mis(p))
    IF = idx_of(p + 1, 1)
    lines = ["template <typename T, typename C_T> __device__ __forceinline__ void sfmm_l2p_%d(const T* am, const C_T* C, T* out) {" % p]
    lines.append("  T phi = T(0), ax = T(0), ay = T(0), az = T(0);")
    for b in mis(p):
        i = IQ[b]
        lines.append("  phi = fma(am[%d], T(C[%d]), phi);" % (i, i))
        for d, nm in enumerate(("ax", "ay", "az")):
            e = [0, 0, 0]
            e[d] = 1
            lines.append("  %s = fma(am[%d], T(C[%d]), %s);" % (nm, i, NM + IF[add(b, tuple(e))], nm))
    lines.append("  out[0] = phi; out[1] = ax; out[2] = ay; out[3] = az;")
    lines.append("}")
    return "\n".join(lines)


def gen_m2m(p):
    IQ = idx_of(p)
    lines = ["template <typename T> __device__ __forceinline__ void sfmm_m2m_%d(const T* gm, const T* Qc, T* Qp) {" % p]
    for a in mis(p):
        terms = [(IQ[sub(a, b)], IQ[b]) for b in mis(p) if geq(a, b)]
        lines.append("  { T s = Qp[%d];" % IQ[a])
        for gi, bi in terms:
            lines.append("    s = fma(gm[%d], Qc[%d], s);" % (gi, bi))
        lines.append("    Qp[%d] = s; }" % IQ[a])
    lines.append("}")
    return "\n".join(lines)


def gen_tables(p):
    """Lane-parallel L2L: for target coefficient i and source j of the same
    block (M or F) with gamma_j >= beta_i, index of h^(gamma_j - beta_i)/()!
    in sfmm_mono_{p+1}; -1 otherwise."""
    IM = mis(p)
    IF = mis(p + 1, 1)
    allc = [("M", g) for g in IM] + [("F", g) for g in IF]
    Imono = idx_of(p + 1)
    n = len(allc)
    rows = []
    for i, (bi, b) in enumerate(allc):
        row = []
        for j, (bj, g) in enumerate(allc):
            row.append(Imono[sub(g, b)] if (bi == bj and geq(g, b)) else -1)
        rows.append(row)
    body = ",\n  ".join("{" + ", ".join("%d" % v for v in r) + "}" for r in rows)
    mi_rows = ", ".join("{%d,%d,%d}" % g for g in IM)
    return ("static __device__ const signed char sfmm_l2l_table_%d[%d][%d] = {\n  %s};\n" % (p, n, n, body)
            + "static const int sfmm_moment_mi_%d[%d][3] = {%s};\n" % (p, len(IM), mi_rows))


def main():
    out = [
        "// GENERATED by gen_expansion.py -- do not edit by hand.",
        "// Straight-line Cartesian expansion pieces over scaled symmetric",
        "// coefficients (multi-index alpha, divided by alpha!).  Multi-indices are",
        "// ordered by degree, then a descending, then b descending.",
        "#pragma once",
        "",
    ]
    for p in range(PMAX + 1):
        nm = len(mis(p))
        nf = len(mis(p + 1, 1))
        out.append("#define SFMM_NM_%d %d  /* potential coefficients, |beta| <= %d */" % (p, nm, p))
        out.append("#define SFMM_NF_%d %d  /* acceleration coefficients, 1 <= |gamma| <= %d */" % (p, nf, p + 1))
    out.append("")
    for K in range(PMAX + 2):
        out.append(gen_mono(K))
        out.append("")
    for K in range(1, PMAX + 2):
        out.append(gen_derivs(K))
        out.append("")
    for p in range(PMAX + 1):
        out.append(gen_m2l(p, False))
        out.append("")
        out.append(gen_m2l(p, True))
        out.append("")
        out.append(gen_l2p(p))
        out.append("")
        out.append(gen_m2m(p))
        out.append("")
        out.append(gen_tables(p))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expansion_gen.cuh")
    text = "\n".join(out) + "\n"
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)
    return path


if __name__ == "__main__":
    print(main())
