"""Derive the golden M4 softening values symbolically from the M4 density.

Independent of the oracle's polynomials: starts from the cubic-spline
density W(q) (Monaghan & Lattanzio 1985; the softening kernel the paper
cites in Sect. 2, Price & Monaghan 2007), integrates the enclosed mass
M(q) = int 4 pi x^2 W dx, and forms g(q) = M(q)/q^3 and
phi(q) = -int_q^inf M(x)/x^2 dx (h = 1).  Writes m4_softening.txt.
"""
import os

import sympy as sp

x, q = sp.symbols("x q", positive=True)
W1 = (1 - sp.Rational(3, 2) * x**2 + sp.Rational(3, 4) * x**3) / sp.pi
W2 = (2 - x) ** 3 / (4 * sp.pi)


def mass(qv):
    if qv <= 1:
        return sp.integrate(4 * sp.pi * x**2 * W1, (x, 0, qv))
    m1 = sp.integrate(4 * sp.pi * x**2 * W1, (x, 0, 1))
    if qv <= 2:
        return m1 + sp.integrate(4 * sp.pi * x**2 * W2, (x, 1, qv))
    return m1 + sp.integrate(4 * sp.pi * x**2 * W2, (x, 1, 2))


def enclosed(xx):
    return sp.Piecewise(
        (sp.integrate(4 * sp.pi * q**2 * W1.subs(x, q), (q, 0, xx)), xx <= 1),
        (sp.integrate(4 * sp.pi * q**2 * W1.subs(x, q), (q, 0, 1))
         + sp.integrate(4 * sp.pi * q**2 * W2.subs(x, q), (q, 1, xx)), xx <= 2),
        (1, True))


def phi(qv):
    # -int_q^inf M(x)/x^2 dx, split at 1 and 2
    total = 0
    edges = [qv] + [e for e in (1, 2) if e > qv]
    for a, b in zip(edges[:-1], edges[1:]):
        mid = (a + b) / 2
        if mid < 1:
            Mx = sp.integrate(4 * sp.pi * q**2 * W1.subs(x, q), (q, 0, x))
        else:
            Mx = mass(1) + sp.integrate(4 * sp.pi * q**2 * W2.subs(x, q), (q, 1, x))
        total += sp.integrate(Mx / x**2, (x, a, b))
    tail = 1 / max(qv, 2)
    return -(total + tail)


rows = []
for qv in (sp.Integer(0), sp.Integer(1), sp.Integer(2), sp.Integer(3), sp.Rational(1, 2), sp.Rational(3, 2)):
    M = mass(qv)
    g = sp.limit(sp.integrate(4 * sp.pi * x**2 * W1, (x, 0, q)) / q**3, q, 0) if qv == 0 else M / qv**3
    rows.append((float(qv), float(sp.nsimplify(phi(qv))), float(g)))

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "m4_softening.txt")
with open(out, "w") as f:
    f.write("# Closed-form values of the cubic-spline (M4) softening kernel, compact\n")
    f.write("# support 2h, h = 1: the softening kernel cited for the softened sum\n")
    f.write("# (Sect. 2, Eq. softdirectsum; Price & Monaghan 2007).  Written by\n")
    f.write("# make_m4_softening.py, which integrates the M4 density symbolically.\n")
    f.write("# columns: q  phi(q)  g(q) = phi'(q)/q\n")
    for r in rows:
        f.write("%.17g %.17g %.17g\n" % r)
print(open(out).read())
