"""ctypes wrapper of the plain FP64 C oracle (``sfmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg are the only callers.  The CUDA
solver never imports this package and shares no code with it.

Parity status per function (how each is pinned; see tests/test_oracle_*.py):
  kernel (M4 softening)      pinned: published closed-form values, continuity,
                             Poisson density = M4 kernel, unit mass integral
  direct                     pinned: two-body law, uniform-sphere and Plummer
                             closed forms, Newton's third law
  derivs (D_gamma)           pinned: closed forms to order 2, Laplace trace,
                             finite differences to order 5
  p2m / m2m                  pinned: brute-force moments, shift identity
  m2l / l2l / l2p            pinned: exact for single particles (a = b),
                             geometric convergence in p, shift invariance
  build (tree)               pinned: brute-force partition, split rule,
                             centre/size/h_max recomputed by hand
  sfmm (Algorithms 1-2)      pinned: theta = 0 equals the direct sum, list
                             symmetry, momentum to round-off, an independent
                             recursive dual-tree walk gives the same pairs
  leapfrog (kick-drift-kick) pinned: exact time reversal, Kepler two-body
                             orbit closes with O(dt^2) energy error, linear
                             momentum constant to round-off
  softening pair rule        parity unpinned: the paper does not print how the
                             two smoothing lengths of a pair combine (mean of
                             the two kernels is the reading taken)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfmm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsfmm_oracle.so")
_lock = threading.Lock()
_lib = None

PMAX = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.orc_build.restype = P
            lib.orc_build.argtypes = [i64, P, P, P, i32, i32, i32]
            lib.orc_build_kd.restype = P
            lib.orc_build_kd.argtypes = [i64, P, P, P, i32, i32, i32]
            lib.orc_free.argtypes = [P]
            lib.orc_tree_nnodes.restype = i64
            lib.orc_tree_nnodes.argtypes = [P]
            lib.orc_tree_nleaves.restype = i64
            lib.orc_tree_nleaves.argtypes = [P]
            lib.orc_tree_export.argtypes = [P] + [P] * 15
            lib.orc_sfmm.restype = i32
            lib.orc_sfmm.argtypes = [P, dbl, dbl, i32, i64, P, P, P, P, i32]
            lib.orc_lists_dump.restype = i32
            lib.orc_lists_dump.argtypes = [P, dbl, P, P, P, P, P]
            lib.orc_accept.restype = i32
            lib.orc_accept.argtypes = [P, i32, i32, dbl]
            lib.orc_direct.argtypes = [i64, P, P, P, dbl, i32, i64, P, P, P, i32]
            lib.orc_kernel.argtypes = [i64, P, P, P, P]
            lib.orc_derivs.argtypes = [i32, P, i32, P, P]
            lib.orc_p2m.argtypes = [i32, i64, P, P, P, P]
            lib.orc_m2m.argtypes = [i32, P, P, P]
            lib.orc_m2l_eval.argtypes = [i32, P, P, i64, P, P, i64, P, dbl, P, P]
            lib.orc_m2l_l2l_eval.argtypes = [i32, P, P, P, i64, P, P, i64, P, dbl, P, P]
            lib.orc_m2l_coeffs.argtypes = [i32, P, P, P, P]
            lib.orc_packed_size.restype = i32
            lib.orc_packed_size.argtypes = [i32]
            lib.orc_dm_size.restype = i32
            lib.orc_dm_size.argtypes = [i32]
            lib.orc_max_threads.restype = i32
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return _load().orc_max_threads()


# --------------------------------------------------------------------------
# Kernel and direct sum
# --------------------------------------------------------------------------

def kernel(r, h):
    """M4 softening kernel: returns (phi(r,h), g(r,h)) with phi -> -1/r and
    g = phi'(r)/r -> 1/r^3 outside 2h."""
    r = _f64(np.atleast_1d(r))
    h = _f64(np.broadcast_to(h, r.shape))
    phi = np.empty_like(r)
    g = np.empty_like(r)
    _load().orc_kernel(r.size, _p(r), _p(h), _p(phi), _p(g))
    return phi, g


def direct(pos, m, h, G=1.0, self_potential=False, targets=None, nthreads=0):
    """Softened O(N^2) direct sum; returns (acc (nt,3), pot (nt,))."""
    pos = _f64(pos, (-1, 3))
    m, h = _f64(m), _f64(h)
    n = len(m)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else len(t)
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    _load().orc_direct(n, _p(pos), _p(m), _p(h), float(G), int(bool(self_potential)), nt, _p(t),
                       _p(acc), _p(pot), int(nthreads))
    return acc, pot


# --------------------------------------------------------------------------
# Expansion pieces
# --------------------------------------------------------------------------

def derivs(P, r, gammas):
    """D_gamma(r) = d^gamma (1/|r|) for the given multi-indices (k x 3)."""
    g = np.ascontiguousarray(gammas, dtype=np.int32).reshape(-1, 3)
    r = _f64(r)
    out = np.empty(len(g))
    _load().orc_derivs(int(P), _p(r), len(g), _p(g), _p(out))
    return out


def packed_size(p):
    return _load().orc_packed_size(p)


def dm_size(p):
    return _load().orc_dm_size(p)


def rank_offset(n):
    return sum(3 ** k for k in range(n))


def p2m(p, pos, m, centre):
    """Full-tensor mass moments Q_0..Q_p about centre, packed by rank."""
    pos = _f64(pos, (-1, 3))
    m = _f64(m)
    Q = np.zeros(packed_size(p))
    _load().orc_p2m(int(p), len(m), _p(pos), _p(m), _p(_f64(centre)), _p(Q))
    return Q


def m2m(p, Qc, g):
    Qc = _f64(Qc)
    Qp = np.zeros(packed_size(p))
    _load().orc_m2m(int(p), _p(Qc), _p(_f64(g)), _p(Qp))
    return Qp


def m2l_eval(p, sA, sB, xB, mB, xA, G=1.0):
    """Expand the particles of B about sB, translate to sA (M2L) and evaluate
    at the points xA about sA."""
    xB, xA, mB = _f64(xB, (-1, 3)), _f64(xA, (-1, 3)), _f64(mB)
    acc = np.zeros((len(xA), 3))
    pot = np.zeros(len(xA))
    _load().orc_m2l_eval(int(p), _p(_f64(sA)), _p(_f64(sB)), len(mB), _p(xB), _p(mB), len(xA), _p(xA),
                         float(G), _p(acc), _p(pot))
    return acc, pot


def m2l_l2l_eval(p, sA, sA2, sB, xB, mB, xA, G=1.0):
    xB, xA, mB = _f64(xB, (-1, 3)), _f64(xA, (-1, 3)), _f64(mB)
    acc = np.zeros((len(xA), 3))
    pot = np.zeros(len(xA))
    _load().orc_m2l_l2l_eval(int(p), _p(_f64(sA)), _p(_f64(sA2)), _p(_f64(sB)), len(mB), _p(xB), _p(mB),
                             len(xA), _p(xA), float(G), _p(acc), _p(pot))
    return acc, pot


def m2l_coeffs(p, r, Q):
    """Raw M (packed ranks 0..p) and dM (packed ranks 1..p+1) of one M2L."""
    M = np.zeros(packed_size(p))
    dM = np.zeros(dm_size(p))
    _load().orc_m2l_coeffs(int(p), _p(_f64(r)), _p(_f64(Q)), _p(M), _p(dM))
    return M, dM


def full_index(gamma):
    """Row-major full-tensor index of the sorted axis tuple of a multi-index."""
    axes = [0] * gamma[0] + [1] * gamma[1] + [2] * gamma[2]
    idx = 0
    for a in axes:
        idx = idx * 3 + a
    return idx


# --------------------------------------------------------------------------
# Tree and SFMM
# --------------------------------------------------------------------------

class Tree:
    """Oracle tree: sorted particles, nodes in pre-order, direct moments."""

    def __init__(self, pos, m, h, leaf_size, p=2, nthreads=0, tree="morton"):
        self._lib = _load()
        if tree not in ("morton", "kd"):
            raise ValueError("tree must be 'morton' or 'kd'")
        self.tree = tree
        self.pos = _f64(pos, (-1, 3))
        self.m, self.h = _f64(m), _f64(h)
        self.n = len(self.m)
        self.p = int(p)
        self.leaf_size = int(leaf_size)
        build = self._lib.orc_build_kd if tree == "kd" else self._lib.orc_build
        ptr = build(self.n, _p(self.pos), _p(self.m), _p(self.h), self.leaf_size, self.p, int(nthreads))
        if not ptr:
            raise ValueError("oracle tree build rejected its arguments")
        self._ptr = ctypes.c_void_p(ptr)
        self.nnodes = self._lib.orc_tree_nnodes(self._ptr)
        self.nleaves = self._lib.orc_tree_nleaves(self._ptr)
        nn, n = self.nnodes, self.n
        self.perm = np.empty(n, np.int64)
        self.keys = np.empty(n, np.uint64)
        self.first = np.empty(nn, np.int32)
        self.count = np.empty(nn, np.int32)
        self.left = np.empty(nn, np.int32)
        self.right = np.empty(nn, np.int32)
        self.parent = np.empty(nn, np.int32)
        self.depth = np.empty(nn, np.int32)
        self.centre = np.empty((nn, 3))
        self.size = np.empty(nn)
        self.hmax = np.empty(nn)
        self.mass = np.empty(nn)
        self.Q = np.empty((nn, packed_size(self.p)))
        self.leaves = np.empty(self.nleaves, np.int32)
        self.bbox = np.empty(5)
        self._lib.orc_tree_export(self._ptr, *[_p(a) for a in (
            self.perm, self.keys, self.first, self.count, self.left, self.right, self.parent,
            self.depth, self.centre, self.size, self.hmax, self.mass, self.Q, self.leaves, self.bbox)])

    def __del__(self):
        ptr = getattr(self, "_ptr", None)
        if ptr is not None and ptr.value:
            self._lib.orc_free(ptr)
            self._ptr = None

    def accept(self, A, B, theta):
        return bool(self._lib.orc_accept(self._ptr, int(A), int(B), float(theta)))

    def sfmm(self, theta, G=1.0, self_potential=False, leaf_sample=None, nthreads=0):
        """Run Algorithms 1-2 for every leaf (or the given leaf indices).
        Returns (acc, pot, stats) in caller order; stats keys m2l, m2l_unique,
        p2p_leaves, p2p_pairs, max_stack."""
        acc = np.zeros((self.n, 3))
        pot = np.zeros(self.n)
        st = np.zeros(5, np.int64)
        sel = None if leaf_sample is None else np.ascontiguousarray(leaf_sample, dtype=np.int32)
        rc = self._lib.orc_sfmm(self._ptr, float(theta), float(G), int(bool(self_potential)),
                                0 if sel is None else len(sel), _p(sel), _p(acc), _p(pot), _p(st),
                                int(nthreads))
        if rc != 0:
            raise RuntimeError("oracle walk stack overflow")
        keys = ("m2l", "m2l_unique", "p2p_leaves", "p2p_pairs", "max_stack")
        return acc, pot, dict(zip(keys, (int(v) for v in st)))

    def lists(self, theta):
        """Per-leaf interaction lists in walk order: (m2l_off, m2l_level,
        m2l_src, p2p_off, p2p_src); offsets have nleaves + 1 entries."""
        mo = np.zeros(self.nleaves + 1, np.int64)
        po = np.zeros(self.nleaves + 1, np.int64)
        self._lib.orc_lists_dump(self._ptr, float(theta), _p(mo), None, None, _p(po), None)
        lv = np.empty(mo[-1], np.int32)
        src = np.empty(mo[-1], np.int32)
        ps = np.empty(po[-1], np.int32)
        rc = self._lib.orc_lists_dump(self._ptr, float(theta), _p(mo), _p(lv), _p(src), _p(po), _p(ps))
        if rc != 0:
            raise RuntimeError("oracle walk stack overflow")
        return mo, lv, src, po, ps


def _momentum_record(t, x, v, m):
    p = m[:, None] * v
    return np.concatenate([[t], p.sum(0), np.cross(x, p).sum(0), [np.abs(p).sum()]])


def leapfrog(pos, vel, m, h, theta, p=2, leaf_size=16, dt=0.01, nsteps=1, record_every=1, G=1.0, nthreads=0):
    """Gravity-only kick-drift-kick leapfrog with these SFMM accelerations
    (the integration of the binary-polytrope test, Sect. 4): v += a dt/2,
    x += v dt, new tree and accelerations, v += a dt/2.  Returns (pos, vel,
    records); a record (t, P = sum m v, L = sum m x cross v, sum |m v_d|) is
    taken before the first step and after every record_every-th step."""
    x = np.array(pos, dtype=np.float64, copy=True)
    v = np.array(vel, dtype=np.float64, copy=True)
    m = np.asarray(m, dtype=np.float64)
    hdt = 0.5 * dt
    a, _, _ = sfmm(x, m, h, theta, p, leaf_size, G=G, nthreads=nthreads)
    recs = [_momentum_record(0.0, x, v, m)]
    for s in range(1, int(nsteps) + 1):
        v = v + a * hdt
        x = x + v * dt
        a, _, _ = sfmm(x, m, h, theta, p, leaf_size, G=G, nthreads=nthreads)
        v = v + a * hdt
        if s % record_every == 0:
            recs.append(_momentum_record(s * dt, x, v, m))
    return x, v, np.array(recs)


def sfmm(pos, m, h, theta, p=2, leaf_size=10, G=1.0, self_potential=False, nthreads=0, tree="morton"):
    """Convenience: build the oracle tree and run the SFMM; returns
    (acc, pot, stats)."""
    t = Tree(pos, m, h, leaf_size, p, nthreads=nthreads, tree=tree)
    return t.sfmm(theta, G=G, self_potential=self_potential, nthreads=nthreads)
