"""Thin ctypes binding of the C ABI in ``include/sfmm.h``.

Argument marshalling only: every step of the solver runs in the CUDA
library ``_build/libsfmm.so``.  Loading fails loudly when the library is
missing; there is no CPU fallback.  Functions carry the C names; the
``Solver`` class is a convenience wrapper over them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfmm.so")

SFMM_OK, SFMM_EINVAL, SFMM_ENOMEM, SFMM_ECUDA, SFMM_ESTATE = 0, 1, 2, 3, 4
SFMM_ESTACK, SFMM_ECAPACITY, SFMM_ENONFINITE, SFMM_ENOTIMPL = 5, 6, 7, 8
SFMM_FP64, SFMM_FP32 = 0, 1

# every symbol include/sfmm.h declares
EXPORTS = ("sfmm_create", "sfmm_destroy", "sfmm_set_stream", "sfmm_set_option", "sfmm_build", "sfmm_gravity",
           "sfmm_solve_host", "sfmm_get_stats", "sfmm_tree_size", "sfmm_tree_export", "sfmm_moments_export",
           "sfmm_lists", "sfmm_strerror", "sfmm_last_error", "sfmm_version", "sfmm_reduce_noalloc",
           "sfmm_build_batch", "sfmm_gravity_batch", "sfmm_batch_sums", "sfmm_leapfrog", "sfmm_fma_peak",
           "sfmm_autotune_batch", "sfmm_autotune_cache", "sfmm_solve_graph")
SFMM_NOALLOC_MAX_N = 67108864


class sfmm_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnodes", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("m2l", ctypes.c_int64), ("m2l_unique", ctypes.c_int64), ("p2p_leaves", ctypes.c_int64),
                ("p2p_pairs", ctypes.c_int64), ("mac_fallbacks", ctypes.c_int64),
                ("momentum", ctypes.c_double * 3), ("abs_momentum", ctypes.c_double), ("W", ctypes.c_double),
                ("ms_build", ctypes.c_double), ("ms_moments", ctypes.c_double), ("ms_walk", ctypes.c_double),
                ("ms_p2p", ctypes.c_double), ("ms_reduce", ctypes.c_double), ("ms_gravity", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("graph_replays", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["momentum"] = list(self.momentum)
        return d


class SFMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sfmm error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libsfmm.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libsfmm.so not found at %s; run paper_2602_05804_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.sfmm_create.argtypes = [ctypes.POINTER(P), i32, i32, P]
    lib.sfmm_destroy.argtypes = [P]
    lib.sfmm_destroy.restype = None
    lib.sfmm_set_stream.argtypes = [P, P]
    lib.sfmm_set_option.argtypes = [P, ctypes.c_char_p, dbl]
    lib.sfmm_build.argtypes = [P, i64, P, P, P, i32]
    lib.sfmm_gravity.argtypes = [P, dbl, i32, P, P]
    lib.sfmm_solve_host.argtypes = [P, i64, P, P, P, i32, dbl, i32, P, P]
    lib.sfmm_get_stats.argtypes = [P, ctypes.POINTER(sfmm_stats)]
    lib.sfmm_tree_size.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.sfmm_tree_export.argtypes = [P] + [P] * 12
    lib.sfmm_moments_export.argtypes = [P, i32, P, P]
    lib.sfmm_lists.argtypes = [P, dbl, P, P, P, i64, P, P, i64]
    lib.sfmm_strerror.argtypes = [i32]
    lib.sfmm_strerror.restype = ctypes.c_char_p
    lib.sfmm_last_error.argtypes = [P]
    lib.sfmm_last_error.restype = ctypes.c_char_p
    lib.sfmm_version.restype = ctypes.c_char_p
    lib.sfmm_build_batch.argtypes = [P, i32, P, P, P, P, P]
    lib.sfmm_gravity_batch.argtypes = [P, dbl, i32, P, P]
    lib.sfmm_batch_sums.argtypes = [P, i32, P]
    lib.sfmm_reduce_noalloc.argtypes = [i64, P, P, P, P, P]
    lib.sfmm_reduce_noalloc.restype = i32
    lib.sfmm_leapfrog.argtypes = [P, i64, P, P, P, P, i32, dbl, i32, dbl, i64, i64, P, P]
    lib.sfmm_fma_peak.argtypes = [i32, i32, P, dbl, i32, P, P]
    lib.sfmm_fma_peak.restype = i32
    lib.sfmm_autotune_batch.argtypes = [P, i32, P, P, P, P, dbl, i32, P]
    lib.sfmm_autotune_cache.argtypes = [P, ctypes.c_char_p]
    lib.sfmm_solve_graph.argtypes = [P, i32, P, P, P, P, P, dbl, i32, P, P]
    for name in ("sfmm_create", "sfmm_set_stream", "sfmm_set_option", "sfmm_build", "sfmm_gravity",
                 "sfmm_solve_host", "sfmm_get_stats", "sfmm_tree_size", "sfmm_tree_export", "sfmm_moments_export",
                 "sfmm_lists", "sfmm_build_batch", "sfmm_gravity_batch", "sfmm_batch_sums", "sfmm_leapfrog", "sfmm_fma_peak",
           "sfmm_autotune_batch", "sfmm_autotune_cache", "sfmm_solve_graph"):
        getattr(lib, name).restype = i32
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != SFMM_OK:
        lib = load()
        msg = lib.sfmm_last_error(ctx).decode() if ctx else lib.sfmm_strerror(rc).decode()
        raise SFMMError(rc, msg)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


# --- C-named wrappers (marshalling only) ------------------------------------

def sfmm_create(device: int = 0, precision: int = SFMM_FP64, stream: int | None = None):
    ctx = ctypes.c_void_p()
    _check(load().sfmm_create(ctypes.byref(ctx), int(device), int(precision),
                              ctypes.c_void_p(stream) if stream else None))
    return ctx


def sfmm_destroy(ctx):
    load().sfmm_destroy(ctx)


def sfmm_set_stream(ctx, stream):
    _check(load().sfmm_set_stream(ctx, ctypes.c_void_p(stream) if stream else None), ctx)


def sfmm_set_option(ctx, key: str, value: float):
    _check(load().sfmm_set_option(ctx, key.encode(), float(value)), ctx)


def sfmm_build(ctx, n, pos, mass, h, leaf_size):
    _check(load().sfmm_build(ctx, int(n), _ptr(pos), _ptr(mass), _ptr(h), int(leaf_size)), ctx)


def sfmm_gravity(ctx, theta, order, acc, pot):
    _check(load().sfmm_gravity(ctx, float(theta), int(order), _ptr(acc), _ptr(pot)), ctx)


def sfmm_solve_host(ctx, n, pos, mass, h, leaf_size, theta, order, acc, pot):
    _check(load().sfmm_solve_host(ctx, int(n), _ptr(pos), _ptr(mass), _ptr(h), int(leaf_size), float(theta),
                                  int(order), _ptr(acc), _ptr(pot)), ctx)


def sfmm_get_stats(ctx) -> dict:
    s = sfmm_stats()
    _check(load().sfmm_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


def sfmm_tree_size(ctx):
    nn, nl = ctypes.c_int64(), ctypes.c_int64()
    _check(load().sfmm_tree_size(ctx, ctypes.byref(nn), ctypes.byref(nl)), ctx)
    return nn.value, nl.value


def sfmm_tree_export(ctx, n=None):
    """The built tree as numpy arrays (sized from the context's own counts;
    n, if given, must equal the built particle count)."""
    nn, nl = sfmm_tree_size(ctx)
    nb = int(sfmm_get_stats(ctx)["n"])
    if n is not None and int(n) != nb:
        raise ValueError("n = %d differs from the built particle count %d" % (int(n), nb))
    n = nb
    t = dict(perm=np.empty(n, np.int64), keys=np.empty(n, np.uint64), first=np.empty(nn, np.int32),
             count=np.empty(nn, np.int32), right=np.empty(nn, np.int32), parent=np.empty(nn, np.int32),
             depth=np.empty(nn, np.int32), centre=np.empty((nn, 3)), size=np.empty(nn), hmax=np.empty(nn),
             mass=np.empty(nn), leaves=np.empty(nl, np.int32))
    _check(load().sfmm_tree_export(ctx, *[_ptr(t[k]) for k in ("perm", "keys", "first", "count", "right", "parent",
                                                                "depth", "centre", "size", "hmax", "mass",
                                                                "leaves")]), ctx)
    return t


def sfmm_moments_export(ctx, order):
    nn, _ = sfmm_tree_size(ctx)
    nq = (order + 1) * (order + 2) * (order + 3) // 6
    Q = np.empty((nn, nq))
    mi = np.empty((nq, 3), np.int32)
    _check(load().sfmm_moments_export(ctx, int(order), _ptr(Q), _ptr(mi)), ctx)
    return Q, mi


def sfmm_lists(ctx, theta):
    _, nl = sfmm_tree_size(ctx)
    mo = np.zeros(nl + 1, np.int64)
    po = np.zeros(nl + 1, np.int64)
    _check(load().sfmm_lists(ctx, float(theta), _ptr(mo), None, None, 0, _ptr(po), None, 0), ctx)
    lv = np.empty(max(1, mo[-1]), np.int32)
    src = np.empty(max(1, mo[-1]), np.int32)
    ps = np.empty(max(1, po[-1]), np.int32)
    _check(load().sfmm_lists(ctx, float(theta), _ptr(mo), _ptr(lv), _ptr(src), int(mo[-1]), _ptr(po), _ptr(ps),
                             int(po[-1])), ctx)
    return mo, lv[:mo[-1]], src[:mo[-1]], po, ps[:po[-1]]


def sfmm_build_batch(ctx, offsets, pos, mass, h, leaf_size=None):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ls = None if leaf_size is None else np.ascontiguousarray(leaf_size, dtype=np.int32)
    _check(load().sfmm_build_batch(ctx, len(off) - 1, _ptr(off), _ptr(pos), _ptr(mass), _ptr(h), _ptr(ls)), ctx)


def sfmm_autotune_batch(ctx, offsets, pos, mass, h, theta, order):
    """Autotune and build a batch; returns the chosen leaf sizes."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    out = np.empty(len(off) - 1, np.int32)
    _check(load().sfmm_autotune_batch(ctx, len(off) - 1, _ptr(off), _ptr(pos), _ptr(mass), _ptr(h), float(theta),
                                      int(order), _ptr(out)), ctx)
    return out


def sfmm_autotune_cache(ctx, path):
    _check(load().sfmm_autotune_cache(ctx, path.encode() if path else None), ctx)


def sfmm_solve_graph(ctx, offsets, pos, mass, h, leaf_size, theta, order, acc, pot):
    """Build + gravity as one captured CUDA graph per shape class (see
    include/sfmm.h); offsets (nsys + 1) host, leaf sizes per system or None."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ls = None if leaf_size is None else np.ascontiguousarray(leaf_size, dtype=np.int32)
    _check(load().sfmm_solve_graph(ctx, len(off) - 1, _ptr(off), _ptr(pos), _ptr(mass), _ptr(h), _ptr(ls),
                                   float(theta), int(order), _ptr(acc), _ptr(pot)), ctx)


def sfmm_gravity_batch(ctx, theta, order, acc, pot):
    _check(load().sfmm_gravity_batch(ctx, float(theta), int(order), _ptr(acc), _ptr(pot)), ctx)


def sfmm_batch_sums(ctx, nsys):
    out = np.empty((nsys, 5))
    _check(load().sfmm_batch_sums(ctx, int(nsys), _ptr(out)), ctx)
    return out


def sfmm_leapfrog(ctx, n, pos, vel, mass, h, leaf_size, theta, order, dt, nsteps, record_every=1, acc=None):
    """Leapfrog in place on device arrays; returns the momentum records
    (rows: t, P (3), L (3), sum |m v_d|)."""
    nrec = int(nsteps) // int(record_every) + 1 if int(record_every) >= 1 and int(nsteps) >= 0 else 1
    rec = np.empty((nrec, 8))
    _check(load().sfmm_leapfrog(ctx, int(n), _ptr(pos), _ptr(vel), _ptr(mass), _ptr(h), int(leaf_size),
                                float(theta), int(order), float(dt), int(nsteps), int(record_every), _ptr(rec),
                                _ptr(acc)), ctx)
    return rec


def sfmm_reduce_noalloc(n, mass, acc, pot, out, stream=None):
    """Momentum/energy sums over device arrays without any device allocation
    (see include/sfmm.h); ``out`` is a device buffer of 5 float64."""
    _check(load().sfmm_reduce_noalloc(int(n), _ptr(mass), _ptr(acc), _ptr(pot), _ptr(out),
                                      ctypes.c_void_p(stream) if stream else None))


def sfmm_fma_peak(device=0, form=1, stream=None, target_ms=20.0, reps=5):
    """Measured FMA throughput (TFLOP/s, ms of the best launch); form 0 FP64,
    1 FP32, 2 packed FP32."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().sfmm_fma_peak(int(device), int(form), ctypes.c_void_p(stream) if stream else None,
                                float(target_ms), int(reps), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def sfmm_strerror(code: int) -> str:
    return load().sfmm_strerror(int(code)).decode()


def sfmm_version() -> str:
    return load().sfmm_version().decode()


# --- convenience wrapper over torch tensors ---------------------------------

class Solver:
    """One context: ``build`` then ``gravity`` on torch CUDA float64 tensors.

    precision: "fp64" or "fp32" (the FP32 form).  Work is issued on the
    current torch stream of the device at creation time (or ``stream``).
    """

    def __init__(self, device: int = 0, precision: str = "fp32", stream=None, **options):
        import torch

        self.torch = torch
        self.device = int(device)
        prec = {"fp64": SFMM_FP64, "fp32": SFMM_FP32}[precision]
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.ctx = sfmm_create(self.device, prec, stream.cuda_stream)
        self.n = 0
        for k, v in options.items():
            sfmm_set_option(self.ctx, k, v)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            sfmm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        sfmm_set_option(self.ctx, key, value)

    def _dev(self, a, shape):
        t = self.torch
        if not isinstance(a, t.Tensor):
            a = t.as_tensor(np.asarray(a, dtype=np.float64))
        a = a.to(device="cuda:%d" % self.device, dtype=t.float64).contiguous()
        if tuple(a.shape) != shape:
            a = a.reshape(shape)
        return a

    def build(self, pos, mass, h, leaf_size: int = 16):
        n = int(mass.shape[0])
        self._inputs = (self._dev(pos, (n, 3)), self._dev(mass, (n,)), self._dev(h, (n,)))
        sfmm_build(self.ctx, n, *self._inputs, leaf_size)
        self.n = n

    def gravity(self, theta: float = 0.5, order: int = 2, acc=None, pot=None, want_pot: bool = True):
        t = self.torch
        if acc is None:
            acc = t.empty((self.n, 3), dtype=t.float64, device="cuda:%d" % self.device)
        if pot is None and want_pot:
            pot = t.empty((self.n,), dtype=t.float64, device="cuda:%d" % self.device)
        sfmm_gravity(self.ctx, theta, order, acc, pot)
        return acc, pot

    def build_batch(self, offsets, pos, mass, h, leaf_size=None):
        """Packed systems: offsets (nsys + 1), per-system leaf sizes or None."""
        n = int(offsets[-1])
        self._inputs = (self._dev(pos, (n, 3)), self._dev(mass, (n,)), self._dev(h, (n,)))
        sfmm_build_batch(self.ctx, offsets, *self._inputs, leaf_size)
        self.n = n
        self.nsys = len(offsets) - 1

    def autotune_batch(self, offsets, pos, mass, h, theta=0.5, order=2):
        """Autotune leaf sizes and launch knobs on these systems and build the
        batch; returns the chosen leaf sizes."""
        n = int(offsets[-1])
        self._inputs = (self._dev(pos, (n, 3)), self._dev(mass, (n,)), self._dev(h, (n,)))
        ls = sfmm_autotune_batch(self.ctx, offsets, *self._inputs, theta, order)
        self.n = n
        self.nsys = len(offsets) - 1
        return ls

    def batch_sums(self):
        return sfmm_batch_sums(self.ctx, self.nsys)

    def leapfrog(self, pos, vel, mass, h, leaf_size, theta, order, dt, nsteps, record_every=1):
        """Kick-drift-kick steps on host or device arrays.  Returns (pos, vel,
        records) as device tensors and a numpy array of records."""
        n = int(mass.shape[0])
        pos, vel = self._dev(pos, (n, 3)).clone(), self._dev(vel, (n, 3)).clone()
        mass, h = self._dev(mass, (n,)), self._dev(h, (n,))
        rec = sfmm_leapfrog(self.ctx, int(mass.shape[0]), pos, vel, mass, h, leaf_size, theta, order, dt, nsteps,
                            record_every)
        self.n = int(mass.shape[0])
        return pos, vel, rec

    def solve_host(self, pos, mass, h, leaf_size, theta, order, acc, pot):
        """Host (numpy or pinned torch CPU) buffers in and out."""
        sfmm_solve_host(self.ctx, int(mass.shape[0]), pos, mass, h, leaf_size, theta, order, acc, pot)
        self.n = int(mass.shape[0])

    def stats(self) -> dict:
        return sfmm_get_stats(self.ctx)

    def tree(self):
        return sfmm_tree_export(self.ctx, self.n)

    def moments(self, order):
        return sfmm_moments_export(self.ctx, order)

    def lists(self, theta):
        return sfmm_lists(self.ctx, theta)
