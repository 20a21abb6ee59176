"""Plain FP64 CPU oracle of the hybrid tree force path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. The CUDA library shares no code with it.

The arithmetic lives in ``hybrid_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only marshals numpy arrays through ctypes.
Function names follow the paper (Watanabe & Nakasato): Eq. (2) softened force,
Eq. (3)-(4) leap-frog, Eq. (5)-(6) absolute MAC, Eq. (7)-(10) hard/soft split,
Eq. (11) group distance, Eq. (15) neighbour criterion, Sec. III-A1 tree build.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hybrid_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle library in place (gcc). Returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _declare(_lib)
    return _lib


@dataclasses.dataclass
class Params:
    """Method parameters (Sec. II, Sec. IV-A). mac: 0 opening angle, 1 absolute MAC."""

    G: float = 1.0
    eps: float = 1.0 / 64
    theta: float = 0.5
    R1: float = 0.0
    R2: float = 0.0
    dt_soft: float = 1.0 / 128
    a_err: float = 2.0 ** -8
    n_hard: int = 4
    n_leaf: int = 16
    n_crit: int = 64
    mac: int = 0


class _CParams(C.Structure):
    _fields_ = [
        ("G", C.c_double), ("eps", C.c_double), ("theta", C.c_double), ("R1", C.c_double),
        ("R2", C.c_double), ("dt_soft", C.c_double), ("a_err", C.c_double),
        ("n_hard", C.c_int32), ("n_leaf", C.c_int32), ("n_crit", C.c_int32), ("mac", C.c_int32),
    ]


def _cp(p: Params) -> _CParams:
    return _CParams(p.G, p.eps, p.theta, p.R1, p.R2, p.dt_soft, p.a_err, p.n_hard, p.n_leaf, p.n_crit, p.mac)


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_VP = C.c_void_p


def _declare(L: C.CDLL) -> None:
    L.orc_cutoff_K.restype = C.c_double
    L.orc_cutoff_K.argtypes = [C.c_double, C.c_double, C.c_double]
    L.orc_direct.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double, C.c_double, C.c_double, C.c_double,
                             C.c_int32, C.c_int64, _I64, _D, _D, _D, _D]
    L.orc_energy.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, _D, C.c_double, C.c_double,
                             C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.orc_root_box.argtypes = [C.c_int64, _D, _D, _D, _D, C.POINTER(C.c_double)]
    L.orc_morton_keys.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double, _U64]
    L.orc_sort.argtypes = [C.c_int64, _U64, _I64]
    L.orc_tree_new.restype = _VP
    L.orc_tree_new.argtypes = [C.c_int64, _D, _D, _D, _D, C.POINTER(_CParams)]
    L.orc_tree_free.argtypes = [_VP]
    for f in ("orc_tree_n", "orc_tree_nn", "orc_tree_ng"):
        getattr(L, f).restype = C.c_int64
        getattr(L, f).argtypes = [_VP]
    L.orc_tree_box.argtypes = [_VP, _D]
    L.orc_tree_particles.argtypes = [_VP, _U64, _I64, _D, _D, _D, _D]
    L.orc_tree_nodes.argtypes = [_VP, _I32, _I64, _I64, _I64, _I32, _I64]
    L.orc_tree_moments.argtypes = [_VP, _D]
    L.orc_tree_groups.argtypes = [_VP, _I64, _D, _D]
    L.orc_walk.argtypes = [_VP, C.c_int64, _I64, C.c_int32, _I64, _VP, _VP]
    L.orc_tree_forces.argtypes = [_VP, C.c_int64, _I64, C.c_int32, _VP, _VP, _VP, _VP]
    L.orc_interactions.argtypes = [_VP, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.orc_forces.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, _D, _VP, C.POINTER(_CParams), C.c_int32,
                             _VP, _VP]
    L.orc_hybrid_steps.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, _D, _VP, _D, _D, C.POINTER(_CParams),
                                   C.c_int32, C.c_int32]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a) -> int | None:
    return None if a is None else a.ctypes.data


def cutoff_K(r: float, R1: float, R2: float) -> float:
    """Eq. (10): the DLL cutoff kernel K(r)."""
    return lib().orc_cutoff_K(float(r), float(R1), float(R2))


def direct(x, y, z, m, G=1.0, eps=0.0, R1=0.0, R2=0.0, which=0, sinks=None):
    """Eq. (1)-(2) by direct summation; which 0 full, 1 hard (F K), 2 soft (F (1-K)).

    Returns (a[ns,3], scale[ns]) with scale = sum of term magnitudes."""
    x, y, z, m = map(_f64, (x, y, z, m))
    n = len(x)
    sinks = np.arange(n, dtype=np.int64) if sinks is None else np.ascontiguousarray(sinks, dtype=np.int64)
    ns = len(sinks)
    ax, ay, az, sc = (np.zeros(ns) for _ in range(4))
    lib().orc_direct(n, x, y, z, m, G, eps, R1, R2, which, ns, sinks, ax, ay, az, sc)
    return np.stack([ax, ay, az], axis=1), sc


def energy(x, y, z, vx, vy, vz, m, G=1.0, eps=0.0):
    """Kinetic and softened potential energy (direct sums)."""
    arrs = list(map(_f64, (x, y, z, vx, vy, vz, m)))
    T, W = C.c_double(), C.c_double()
    lib().orc_energy(len(arrs[0]), *arrs, G, eps, C.byref(T), C.byref(W))
    return T.value, W.value


def root_box(x, y, z):
    x, y, z = map(_f64, (x, y, z))
    lo = np.zeros(3)
    L = C.c_double()
    lib().orc_root_box(len(x), x, y, z, lo, C.byref(L))
    return lo, L.value


def morton_keys(x, y, z, lo, L):
    x, y, z = map(_f64, (x, y, z))
    key = np.zeros(len(x), dtype=np.uint64)
    lib().orc_morton_keys(len(x), x, y, z, _f64(lo), float(L), key)
    return key


def stable_sort(key):
    key = np.ascontiguousarray(key, dtype=np.uint64)
    perm = np.zeros(len(key), dtype=np.int64)
    lib().orc_sort(len(key), key, perm)
    return perm


MOMENT_FIELDS = ("M", "cx", "cy", "cz", "bmax", "B2", "delta", "side", "ox", "oy", "oz", "rb")


class Tree:
    """One system's tree (Sec. III-A1): root box, keys, stable sort, split, moments, groups."""

    def __init__(self, x, y, z, m, params: Params):
        L = lib()
        self.params = params
        x, y, z, m = map(_f64, (x, y, z, m))
        self._cp = _cp(params)
        self.h = L.orc_tree_new(len(x), x, y, z, m, C.byref(self._cp))
        self.n = L.orc_tree_n(self.h)
        self.nn = L.orc_tree_nn(self.h)
        self.ng = L.orc_tree_ng(self.h)
        box = np.zeros(4)
        L.orc_tree_box(self.h, box)
        self.lo, self.L = box[:3].copy(), float(box[3])
        n, nn, ng = self.n, self.nn, self.ng
        self.key = np.zeros(n, dtype=np.uint64)
        self.perm = np.zeros(n, dtype=np.int64)
        self.x, self.y, self.z, self.m = (np.zeros(n) for _ in range(4))
        L.orc_tree_particles(self.h, self.key, self.perm, self.x, self.y, self.z, self.m)
        self.level = np.zeros(nn, dtype=np.int32)
        self.first = np.zeros(nn, dtype=np.int64)
        self.count = np.zeros(nn, dtype=np.int64)
        self.child = np.zeros(nn, dtype=np.int64)
        self.nchild = np.zeros(nn, dtype=np.int32)
        self.parent = np.zeros(nn, dtype=np.int64)
        L.orc_tree_nodes(self.h, self.level, self.first, self.count, self.child, self.nchild, self.parent)
        mom = np.zeros((max(nn, 1), 13))
        if nn:
            L.orc_tree_moments(self.h, mom)
        self.moments = {k: mom[:nn, i].copy() for i, k in enumerate(MOMENT_FIELDS)}
        self.gnode = np.zeros(ng, dtype=np.int64)
        self.glo = np.zeros((max(ng, 1), 3))
        self.ghi = np.zeros((max(ng, 1), 3))
        if ng:
            L.orc_tree_groups(self.h, self.gnode, self.glo, self.ghi)
        self.glo, self.ghi = self.glo[:ng], self.ghi[:ng]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_tree_free(h)
            self.h = None

    def walk(self, groups=None, mode=3):
        """Per-group lists (cells, particles, hard particles), each in walk order."""
        sel = np.arange(self.ng, dtype=np.int64) if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
        counts = np.zeros(3 * len(sel), dtype=np.int64)
        lib().orc_walk(self.h, len(sel), sel, mode, counts, None, None)
        tot = counts.reshape(-1, 3).sum(axis=1)
        offs = np.zeros(len(sel) + 1, dtype=np.int64)
        np.cumsum(tot, out=offs[1:])
        out = np.zeros(max(int(offs[-1]), 1), dtype=np.int64)
        offs0 = offs[:-1].copy()
        lib().orc_walk(self.h, len(sel), sel, mode, counts, offs0.ctypes.data, out.ctypes.data)
        res = []
        c3 = counts.reshape(-1, 3)
        for k in range(len(sel)):
            o = offs[k]
            a, b, c = c3[k]
            res.append((out[o:o + a].copy(), out[o + a:o + a + b].copy(), out[o + a + b:o + a + b + c].copy()))
        return res

    def forces(self, groups=None, mode=3):
        """Same-tree soft and hard accelerations (sorted order), with term-magnitude scales.

        Only sinks of the selected groups are filled; others stay NaN."""
        sel = np.arange(self.ng, dtype=np.int64) if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
        n = self.n
        a_s = np.full((n, 3), np.nan)
        a_h = np.full((n, 3), np.nan)
        s_s = np.full(n, np.nan)
        s_h = np.full(n, np.nan)
        lib().orc_tree_forces(self.h, len(sel), sel, mode, _ptr(a_s), _ptr(a_h), _ptr(s_s), _ptr(s_h))
        return a_s, a_h, s_s, s_h

    def interactions(self, mode=3):
        s, h = C.c_int64(), C.c_int64()
        lib().orc_interactions(self.h, mode, C.byref(s), C.byref(h))
        return s.value, h.value


def forces(state: dict, params: Params, mode=3):
    """Forces at the current positions; re-sorts ``state`` (numpy FP64 arrays) in place."""
    n = len(state["x"])
    a_s = np.zeros((n, 3))
    a_h = np.zeros((n, 3))
    ids = state.get("id")
    cp = _cp(params)
    lib().orc_forces(n, *(state[k] for k in ("x", "y", "z", "vx", "vy", "vz", "m")), _ptr(ids), C.byref(cp), mode,
                     _ptr(a_s), _ptr(a_h))
    return a_s, a_h


def hybrid_steps(state: dict, params: Params, nsteps: int, a_s=None, a_h=None):
    """Advance ``state`` by nsteps soft steps (Sec. II-C). Returns (a_s, a_h) at the end.

    state holds contiguous FP64 arrays x, y, z, vx, vy, vz, m and optionally int64 id."""
    n = len(state["x"])
    valid = a_s is not None and a_h is not None
    a_s = np.zeros((n, 3)) if a_s is None else np.ascontiguousarray(a_s, dtype=np.float64).copy()
    a_h = np.zeros((n, 3)) if a_h is None else np.ascontiguousarray(a_h, dtype=np.float64).copy()
    cp = _cp(params)
    lib().orc_hybrid_steps(n, *(state[k] for k in ("x", "y", "z", "vx", "vy", "vz", "m")), _ptr(state.get("id")),
                           a_s, a_h, C.byref(cp), int(nsteps), int(valid))
    return a_s, a_h
