"""Thin ctypes binding of the C-ABI in include/hybrid.h (libhybrid.so).

Argument marshalling only: every step of the force path runs in the CUDA
library. Torch tensors provide device memory and streams. Importing this
module loads the library and raises if it is missing -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhybrid.so")

OK, EINVAL, ENOMEM, ECUDA, ECAPACITY, ETIMEOUT, ETOOLARGE = range(7)
STATUS_NAMES = {0: "HYBRID_OK", 1: "HYBRID_EINVAL", 2: "HYBRID_ENOMEM", 3: "HYBRID_ECUDA",
                4: "HYBRID_ECAPACITY", 5: "HYBRID_ETIMEOUT", 6: "HYBRID_ETOOLARGE"}
# largest n hybrid_energy_noalloc accepts (its fixed scratch size)
ENERGY_NOALLOC_MAX_N = 4194304

# every entry point declared in include/hybrid.h
EXPORTS = (
    "hybrid_create", "hybrid_destroy", "hybrid_build_tree", "hybrid_soft_force", "hybrid_hard_force",
    "hybrid_kick", "hybrid_drift", "hybrid_step", "hybrid_step_batched", "hybrid_get_perm", "hybrid_sync",
    "hybrid_last_error", "hybrid_tree_info", "hybrid_tree_copy", "hybrid_lists_copy", "hybrid_interactions",
    "hybrid_profile", "hybrid_profile_read", "hybrid_launch_count", "hybrid_sort_fallbacks", "hybrid_energy",
    "hybrid_energy_noalloc",
    "hybrid_autotune", "hybrid_selftest_wait", "hybrid_server_create", "hybrid_server_destroy", "hybrid_server_submit",
    "hybrid_server_step", "hybrid_server_next", "hybrid_server_used_bytes", "hybrid_server_last_error",
)
SERVER_BYTES_PER_PARTICLE = 1536


class hybrid_params(C.Structure):
    _fields_ = [
        ("G", C.c_double), ("eps", C.c_double), ("theta", C.c_double), ("R1", C.c_double), ("R2", C.c_double),
        ("dt_soft", C.c_double), ("a_err", C.c_double),
        ("n_hard", C.c_int32), ("n_leaf", C.c_int32), ("n_crit", C.c_int32),
        ("precision", C.c_int32), ("mac", C.c_int32), ("threads_per_group", C.c_int32), ("tile_depth", C.c_int32),
        ("skin", C.c_double),
    ]


class hybrid_system(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
        ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p), ("m", C.c_void_p),
        ("id", C.c_void_p),
        ("ax_s", C.c_void_p), ("ay_s", C.c_void_p), ("az_s", C.c_void_p),
        ("ax_h", C.c_void_p), ("ay_h", C.c_void_p), ("az_h", C.c_void_p),
        ("params", C.POINTER(hybrid_params)),
        ("forces_valid", C.c_int32),
    ]


class HybridError(RuntimeError):
    def __init__(self, func, code, msg):
        super().__init__("%s -> %s: %s" % (func, STATUS_NAMES.get(code, code), msg))
        self.code = code


_lib = None


def load() -> C.CDLL:
    """Loads libhybrid.so (built by paper_1406_6158_gb300.build). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libhybrid.so is not built (run paper_1406_6158_gb300.build.build())")
    L = C.CDLL(LIB_PATH)
    P, VP, I32, I64, D = C.POINTER, C.c_void_p, C.c_int32, C.c_int64, C.c_double
    ctx = VP
    sysp = P(hybrid_system)
    sig = {
        "hybrid_create": [P(VP), P(hybrid_params), VP],
        "hybrid_destroy": [ctx],
        "hybrid_build_tree": [ctx, sysp],
        "hybrid_soft_force": [ctx, sysp],
        "hybrid_hard_force": [ctx, sysp],
        "hybrid_kick": [ctx, sysp, C.c_int, D],
        "hybrid_drift": [ctx, sysp, D],
        "hybrid_step": [ctx, sysp, C.c_int],
        "hybrid_step_batched": [ctx, sysp, C.c_int, C.c_int],
        "hybrid_get_perm": [ctx, VP],
        "hybrid_sync": [ctx],
        "hybrid_tree_info": [ctx, P(I64), P(I64)],
        "hybrid_tree_copy": [ctx, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "hybrid_lists_copy": [ctx, VP, VP, I64],
        "hybrid_interactions": [ctx, P(I64), P(I64)],
        "hybrid_profile": [ctx, C.c_int],
        "hybrid_profile_read": [ctx, C.c_int, P(D), P(I64), C.c_int],
        "hybrid_energy": [ctx, sysp, P(D), P(D)],
        "hybrid_energy_noalloc": [I64, VP, VP, VP, VP, VP, VP, VP, D, D, VP, P(D), P(D)],
        "hybrid_autotune": [ctx, sysp, C.c_int, VP, C.c_int, VP, P(I32)],
        "hybrid_selftest_wait": [ctx, I32],
        "hybrid_server_create": [P(VP), P(hybrid_params), D, VP],
        "hybrid_server_destroy": [VP],
        "hybrid_server_submit": [VP, I64, I64, VP, VP, VP, VP, VP, VP, VP, P(hybrid_params), I32],
        "hybrid_server_step": [VP, P(I32), P(I32), P(I32)],
        "hybrid_server_next": [VP, P(I64), P(I64), VP, VP, VP, VP, VP, VP, VP],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.hybrid_last_error.argtypes = [ctx]
    L.hybrid_last_error.restype = C.c_char_p
    L.hybrid_launch_count.argtypes = [ctx]
    L.hybrid_launch_count.restype = C.c_int64
    L.hybrid_sort_fallbacks.argtypes = [ctx]
    L.hybrid_sort_fallbacks.restype = C.c_int64
    L.hybrid_server_used_bytes.argtypes = [VP]
    L.hybrid_server_used_bytes.restype = C.c_double
    L.hybrid_server_last_error.argtypes = [VP]
    L.hybrid_server_last_error.restype = C.c_char_p
    _lib = L
    return L


@dataclasses.dataclass
class Params:
    """hybrid_params with the defaults used across the tests and benchmark."""

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
    precision: int = 1
    mac: int = 0
    threads_per_group: int = 0
    tile_depth: int = 0
    skin: float = 0.0

    def c(self) -> hybrid_params:
        return hybrid_params(self.G, self.eps, self.theta, self.R1, self.R2, self.dt_soft, self.a_err, self.n_hard,
                             self.n_leaf, self.n_crit, self.precision, self.mac, self.threads_per_group,
                             self.tile_depth, self.skin)


def _ptr(t):
    return None if t is None else t.data_ptr()


class System:
    """One system's device state as torch tensors (FP64 state; accelerations
    float32 for precision 1, float64 for precision 0)."""

    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m")

    def __init__(self, state: dict, precision: int = 1, device="cuda", ids=True, params: Params | None = None):
        import torch
        self.n = int(len(state["x"]))
        self.t = {k: torch.as_tensor(np.ascontiguousarray(state[k], dtype=np.float64), device=device).contiguous()
                  for k in self.FIELDS}
        adt = torch.float32 if precision == 1 else torch.float64
        for k in ("ax_s", "ay_s", "az_s", "ax_h", "ay_h", "az_h"):
            self.t[k] = torch.zeros(self.n, dtype=adt, device=device)
        self.t["id"] = torch.arange(self.n, dtype=torch.int32, device=device) if ids else None
        self.params = params
        self._cparams = params.c() if params is not None else None
        self.c = hybrid_system()
        self.c.forces_valid = 0
        self.refresh()

    def refresh(self):
        t = self.t
        s = self.c
        s.n = self.n
        for k in self.FIELDS + ("ax_s", "ay_s", "az_s", "ax_h", "ay_h", "az_h"):
            setattr(s, k, _ptr(t[k]))
        s.id = _ptr(t["id"])
        s.params = C.pointer(self._cparams) if self._cparams is not None else None

    def numpy(self) -> dict:
        out = {k: v.detach().cpu().numpy() for k, v in self.t.items() if v is not None}
        return out

    def acc(self, which: str):
        import torch
        return torch.stack([self.t["a%s_%s" % (d, which)] for d in "xyz"], dim=1)


def hybrid_energy_noalloc(x, y, z, vx, vy, vz, m, G: float, eps: float, stream=None):
    """Kinetic and potential energy of one system through the allocation-free
    entry point. Arrays are contiguous FP64 tensors of one length on the
    current CUDA device (anything else raises ValueError before the C call:
    the kernels read n doubles through each pointer); `stream` is a
    torch.cuda.Stream or None (torch's current stream). Raises HybridError on
    a non-OK status (ETOOLARGE above ENERGY_NOALLOC_MAX_N)."""
    import torch
    n = int(x.numel())
    arrays = (x, y, z, vx, vy, vz, m)
    if any(t.numel() != n or not t.is_contiguous() for t in arrays):
        raise ValueError("arrays must be contiguous and of one length")
    for t in arrays:
        if t.dtype != torch.float64:
            raise ValueError("arrays must be float64, got %s" % t.dtype)
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError("arrays must be on the current CUDA device, got %s" % t.device)
    L = load()
    T, W = C.c_double(), C.c_double()
    st = (torch.cuda.current_stream() if stream is None else stream).cuda_stream
    code = L.hybrid_energy_noalloc(n, *[_ptr(t) for t in (x, y, z, vx, vy, vz, m)], float(G), float(eps), st,
                                   C.byref(T), C.byref(W))
    if code != OK:
        msg = ("n = %d exceeds the fixed scratch limit %d" % (n, ENERGY_NOALLOC_MAX_N)) if code == ETOOLARGE else ""
        raise HybridError("hybrid_energy_noalloc", code, msg)
    return T.value, W.value


class Context:
    """Owns a hybrid_ctx bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, params: Params, stream=None):
        import torch
        self.L = load()
        self.params = params
        self._cp = params.c()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        self._check("hybrid_create", self.L.hybrid_create(C.byref(h), C.byref(self._cp), C.c_void_p(stream.cuda_stream)))
        self.h = h

    def _check(self, func, code):
        if code != OK:
            msg = ""
            if getattr(self, "h", None):
                msg = (self.L.hybrid_last_error(self.h) or b"").decode()
            raise HybridError(func, code, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.hybrid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the C-ABI, by name ----
    def hybrid_build_tree(self, s: System):
        self._check("hybrid_build_tree", self.L.hybrid_build_tree(self.h, C.byref(s.c)))

    def hybrid_soft_force(self, s: System):
        self._check("hybrid_soft_force", self.L.hybrid_soft_force(self.h, C.byref(s.c)))

    def hybrid_hard_force(self, s: System):
        self._check("hybrid_hard_force", self.L.hybrid_hard_force(self.h, C.byref(s.c)))

    def hybrid_kick(self, s: System, which: int, dt: float):
        self._check("hybrid_kick", self.L.hybrid_kick(self.h, C.byref(s.c), int(which), float(dt)))

    def hybrid_drift(self, s: System, dt: float):
        self._check("hybrid_drift", self.L.hybrid_drift(self.h, C.byref(s.c), float(dt)))

    def hybrid_step(self, s: System, n_soft_steps: int):
        self._check("hybrid_step", self.L.hybrid_step(self.h, C.byref(s.c), int(n_soft_steps)))

    def hybrid_step_batched(self, systems, n_soft_steps: int):
        arr = (hybrid_system * len(systems))(*[s.c for s in systems])
        code = self.L.hybrid_step_batched(self.h, arr, len(systems), int(n_soft_steps))
        for k, s in enumerate(systems):
            s.c.forces_valid = arr[k].forces_valid
        self._check("hybrid_step_batched", code)

    def hybrid_get_perm(self, n: int):
        import torch
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        self._check("hybrid_get_perm", self.L.hybrid_get_perm(self.h, C.c_void_p(out.data_ptr())))
        return out

    def hybrid_sync(self):
        self._check("hybrid_sync", self.L.hybrid_sync(self.h))

    def hybrid_interactions(self):
        s, h = C.c_int64(), C.c_int64()
        self._check("hybrid_interactions", self.L.hybrid_interactions(self.h, C.byref(s), C.byref(h)))
        return s.value, h.value

    def hybrid_profile(self, enable):
        """True (or 2): every stage; 1: the pair kernels only; False (or 0): off."""
        level = 2 if enable is True else (0 if enable is False else int(enable))
        self._check("hybrid_profile", self.L.hybrid_profile(self.h, level))

    def hybrid_profile_read(self, kind: int, reset: bool = False):
        ms, n = C.c_double(), C.c_int64()
        self._check("hybrid_profile_read", self.L.hybrid_profile_read(self.h, kind, C.byref(ms), C.byref(n),
                                                                      int(bool(reset))))
        return ms.value, n.value

    def hybrid_selftest_wait(self, max_polls: int) -> int:
        """Runs the bounded device wait on a flag nothing sets; returns the status code (ETIMEOUT expected)."""
        return int(self.L.hybrid_selftest_wait(self.h, int(max_polls)))

    def hybrid_launch_count(self) -> int:
        return int(self.L.hybrid_launch_count(self.h))

    def hybrid_sort_fallbacks(self) -> int:
        """Tree builds repeated with the radix sort after a sample-sort bucket overflowed."""
        return int(self.L.hybrid_sort_fallbacks(self.h))

    def hybrid_autotune(self, systems, candidates=None):
        """Runs the autotuner over `systems` (a System or a list); candidates is a
        list of (n_crit, threads_per_group, tile_depth) or None for the built-in
        list. Returns (chosen triple, estimated ms per soft step of every
        candidate) and records the choice in self.params."""
        systems = [systems] if isinstance(systems, System) else list(systems)
        arr = (hybrid_system * len(systems))(*[s.c for s in systems])
        if candidates is None:
            cand, nc, nout = None, 0, 18
        else:
            flat = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32).reshape(-1, 3))
            cand, nc, nout = flat, len(flat), len(flat)
        ms = np.zeros(nout)
        best = C.c_int32(-1)
        self._check("hybrid_autotune", self.L.hybrid_autotune(
            self.h, arr, len(systems), None if cand is None else cand.ctypes.data, nc, ms.ctypes.data, C.byref(best)))
        defaults = [(16, 4, 0), (16, 8, 0), (32, 8, 0), (32, 16, 0), (64, 16, 0), (64, 32, 0), (128, 32, 0),
                    (128, 64, 0), (32, 8, 2), (32, 8, 4), (64, 16, 2), (64, 16, 4), (128, 32, 2), (128, 32, 4),
                    (256, 64, 0), (256, 64, 2), (128, 16, 0), (256, 32, 0)]
        table = defaults if cand is None else [tuple(int(v) for v in row) for row in cand]
        chosen = table[best.value]
        self.params = dataclasses.replace(self.params, n_crit=chosen[0], threads_per_group=chosen[1],
                                          tile_depth=chosen[2])
        return chosen, ms

    def hybrid_energy(self, s: System):
        T, W = C.c_double(), C.c_double()
        self._check("hybrid_energy", self.L.hybrid_energy(self.h, C.byref(s.c), C.byref(T), C.byref(W)))
        return T.value, W.value

    # ---- inspection ----
    def tree_info(self):
        """(nodes, groups) of the last tree build."""
        nn, ng = C.c_int64(), C.c_int64()
        self._check("hybrid_tree_info", self.L.hybrid_tree_info(self.h, C.byref(nn), C.byref(ng)))
        return nn.value, ng.value

    def tree(self, n: int) -> dict:
        nn, ng = C.c_int64(), C.c_int64()
        self._check("hybrid_tree_info", self.L.hybrid_tree_info(self.h, C.byref(nn), C.byref(ng)))
        nn, ng = nn.value, ng.value
        out = {
            "key": np.zeros(n, dtype=np.uint64), "level": np.zeros(nn, dtype=np.int32),
            "first": np.zeros(nn, dtype=np.int64), "count": np.zeros(nn, dtype=np.int64),
            "child": np.zeros(nn, dtype=np.int64), "nchild": np.zeros(nn, dtype=np.int32),
            "parent": np.zeros(nn, dtype=np.int64), "moments": np.zeros((max(nn, 1), 13)),
            "gnode": np.zeros(ng, dtype=np.int64), "glo": np.zeros((max(ng, 1), 3)), "ghi": np.zeros((max(ng, 1), 3)),
        }
        a = [out[k].ctypes.data for k in ("key", "level", "first", "count", "child", "nchild", "parent", "moments",
                                          "gnode", "glo", "ghi")]
        self._check("hybrid_tree_copy", self.L.hybrid_tree_copy(self.h, *a))
        out["moments"] = out["moments"][:nn]
        out["glo"], out["ghi"] = out["glo"][:ng], out["ghi"][:ng]
        return out

    def lists(self, ng: int, groups=None):
        """Per-group lists (cells, particles, hard particles) of the last walk; with `groups`, a dict of the
        selected groups' lists only (the copy from the device is whole either way)."""
        counts = np.zeros(3 * ng, dtype=np.int64)
        self._check("hybrid_lists_copy", self.L.hybrid_lists_copy(self.h, counts.ctypes.data, None, 0))
        tot = int(counts.sum())
        ent = np.zeros(max(tot, 1), dtype=np.int64)
        self._check("hybrid_lists_copy", self.L.hybrid_lists_copy(self.h, counts.ctypes.data, ent.ctypes.data, tot))
        c3 = counts.reshape(-1, 3)
        start = np.zeros(ng + 1, dtype=np.int64)
        np.cumsum(c3.sum(axis=1), out=start[1:])

        def one(g):
            o, (a, b, c) = start[g], c3[g]
            return ent[o:o + a].copy(), ent[o + a:o + a + b].copy(), ent[o + a + b:o + a + b + c].copy()
        if groups is not None:
            return {int(g): one(int(g)) for g in groups}
        return [one(g) for g in range(ng)]


class Server:
    """Continuous-batching server over the C-ABI (hybrid_server_*): requests are
    host state dicts (FP64 x..m), each with its own Params and step count."""

    FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m")

    def __init__(self, params: Params, budget_bytes: float, stream=None):
        import torch
        self.L = load()
        self._cp = params.c()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        code = self.L.hybrid_server_create(C.byref(h), C.byref(self._cp), float(budget_bytes),
                                           C.c_void_p(stream.cuda_stream))
        if code != OK:
            raise HybridError("hybrid_server_create", code, "")
        self.h = h
        self._keep = {}

    def _check(self, func, code):
        if code != OK:
            raise HybridError(func, code, self.L.hybrid_server_last_error(self.h).decode(errors="replace"))

    def submit(self, tag: int, state: dict, params: Params | None, n_steps: int):
        arrs = [np.ascontiguousarray(state[k], dtype=np.float64) for k in self.FIELDS]
        cp = params.c() if params is not None else None
        self._check("hybrid_server_submit", self.L.hybrid_server_submit(
            self.h, int(tag), len(arrs[0]), *[a.ctypes.data for a in arrs],
            C.byref(cp) if cp is not None else None, int(n_steps)))

    def step(self):
        a, q, f = C.c_int32(), C.c_int32(), C.c_int32()
        self._check("hybrid_server_step", self.L.hybrid_server_step(self.h, C.byref(a), C.byref(q), C.byref(f)))
        return a.value, q.value, f.value

    def next(self):
        """(tag, state dict in input order) of the oldest finished request, or None."""
        tag, n = C.c_int64(), C.c_int64()
        self._check("hybrid_server_next", self.L.hybrid_server_next(self.h, C.byref(tag), C.byref(n),
                                                                     *([None] * 7)))
        if tag.value < 0:
            return None
        out = {k: np.empty(n.value) for k in self.FIELDS}
        self._check("hybrid_server_next", self.L.hybrid_server_next(
            self.h, C.byref(tag), C.byref(n), *[out[k].ctypes.data for k in self.FIELDS]))
        return tag.value, out

    def used_bytes(self) -> float:
        return float(self.L.hybrid_server_used_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.L.hybrid_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
