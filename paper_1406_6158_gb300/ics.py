"""Seeded synthetic initial conditions (inputs only; none of the force method lives here).

Both the CUDA path and the CPU oracle take their particles from these
generators, so the two see bit-identical inputs. Units: G = 1, total mass 1,
scale radius a = 1, equal particle masses 1/N, centre-of-mass frame.

* Plummer sphere (the model of the paper's Sec. IV-A), sampled with the
  Aarseth-Henon-Wielen (1974) recipe: enclosed-mass fraction X uniform in
  (0, 0.999], r = (X^{-2/3} - 1)^{-1/2}; speed q v_esc with q drawn by von
  Neumann rejection from q^2 (1 - q^2)^{7/2}, v_esc = sqrt(2) (1 + r^2)^{-1/4};
  isotropic directions.
* Hernquist (1990) sphere truncated at r_max: M(<r) = M_h r^2 / (r + a)^2 with
  M_h chosen so that M(<r_max) = 1, r = a sqrt(X) / (1 - sqrt(X)) for X uniform
  in [0, 1); speeds by rejection from v^2 f(E) with the closed-form isotropic
  distribution function of Hernquist (1990), Eq. (17).

Random numbers come from numpy's PCG64 generator seeded with ``seed``.
"""
from __future__ import annotations

import numpy as np


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sth = np.sqrt(1.0 - cth * cth)
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _finish(pos: np.ndarray, vel: np.ndarray, n: int) -> dict:
    m = np.full(n, 1.0 / n)
    pos = pos - (m[:, None] * pos).sum(axis=0) / m.sum()
    vel = vel - (m[:, None] * vel).sum(axis=0) / m.sum()
    return {
        "x": np.ascontiguousarray(pos[:, 0]), "y": np.ascontiguousarray(pos[:, 1]),
        "z": np.ascontiguousarray(pos[:, 2]), "vx": np.ascontiguousarray(vel[:, 0]),
        "vy": np.ascontiguousarray(vel[:, 1]), "vz": np.ascontiguousarray(vel[:, 2]),
        "m": m,
    }


def plummer(n: int, seed: int, a: float = 1.0) -> dict:
    """Plummer sphere of n equal-mass particles (G = M = 1, scale radius a)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.0, 1.0, n)
    X = np.minimum(1.0 - X, 0.999)          # (0, 1] capped at 0.999
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        yy = rng.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = np.sqrt(2.0) * (1.0 + (r / a) ** 2) ** -0.25 / np.sqrt(a)
    vel = (q * vesc)[:, None] * _isotropic(rng, n)
    return _finish(pos, vel, n)


def _hernquist_df(E_rel: np.ndarray, Mh: float, a: float) -> np.ndarray:
    """Isotropic Hernquist DF f(E) (up to a constant) at relative energy E_rel = Psi - v^2/2 > 0."""
    q2 = np.clip(E_rel * a / Mh, 0.0, 1.0 - 1e-12)
    q = np.sqrt(q2)
    s = np.sqrt(1.0 - q2)
    br = 3.0 * np.arcsin(q) + q * s * (1.0 - 2.0 * q2) * (8.0 * q2 * q2 - 8.0 * q2 - 3.0)
    return np.maximum(br, 0.0) / (1.0 - q2) ** 2.5


def hernquist(n: int, seed: int, a: float = 1.0, rmax: float = 100.0, chunk: int = 1 << 20) -> dict:
    """Hernquist sphere truncated at rmax, n equal-mass particles, total mass 1."""
    return _hernquist(n, seed, a, rmax, chunk)[0]


def hernquist_envelope(r: np.ndarray, a: float = 1.0, rmax: float = 100.0) -> np.ndarray:
    """The rejection envelope the sampler uses at radii r (for checks)."""
    return _hernquist(0, 0, a, rmax, 1 << 20, r)[1]


def _hernquist(n, seed, a, rmax, chunk, env_at=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    Xmax = (rmax / (rmax + a)) ** 2
    Mh = 1.0 / Xmax
    sX = np.sqrt(rng.uniform(0.0, Xmax, n))
    r = a * sX / (1.0 - sX)
    pos = r[:, None] * _isotropic(rng, n)
    speed = np.empty(n)
    # fractions of v_esc for the envelope, geometric: near the centre the peak of v^2 f sits at v << v_esc
    vgrid = np.geomspace(1e-6, 1.0, 512)

    def envelope(rr):   # max over the v grid of v^2 f(Psi - v^2 / 2) at radii rr
        psi = Mh / (rr + a)
        vesc = np.sqrt(2.0 * psi)
        g = (vgrid[None, :] * vesc[:, None]) ** 2 * _hernquist_df(
            psi[:, None] - 0.5 * (vgrid[None, :] * vesc[:, None]) ** 2, Mh, a)
        return g.max(axis=1)

    # envelope tabulated on a log grid in r (ratio 1.005 between nodes); each particle takes 1.25 x the
    # larger of its two bracketing nodes, and particles inside the first node get their own
    rg = np.geomspace(1e-6 * a, rmax * (1 + 1e-9), 4096)
    eg = envelope(rg)
    if env_at is not None:
        j = np.clip(np.searchsorted(rg, env_at) - 1, 0, rg.size - 2)
        env = 1.25 * np.maximum(eg[j], eg[j + 1])
        inner = env_at < rg[0]
        if inner.any():
            env[inner] = 1.25 * envelope(env_at[inner])
        return None, env
    for c0 in range(0, n, chunk):
        rc = r[c0:c0 + chunk]
        psi = Mh / (rc + a)
        vesc = np.sqrt(2.0 * psi)
        j = np.clip(np.searchsorted(rg, rc) - 1, 0, rg.size - 2)
        env = 1.25 * np.maximum(eg[j], eg[j + 1])
        inner = rc < rg[0]
        if inner.any():
            env[inner] = 1.25 * envelope(rc[inner])
        out = np.empty(rc.size)
        todo = np.arange(rc.size)
        while todo.size:
            v = rng.uniform(0.0, 1.0, todo.size) * vesc[todo]
            u = rng.uniform(0.0, 1.0, todo.size) * env[todo]
            ok = u < v * v * _hernquist_df(psi[todo] - 0.5 * v * v, Mh, a)
            out[todo[ok]] = v[ok]
            todo = todo[~ok]
        speed[c0:c0 + chunk] = out
    vel = speed[:, None] * _isotropic(rng, n)
    return _finish(pos, vel, n), None


def ensemble_sizes(count: int, lo_log2: float, hi_log2: float, seed: int) -> np.ndarray:
    """Particle counts log-uniform in [2^lo, 2^hi] (batched and served workloads)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.floor(2.0 ** rng.uniform(lo_log2, hi_log2, count)).astype(np.int64)
