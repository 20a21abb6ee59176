"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test pins one part of the oracle to something other than the oracle
itself: a closed form, an exact integral, a hand-derived fixture under
tests/golden/, an invariant, or brute force on a tiny input.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1406_6158_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_system(n, seed, spread=1.0, unequal=True):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=(n, 3)) * spread
    m = rng.uniform(0.5, 2.0, n) if unequal else np.full(n, 1.0 / n)
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m


# --------------------------------------------------------------------------
# Eq. (10): the DLL cutoff kernel
# --------------------------------------------------------------------------
def test_cutoff_endpoints_exact():
    R1, R2 = 0.3, 0.7
    assert oracle.cutoff_K(0.0, R1, R2) == 1.0
    assert oracle.cutoff_K(R1, R1, R2) == 1.0          # Y = 1
    assert oracle.cutoff_K(R2, R1, R2) == 0.0          # Y = 0
    assert oracle.cutoff_K(5.0, R1, R2) == 0.0
    assert oracle.cutoff_K(0.0, 0.0, 0.0) == 0.0       # no hard part


def test_cutoff_integrals_closed_form():
    # int_0^1 (10Y^6 - 15Y^8 + 6Y^10) dY = 10/7 - 15/9 + 6/11 = 71/231 and
    # int_0^1 Y (...) dY = 10/8 - 15/10 + 6/12 = 1/4. With R1 = 0, R2 = 1,
    # Y = 1 - r, so these are integrals of K over r in [0, 1].
    xs, ws = np.polynomial.legendre.leggauss(24)
    r = 0.5 * (xs + 1.0)
    K = np.array([oracle.cutoff_K(v, 0.0, 1.0) for v in r])
    Y = 1.0 - r
    assert abs(0.5 * np.sum(ws * K) - 71.0 / 231.0) < 1e-14
    assert abs(0.5 * np.sum(ws * Y * K) - 0.25) < 1e-14


def test_cutoff_c1_and_monotone():
    R1, R2 = 0.25, 0.5
    h = 1e-7
    for r0 in (R1, R2):   # dK/dY = 60 Y^5 (1 - Y^2)^2 vanishes at both ends
        d = (oracle.cutoff_K(r0 + h, R1, R2) - oracle.cutoff_K(r0 - h, R1, R2)) / (2 * h)
        assert abs(d) < 1e-5
    rs = np.linspace(0, 0.6, 601)
    Ks = np.array([oracle.cutoff_K(v, R1, R2) for v in rs])
    assert np.all(np.diff(Ks) <= 0.0)
    # the slope in the middle of the transition: dK/dr = -60 Y^5 (1-Y^2)^2 / (R2-R1) at Y = 1/2
    mid = 0.5 * (R1 + R2)
    d = (oracle.cutoff_K(mid + 1e-6, R1, R2) - oracle.cutoff_K(mid - 1e-6, R1, R2)) / 2e-6
    assert abs(d - (-60 * 0.5 ** 5 * (1 - 0.25) ** 2 / (R2 - R1))) < 1e-6


# --------------------------------------------------------------------------
# Eq. (1)-(2): softened gravity by direct summation
# --------------------------------------------------------------------------
def test_two_body_closed_form():
    # sink at the origin, source m = 2 at (3, 4, 0), G = 1.5:
    # a = G m d / (|d|^2 + eps^2)^{3/2}; eps = 0 -> |d|^3 = 125, eps = 12 -> 169^{3/2} = 2197
    x, y, z, m = np.array([0.0, 3.0]), np.array([0.0, 4.0]), np.zeros(2), np.array([7.0, 2.0])
    a, _ = oracle.direct(x, y, z, m, G=1.5, eps=0.0, sinks=[0])
    assert np.allclose(a[0], [3.0 * 3 / 125, 3.0 * 4 / 125, 0.0], rtol=1e-15, atol=0)
    a, _ = oracle.direct(x, y, z, m, G=1.5, eps=12.0, sinks=[0])
    assert np.allclose(a[0], [9.0 / 2197, 12.0 / 2197, 0.0], rtol=1e-15, atol=0)
    # the source mass, not the sink mass, sets the pull (the sink's m = 7 is irrelevant)
    a1, _ = oracle.direct(x, y, z, m, G=1.5, eps=0.0, sinks=[1])
    assert np.allclose(a1[0], [-7 * 1.5 * 3 / 125, -7 * 1.5 * 4 / 125, 0.0], rtol=1e-15)


def test_cube_corner_closed_form():
    # 8 unit masses on the corners of [-1,1]^3, eps = 0: the pull on a corner points to the
    # centre with magnitude 3/(4 sqrt3) + (3/8) sqrt(2/3) + 1/12 (edges, face and body diagonals).
    c = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    a, _ = oracle.direct(c[:, 0], c[:, 1], c[:, 2], np.ones(8), eps=0.0)
    mag = 3 / (4 * math.sqrt(3)) + 3 / 8 * math.sqrt(2 / 3) + 1 / 12
    for i in range(8):
        assert np.allclose(a[i], -c[i] / math.sqrt(3) * mag, rtol=1e-14, atol=1e-15)


def test_momentum_conservation():
    x, y, z, m = rand_system(200, 1)
    a, sc = oracle.direct(x, y, z, m, eps=0.05)
    p = (m[:, None] * a).sum(axis=0)
    assert np.all(np.abs(p) < 1e-13 * np.sum(m * sc))


def test_force_is_minus_gradient_of_potential():
    # a_i = -(1/m_i) dW/dx_i, W the softened potential energy (a separate routine).
    x, y, z, m = rand_system(16, 2)
    eps, h = 0.1, 1e-5
    zero = np.zeros(16)
    a, _ = oracle.direct(x, y, z, m, eps=eps)
    for i in (0, 7, 15):
        for d, arr in enumerate((x, y, z)):
            arr[i] += h
            _, Wp = oracle.energy(x, y, z, zero, zero, zero, m, eps=eps)
            arr[i] -= 2 * h
            _, Wm = oracle.energy(x, y, z, zero, zero, zero, m, eps=eps)
            arr[i] += h
            g = -(Wp - Wm) / (2 * h) / m[i]
            assert abs(g - a[i, d]) < 1e-7 * (1 + abs(a[i, d]))


def test_split_sums_to_full_and_limits():
    x, y, z, m = rand_system(150, 3)
    full, _ = oracle.direct(x, y, z, m, eps=0.02)
    for R1, R2 in ((0.1, 0.2), (0.0, 0.5), (0.3, 0.31)):
        hard, _ = oracle.direct(x, y, z, m, eps=0.02, R1=R1, R2=R2, which=1)
        soft, _ = oracle.direct(x, y, z, m, eps=0.02, R1=R1, R2=R2, which=2)
        assert np.allclose(hard + soft, full, rtol=1e-12, atol=1e-14)
    diam = 2 * np.max(np.abs(np.stack([x, y, z])))
    hard, _ = oracle.direct(x, y, z, m, eps=0.02, R1=2 * diam, R2=3 * diam, which=1)
    assert np.array_equal(hard, full)
    hard, _ = oracle.direct(x, y, z, m, eps=0.02, R1=0.0, R2=0.0, which=1)
    assert np.all(hard == 0.0)


# --------------------------------------------------------------------------
# Sec. III-A1: root cell, Morton keys, sort, tree
# --------------------------------------------------------------------------
def load_keys():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_keys.txt")) if l.strip() and l[0] != "#"]
    p = np.array([[float(v) for v in r[:3]] for r in rows])
    k = np.array([int(r[3]) for r in rows], dtype=np.uint64)
    return p, k


def test_morton_keys_golden():
    p, k = load_keys()
    lo, L = oracle.root_box(p[:, 0], p[:, 1], p[:, 2])
    assert np.all(lo == 0.0) and L == 1.0
    got = oracle.morton_keys(p[:, 0], p[:, 1], p[:, 2], lo, L)
    assert np.array_equal(got, k)


def test_root_box_power_of_two():
    for ext, want in ((0.7, 1.0), (1.0, 1.0), (1.5, 2.0), (3.0, 4.0), (0.25, 0.25), (0.3, 0.5)):
        x = np.array([-2.0, -2.0 + ext])
        lo, L = oracle.root_box(x, np.zeros(2), np.zeros(2))
        assert L == want and lo[0] == -2.0
    lo, L = oracle.root_box(np.ones(3), np.ones(3), np.ones(3))
    assert L == 1.0


def test_sort_is_stable_and_ordered():
    rng = np.random.default_rng(5)
    key = rng.integers(0, 40, 3000).astype(np.uint64)        # many ties
    perm = oracle.stable_sort(key)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))


def load_tree_golden():
    perm, nodes, groups = None, [], None
    for l in open(os.path.join(GOLDEN, "tree_small.txt")):
        if not l.strip() or l[0] == "#":
            continue
        w = l.split()
        if w[0] == "perm":
            perm = [int(v) for v in w[1:]]
        elif w[0] == "node":
            nodes.append([int(v) for v in w[1:]])
        elif w[0] == "groups":
            groups = [int(v) for v in w[1:]]
    return perm, np.array(nodes), groups


def test_tree_golden_topology_and_moments():
    perm, nodes, groups = load_tree_golden()
    P = np.array([[0.9, 0.9, 0.9], [0.1, 0.1, 0.1], [0.9, 0.1, 0.1], [0.2, 0.2, 0.2]])
    m = np.array([1.0, 1.0, 1.0, 3.0])
    T = oracle.Tree(P[:, 0], P[:, 1], P[:, 2], m, oracle.Params(n_leaf=1, n_crit=2))
    assert list(T.perm) == perm
    got = np.stack([np.arange(T.nn), T.level, T.first, T.count, T.child, T.nchild, T.parent], axis=1)
    assert np.array_equal(got, nodes)
    assert list(T.gnode) == groups
    mo = T.moments
    assert mo["M"][4] == 4.0
    assert np.allclose([mo["cx"][4], mo["cy"][4], mo["cz"][4]], 0.175, rtol=1e-15)
    assert abs(mo["bmax"][4] - 0.075 * math.sqrt(3)) < 1e-15
    assert abs(mo["B2"][4] - 0.0225) < 1e-15
    assert mo["side"][4] == 0.25
    assert abs(mo["delta"][4] - 0.05 * math.sqrt(3)) < 1e-15
    assert mo["M"][0] == 6.0
    # opening-angle radius r_b = l / theta + delta (theta = 0.5)
    assert abs(mo["rb"][4] - (0.25 / 0.5 + 0.05 * math.sqrt(3))) < 1e-15


def tree_invariants(T: oracle.Tree):
    n, nn = T.n, T.nn
    p = T.params
    # sorted keys non-decreasing; perm a permutation
    assert np.all(np.diff(T.key.astype(np.float64)) >= 0) or np.all(T.key[1:] >= T.key[:-1])
    assert np.array_equal(np.sort(T.perm), np.arange(n))
    for c in range(nn):
        if T.nchild[c]:
            ch = np.arange(T.child[c], T.child[c] + T.nchild[c])
            assert T.count[c] > p.n_leaf and T.level[c] < 21
            assert np.all(T.level[ch] == T.level[c] + 1) and np.all(T.parent[ch] == c)
            assert T.first[ch[0]] == T.first[c] and np.sum(T.count[ch]) == T.count[c]
            assert np.all(T.first[ch[1:]] == T.first[ch[:-1]] + T.count[ch[:-1]])
        else:
            assert T.count[c] <= p.n_leaf or T.level[c] == 21
        # every member's key shares the cell prefix
        a, b = T.first[c], T.first[c] + T.count[c]
        sh = np.uint64(3 * (21 - T.level[c]))
        assert np.all((T.key[a:b] >> sh) == (T.key[a] >> sh))
    # breadth-first order: levels non-decreasing
    assert np.all(np.diff(T.level) >= 0)
    # moments: M is the plain sum; members lie inside the cell cube and within b_max of the COM
    mo = T.moments
    for c in range(0, nn, max(1, nn // 50)):
        a, b = T.first[c], T.first[c] + T.count[c]
        assert abs(mo["M"][c] - T.m[a:b].sum()) <= 2.3e-16 * (b - a) * mo["M"][c]  # sequential-sum bound
        P = np.stack([T.x[a:b], T.y[a:b], T.z[a:b]], axis=1)
        o = np.array([mo["ox"][c], mo["oy"][c], mo["oz"][c]])
        assert np.all(P >= o - 1e-12) and np.all(P <= o + mo["side"][c] * (1 + 1e-12))
        com = np.array([mo["cx"][c], mo["cy"][c], mo["cz"][c]])
        # the oracle sums m (x - x_first): sequential-sum bound on n terms of at most m |x - x_first| each
        spread = np.abs(P - P[0]).max()
        ref = (T.m[a:b, None] * P).sum(0) / T.m[a:b].sum()
        assert np.all(np.abs(com - ref) <= 1e-12 * np.abs(ref) + 2.3e-16 * (b - a) * spread + 1e-14)
        if b - a == 1:
            assert np.array_equal(com, P[0]) and mo["B2"][c] == 0.0 and mo["bmax"][c] == 0.0
        r = np.linalg.norm(P - com, axis=1)
        assert abs(r.max() - mo["bmax"][c]) <= 1e-12 * (1 + r.max())
    # groups cover the particles once, in order, and are maximal
    g_first = T.first[T.gnode]
    g_count = T.count[T.gnode]
    assert g_first[0] == 0 and np.all(g_first[1:] == g_first[:-1] + g_count[:-1])
    assert g_first[-1] + g_count[-1] == n
    for c in T.gnode:
        assert T.count[c] <= p.n_crit or T.nchild[c] == 0
        if T.parent[c] >= 0:
            assert T.count[T.parent[c]] > p.n_crit


@pytest.mark.parametrize("n_leaf,n_crit", [(16, 64), (1, 1), (8, 16), (16, 8)])
def test_tree_invariants_plummer(n_leaf, n_crit):
    s = ics.plummer(3000, 11)
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], oracle.Params(n_leaf=n_leaf, n_crit=n_crit))
    tree_invariants(T)


def test_tree_coincident_particles():
    # 40 particles on one point and 3 elsewhere: the split stops at the deepest key level
    x = np.concatenate([np.full(40, 0.3), [0.0, 1.0, 0.5]])
    y = np.concatenate([np.full(40, 0.3), [0.0, 1.0, 0.2]])
    z = np.concatenate([np.full(40, 0.3), [0.0, 1.0, 0.9]])
    m = np.ones(43)
    T = oracle.Tree(x, y, z, m, oracle.Params(n_leaf=4, n_crit=8))
    tree_invariants(T)
    assert T.level.max() == 21
    deep = np.where(T.level == 21)[0]
    assert len(deep) == 1 and T.count[deep[0]] == 40 and T.nchild[deep[0]] == 0


# --------------------------------------------------------------------------
# Sec. II-B traversal with Eq. (11) and Eq. (15): lists and forces
# --------------------------------------------------------------------------
def test_walk_lists_partition_sources():
    # every source is counted once per group: inside exactly one taken cell or listed itself
    s = ics.plummer(2000, 4)
    eps = 1 / 64
    p = oracle.Params(eps=eps, theta=0.6, R1=4 * eps, R2=8 * eps, n_leaf=8, n_crit=32)
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], p)
    lists = T.walk()
    P = np.stack([T.x, T.y, T.z], axis=1)
    for g, (cells, parts, hparts) in enumerate(lists):
        cover = np.zeros(T.n, dtype=np.int64)
        for c in cells:
            cover[T.first[c]:T.first[c] + T.count[c]] += 1
        cover[parts] += 1
        assert np.all(cover == 1)
        # taken cells: every member at least R2 from every sink (so K = 0 for all their pairs)
        gc = T.gnode[g]
        sinks = P[T.first[gc]:T.first[gc] + T.count[gc]]
        for c in cells[:50]:
            mem = P[T.first[c]:T.first[c] + T.count[c]]
            dmin = np.min(np.linalg.norm(sinks[:, None, :] - mem[None, :, :], axis=2))
            assert dmin >= p.R2
        # hard list: exactly the particles that matter are present (brute force)
        d = np.linalg.norm(sinks[:, None, :] - P[None, :, :], axis=2).min(axis=0)
        need = set(np.where(d < p.R2)[0])
        assert need <= set(hparts)
        assert set(hparts) <= set(parts)


def test_theta_zero_lists_are_all_particles():
    s = ics.plummer(500, 6)
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], oracle.Params(theta=0.0, n_leaf=4, n_crit=16))
    for cells, parts, _ in T.walk(mode=1):
        assert len(cells) == 0 and np.array_equal(np.sort(parts), np.arange(T.n))


def load_lists_golden():
    params, parts, order, groups = {}, {}, [], {}
    for line in open(os.path.join(GOLDEN, "lists_small.txt")):
        w = line.split()
        if not w or w[0].startswith("#"):
            continue
        if w[0] == "params":
            params = {w[k]: float(w[k + 1]) for k in range(1, len(w), 2)}
        elif w[0] == "particle":
            parts[w[1]] = tuple(float(v) for v in w[2:5])
        elif w[0] == "order":
            order = w[1:]
        elif w[0] == "group":
            i_c, i_p, i_h = w.index("cells"), w.index("particles"), w.index("hard")
            cells = sorted((int(c.split(":")[0]), frozenset(c.split(":")[1].split(","))) for c in w[i_c + 1:i_p])
            groups[w[1]] = (cells, sorted(w[i_p + 1:i_h]), sorted(w[i_h + 1:]))
    return params, parts, order, groups


def test_walk_lists_golden():
    # hand-derived lists (tests/golden/lists_small.txt): one cell taken exactly at r = r_b (strict opening),
    # one opened just inside r_b, one refused by the R2 + b_max test of Eq. (15) alone
    prm, parts, order, want = load_lists_golden()
    labels = list(parts)
    P = np.array([parts[k] for k in labels])
    p = oracle.Params(theta=prm["theta"], R1=prm["R1"], R2=prm["R2"], n_leaf=int(prm["n_leaf"]),
                      n_crit=int(prm["n_crit"]))
    T = oracle.Tree(P[:, 0], P[:, 1], P[:, 2], np.ones(len(labels)), p)
    assert [labels[i] for i in T.perm] == order
    name = [labels[i] for i in T.perm]               # sorted position -> label
    gid = {name[T.first[c]]: g for g, c in enumerate(T.gnode)}
    sel = [gid[k] for k in want]
    for (gname, (cells, plist, hlist)), (gc, gp, gh) in zip(want.items(), T.walk(sel)):
        got_cells = sorted((int(T.level[c]), frozenset(name[T.first[c] + i] for i in range(T.count[c])))
                           for c in gc)
        assert got_cells == cells, gname
        assert sorted(name[i] for i in gp) == plist, gname
        assert sorted(name[i] for i in gh) == hlist, gname


def test_theta_infinite_no_hard_part_lists_are_root_only():
    # theta -> infinity: r_b -> delta. Unit masses on the eight corners of the unit cube: the root's centre of
    # mass is its geometric centre (delta = 0) and every particle is b_max = sqrt(3)/2 from it. With R2 = 0 the
    # R2 + b_max test is r >= b_max, met with equality by every one-particle group, so each group's list is the
    # root cell alone (its own particle included in the root's monopole).
    c = np.array([[i >> 2 & 1, i >> 1 & 1, i & 1] for i in range(8)], dtype=np.float64)
    for theta in (1e6, math.inf):
        T = oracle.Tree(c[:, 0], c[:, 1], c[:, 2], np.ones(8), oracle.Params(theta=theta, n_leaf=1, n_crit=1))
        assert T.ng == 8 and T.moments["delta"][0] == 0.0
        for cells, plist, hlist in T.walk():
            assert list(cells) == [0] and len(plist) == 0 and len(hlist) == 0
        soft, hard = T.interactions()
        assert (soft, hard) == (8, 0)
    # a finite theta of 1 opens the root for every corner (r_b = 1 > sqrt(3)/2)
    T = oracle.Tree(c[:, 0], c[:, 1], c[:, 2], np.ones(8), oracle.Params(theta=1.0, n_leaf=1, n_crit=1))
    assert all(0 not in set(cells) for cells, _, _ in T.walk())


def test_interaction_counts_closed_forms():
    # the counter is |group| x (list length) summed over groups, a sink's pair with itself included: at
    # theta = 0 every soft list is every particle (N^2); with R2 beyond the system's diameter every hard list is
    # too, and with R2 = 0 there is no hard list
    s = ics.plummer(700, 9)
    n = 700
    diam = 2.0 * np.sqrt(np.max(s["x"] ** 2 + s["y"] ** 2 + s["z"] ** 2)) + 1.0
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], oracle.Params(theta=0.0, R1=diam, R2=2 * diam, n_leaf=8,
                                                                     n_crit=16))
    assert T.interactions() == (n * n, n * n)
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], oracle.Params(theta=0.0, n_leaf=8, n_crit=16))
    assert T.interactions() == (n * n, 0)
    # theta > 0: the same sum from the lists themselves
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], oracle.Params(theta=0.7, R1=0.05, R2=0.1, n_leaf=8, n_crit=16))
    lists = T.walk()
    cnt = T.count[T.gnode]
    want = (int(sum(c * (len(a) + len(b)) for c, (a, b, _) in zip(cnt, lists))),
            int(sum(c * len(h) for c, (_, _, h) in zip(cnt, lists))))
    assert T.interactions() == want and want[0] < n * n


@pytest.mark.parametrize("R1,R2", [(0.0, 0.0), (0.05, 0.1), (0.2, 0.4), (0.0, 0.3)])
def test_tree_theta_zero_equals_direct(R1, R2):
    # with theta = 0 every cell opens: soft + hard is the direct sum for any R1 < R2
    x, y, z, m = rand_system(400, 7, unequal=True)
    p = oracle.Params(eps=0.03, theta=0.0, R1=R1, R2=R2, n_leaf=4, n_crit=16)
    T = oracle.Tree(x, y, z, m, p)
    a_s, a_h, s_s, s_h = T.forces()
    full, sc = oracle.direct(T.x, T.y, T.z, T.m, eps=0.03)
    assert np.all(np.abs(a_s + a_h - full) <= 1e-13 * sc[:, None])
    hard, _ = oracle.direct(T.x, T.y, T.z, T.m, eps=0.03, R1=R1, R2=R2, which=1)
    assert np.all(np.abs(a_h - hard) <= 1e-13 * sc[:, None])


def test_tree_force_error_small_and_hard_exact():
    # theta > 0: the hard part is still exact (all neighbours within R2 are listed);
    # the soft part carries the tree error, about 1e-3 rms at theta = 0.5
    s = ics.plummer(4096, 0)
    eps = 1 / 64
    p = oracle.Params(eps=eps, theta=0.5, R1=4 * eps, R2=8 * eps)
    T = oracle.Tree(s["x"], s["y"], s["z"], s["m"], p)
    a_s, a_h, _, _ = T.forces()
    hard, sc = oracle.direct(T.x, T.y, T.z, T.m, eps=eps, R1=p.R1, R2=p.R2, which=1)
    assert np.all(np.abs(a_h - hard) <= 1e-13 * (sc[:, None] + 1e-300))
    full, _ = oracle.direct(T.x, T.y, T.z, T.m, eps=eps)
    err = np.linalg.norm(a_s + a_h - full, axis=1) / np.linalg.norm(full, axis=1)
    assert np.sqrt(np.mean(err ** 2)) < 2e-3


def test_absolute_mac_special_cases():
    # Eq. (5): a single-particle cell has b_max = B2 = 0 -> r_b = 0; for two particles
    # r_b -> b_max as a_err -> infinity.
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    m = np.array([1.0, 1.0])
    T = oracle.Tree(P[:, 0], P[:, 1], P[:, 2], m, oracle.Params(mac=1, a_err=1e300, n_leaf=1))
    assert T.moments["rb"][0] == pytest.approx(0.5, rel=1e-12)    # b_max = 0.5
    assert T.moments["rb"][1] == 0.0 and T.moments["rb"][2] == 0.0
    T2 = oracle.Tree(P[:, 0], P[:, 1], P[:, 2], m, oracle.Params(mac=1, a_err=3.0, n_leaf=1))
    # B2 = 2 * 0.25 = 0.5, sqrt(3 * 0.5 / 3) = sqrt(0.5); r_b = 0.25 + sqrt(0.0625 + sqrt(0.5))
    assert T2.moments["rb"][0] == pytest.approx(0.25 + math.sqrt(0.0625 + math.sqrt(0.5)), rel=1e-14)


# --------------------------------------------------------------------------
# Sec. II-C integration with Eq. (3)-(4)
# --------------------------------------------------------------------------
def copy_state(s):
    return {k: np.array(v, copy=True) for k, v in s.items()}


def test_reversibility():
    s = ics.plummer(64, 9)
    s["id"] = np.arange(64, dtype=np.int64)
    p = oracle.Params(eps=0.05, theta=0.5, R1=0.1, R2=0.2, dt_soft=1 / 64, n_hard=4, n_leaf=4, n_crit=8)
    st = copy_state(s)
    a_s, a_h = oracle.hybrid_steps(st, p, 16)
    for k in ("vx", "vy", "vz"):
        st[k] = -st[k]
    oracle.hybrid_steps(st, p, 16, a_s, a_h)
    o = np.argsort(st["id"])
    for k in ("x", "y", "z"):
        assert np.allclose(st[k][o], s[k], rtol=0, atol=1e-10)
    for k in ("vx", "vy", "vz"):
        assert np.allclose(-st[k][o], s[k], rtol=0, atol=1e-10)


def total_energy(st, eps):
    T, W = oracle.energy(st["x"], st["y"], st["z"], st["vx"], st["vy"], st["vz"], st["m"], eps=eps)
    return T + W


def test_energy_drift_second_order():
    s = ics.plummer(256, 10)
    drifts = []
    for dt in (1 / 32, 1 / 64):
        p = oracle.Params(eps=0.05, theta=0.0, R1=0.1, R2=0.2, dt_soft=dt, n_hard=2, n_leaf=8, n_crit=16)
        st = copy_state(s)
        E0 = total_energy(st, p.eps)
        oracle.hybrid_steps(st, p, int(round(0.5 / dt)))
        drifts.append(abs(total_energy(st, p.eps) - E0) / abs(E0))
    assert drifts[0] < 1e-3
    assert 2.5 < drifts[0] / drifts[1] < 6.0        # ~4: second order in dt


def test_n1_hybrid_is_plain_kdk():
    # n = 1, theta = 0: one hybrid step is v += dt/2 (a_s + a_h) split into two kicks,
    # drift, then the same at the end -- a plain KDK with the full force.
    s = ics.plummer(100, 12)
    s["id"] = np.arange(100, dtype=np.int64)
    eps, dt = 0.05, 1 / 32
    p = oracle.Params(eps=eps, theta=0.0, R1=0.1, R2=0.2, dt_soft=dt, n_hard=1, n_leaf=4, n_crit=8)
    st = copy_state(s)
    oracle.hybrid_steps(st, p, 5)
    o = np.argsort(st["id"])
    X = np.stack([s["x"], s["y"], s["z"]], 1)
    V = np.stack([s["vx"], s["vy"], s["vz"]], 1)
    a, _ = oracle.direct(X[:, 0], X[:, 1], X[:, 2], s["m"], eps=eps)
    for _ in range(5):
        V = V + 0.5 * dt * a
        X = X + dt * V
        a, _ = oracle.direct(X[:, 0], X[:, 1], X[:, 2], s["m"], eps=eps)
        V = V + 0.5 * dt * a
    assert np.allclose(np.stack([st["x"], st["y"], st["z"]], 1)[o], X, rtol=0, atol=1e-12)
    assert np.allclose(np.stack([st["vx"], st["vy"], st["vz"]], 1)[o], V, rtol=0, atol=1e-12)


def test_kepler_circular_orbit_period():
    # two unit masses 1 apart on a circular orbit (G = 1, eps = 0): omega^2 = G M / d^3 = 2,
    # period 2 pi / sqrt 2; after one period the bodies return to their start.
    w = math.sqrt(2.0)
    s = {"x": np.array([-0.5, 0.5]), "y": np.zeros(2), "z": np.zeros(2),
         "vx": np.zeros(2), "vy": np.array([-0.5 * w, 0.5 * w]), "vz": np.zeros(2), "m": np.ones(2),
         "id": np.arange(2, dtype=np.int64)}
    period = 2 * math.pi / w
    nsteps = 2000
    p = oracle.Params(eps=0.0, theta=0.0, R1=0.0, R2=0.0, dt_soft=period / nsteps, n_hard=1, n_leaf=1, n_crit=1)
    oracle.hybrid_steps(s, p, nsteps)
    o = np.argsort(s["id"])
    assert np.allclose(s["x"][o], [-0.5, 0.5], atol=1e-5)
    assert np.allclose(s["y"][o], [0.0, 0.0], atol=1e-4)


def test_momentum_conserved_by_integration():
    s = ics.plummer(128, 13)
    p = oracle.Params(eps=0.05, theta=0.0, R1=0.1, R2=0.2, dt_soft=1 / 64, n_hard=4, n_leaf=4, n_crit=8)
    P0 = np.array([np.sum(s["m"] * s[k]) for k in ("vx", "vy", "vz")])
    st = copy_state(s)
    oracle.hybrid_steps(st, p, 8)
    P1 = np.array([np.sum(st["m"] * st[k]) for k in ("vx", "vy", "vz")])
    assert np.all(np.abs(P1 - P0) < 1e-13)


# --------------------------------------------------------------------------
# Input generators (not part of the method; checked so the workloads are what they claim)
# --------------------------------------------------------------------------
def test_plummer_profile_and_virial():
    s = ics.plummer(20000, 1)
    r = np.sqrt(s["x"] ** 2 + s["y"] ** 2 + s["z"] ** 2)
    for R in (0.5, 1.0, 2.0):
        want = R ** 3 / (1 + R ** 2) ** 1.5
        assert abs(np.mean(r < R) - want) < 0.015
    T = 0.5 * np.sum(s["m"] * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2))
    assert abs(T - 3 * math.pi / 64) < 0.01        # Plummer: T = -W/2 = 3 pi G M^2 / (64 a)


def test_hernquist_envelope_bounds_target():
    # the speed sampler is a rejection sampler: its envelope must bound v^2 f(Psi - v^2/2) for every v
    from paper_1406_6158_gb300.ics import _hernquist_df
    Mh = (101.0 / 100.0) ** 2
    r = np.exp(np.random.default_rng(0).uniform(np.log(1e-7), np.log(100.0), 3000))
    psi = Mh / (r + 1.0)
    vesc = np.sqrt(2.0 * psi)
    frac = np.concatenate([np.linspace(0.0, 1.0, 4001)[1:], np.geomspace(1e-8, 1.0, 4001)])
    v = frac[None, :] * vesc[:, None]
    target = (v * v * _hernquist_df(psi[:, None] - 0.5 * v * v, Mh, 1.0)).max(axis=1)
    assert np.all(ics.hernquist_envelope(r) >= target)


def test_hernquist_profile():
    s = ics.hernquist(20000, 2)
    r = np.sqrt(s["x"] ** 2 + s["y"] ** 2 + s["z"] ** 2)
    assert r.max() <= 100.0 * (1 + 1e-9) + 1.0   # COM shift allowed
    Mh = (101.0 / 100.0) ** 2
    for R in (0.5, 1.0, 5.0):
        assert abs(np.mean(r < R) - Mh * R ** 2 / (R + 1) ** 2) < 0.015
