"""GPU path vs the FP64 oracle, through the C-ABI (libhybrid.so).

Keys, sort order, tree topology and groups: bit-exact. Moments: 1e-12
relative in the FP64 form; in the FP32 form (FP32 sums of at most 128 terms,
FP64 between chunks) a few 1e-6 of the cell side. Lists: equal as sets
except where a test lies within 1e-6 relative of its threshold. Forces: FP64
form within 1e-12 of the sum of term magnitudes; FP32 form within 1e-5
relative at the 99th percentile.
"""
import numpy as np
import pytest

import oracle
from paper_1406_6158_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIST_BAND = 1e-6


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_6158_gb300 import build, hybrid
    build.build()
    hybrid.load()
    return hybrid


def oparams(P):
    return oracle.Params(G=P.G, eps=P.eps, theta=P.theta, R1=P.R1, R2=P.R2, dt_soft=P.dt_soft, a_err=P.a_err,
                         n_hard=P.n_hard, n_leaf=P.n_leaf, n_crit=P.n_crit, mac=P.mac)


def gpu_tree(H, st, P):
    ctx = H.Context(P)
    s = H.System(st, precision=P.precision)
    ctx.hybrid_build_tree(s)
    torch.cuda.synchronize()
    return ctx, s, ctx.tree(s.n)


def plummer_params(n, prec, **kw):
    eps = kw.pop("eps", 1.0 / 64)
    d = dict(eps=eps, theta=0.5, R1=4 * eps, R2=8 * eps, precision=prec)
    d.update(kw)
    from paper_1406_6158_gb300 import hybrid
    return hybrid.Params(**d)


CASES = [
    ("plummer4096", lambda: ics.plummer(4096, 0), {}),
    ("plummer10007_ragged", lambda: ics.plummer(10007, 3), dict(n_crit=32, n_leaf=8)),
    ("hernquist20000", lambda: ics.hernquist(20000, 2), dict(theta=0.4, eps=1 / 512)),
    ("leaf1_capacity", lambda: ics.plummer(6000, 5), dict(n_leaf=1, n_crit=16)),
]
# the absolute MAC (Eq. 5) with the paper's a_err, and the normal tree (R1 = R2 = 0: K = 0, no hard part)
MODE_CASES = [
    ("absmac8000", lambda: ics.plummer(8000, 11), dict(mac=1, a_err=2.0 ** -8)),
    ("normal6000", lambda: ics.plummer(6000, 12), dict(R1=0.0, R2=0.0)),
    ("normal_absmac6000", lambda: ics.plummer(6000, 13), dict(R1=0.0, R2=0.0, mac=1, a_err=2.0 ** -8)),
]


def coincident_state():
    n = 300
    st = ics.plummer(n, 7)
    for k in ("x", "y", "z"):
        st[k][:100] = 0.125                      # 100 particles on one point
    st["x"][100:130] = st["x"][100]              # 30 on a line
    return st


def check_tree(T, G, prec):
    n = T.n
    assert np.array_equal(G["key"], T.key)
    assert len(G["level"]) == T.nn
    for f in ("level", "first", "count", "child", "nchild", "parent"):
        assert np.array_equal(G[f], getattr(T, f)), f
    assert np.array_equal(G["gnode"], T.gnode)
    assert np.array_equal(G["glo"], T.glo) and np.array_equal(G["ghi"], T.ghi)
    mo, gm = T.moments, G["moments"]
    scale = np.abs(np.stack([mo["cx"], mo["cy"], mo["cz"]], 1)).max(1) + mo["side"]
    side = mo["side"]
    assert np.array_equal(gm[:, 7], side)
    for k, f in ((8, "ox"), (9, "oy"), (10, "oz")):
        assert np.array_equal(gm[:, k], mo[f]), f
    if prec == 0:
        # FP64 form: every moment in FP64
        assert np.all(np.abs(gm[:, 0] - mo["M"]) <= 1e-12 * mo["M"] + 1e-300)
        for k, f in ((1, "cx"), (2, "cy"), (3, "cz")):
            assert np.all(np.abs(gm[:, k] - mo[f]) <= 1e-12 * scale), f
        assert np.all(np.abs(gm[:, 5] - mo["B2"]) <= 1e-12 * (mo["B2"] + mo["M"] * side ** 2))
        assert np.all(np.abs(gm[:, 6] - mo["delta"]) <= 1e-12 * scale)
        assert np.all(np.abs(gm[:, 4] - mo["bmax"]) <= 1e-12 * mo["bmax"] + 1e-12 * scale)
        rtol = 1e-12
    else:
        # FP32 form: sums of at most 128 FP32 terms on exact hi/lo offsets, chunks added in FP64;
        # offsets are good to ~1e-7 of the cell, so moments carry ~1e-6 of the cell side
        assert np.all(np.abs(gm[:, 0] - mo["M"]) <= 2e-6 * mo["M"])
        for k, f in ((1, "cx"), (2, "cy"), (3, "cz")):
            assert np.all(np.abs(gm[:, k] - mo[f]) <= 2e-6 * side), f
        assert np.all(np.abs(gm[:, 5] - mo["B2"]) <= 1e-5 * mo["B2"] + 1e-10 * mo["M"] * side ** 2)
        assert np.all(np.abs(gm[:, 6] - mo["delta"]) <= 4e-6 * side)
        assert np.all(np.abs(gm[:, 4] - mo["bmax"]) <= 2e-6 * mo["bmax"] + 4e-6 * side)
        rtol = 4e-6
    fin = np.isfinite(mo["rb"])
    assert np.array_equal(np.isfinite(gm[:, 11]), fin)
    if T.params.mac == 1:
        # Eq. (5): r_b = b/2 + sqrt(b^2/4 + sqrt(3 B2 / a_err)) is monotone in b_max and B2, so the tolerances
        # held above for b_max and B2 bound it (the fourth root magnifies small B2's errors)
        tb = (1e-12 if prec == 0 else 2e-6) * mo["bmax"] + (1e-12 if prec == 0 else 4e-6) * scale
        tB = (1e-12 if prec == 0 else 1e-5) * mo["B2"] + (1e-12 if prec == 0 else 1e-10) * mo["M"] * side ** 2

        def rb(b, B2):
            return 0.5 * b + np.sqrt(0.25 * b * b + np.sqrt(3.0 * np.maximum(B2, 0.0) / T.params.a_err))
        lo = rb(np.maximum(mo["bmax"] - tb, 0.0), mo["B2"] - tB)
        hi = rb(mo["bmax"] + tb, mo["B2"] + tB)
        slack = rtol * side
        assert np.all(gm[fin, 11] >= lo[fin] - slack[fin]) and np.all(gm[fin, 11] <= hi[fin] + slack[fin])
    else:
        assert np.all(np.abs(gm[fin, 11] - mo["rb"][fin]) <= rtol * (mo["rb"][fin] + side[fin]))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,mk,kw", CASES + MODE_CASES[:1], ids=[c[0] for c in CASES + MODE_CASES[:1]])
def test_tree_bit_exact(H, name, mk, kw, prec):
    st = mk()
    P = plummer_params(len(st["x"]), prec, **kw)
    ctx, s, G = gpu_tree(H, st, P)
    T = oracle.Tree(st["x"], st["y"], st["z"], st["m"], oparams(P))
    out = s.numpy()
    assert np.array_equal(out["id"], T.perm)                       # sort order, ties by input order
    assert np.array_equal(out["x"], T.x) and np.array_equal(out["m"], T.m)
    assert np.array_equal(ctx.hybrid_get_perm(T.n).cpu().numpy(), T.perm)
    check_tree(T, G, prec)


@pytest.mark.parametrize("sizes", [[1 << 21], [700001], [300000, 5, 1 << 20, 77777]],
                         ids=["2M_tiles2048", "700k_tiles1024", "batched_ragged"])
def test_sort_order_large(H, sizes):
    # The radix tile grows with N (512, 1024, 2048 keys): at every tile size the order is the stable order of
    # the oracle's Morton keys, and systems that share the digit passes do not mix.
    states = [ics.plummer(n, 20 + k) for k, n in enumerate(sizes)]
    P = plummer_params(max(sizes), 1, eps=1 / 256)
    ctx = H.Context(P)
    systems = [H.System(st, precision=1) for st in states]
    if len(systems) == 1:
        ctx.hybrid_build_tree(systems[0])
    else:
        ctx.hybrid_step_batched(systems, 0)
    torch.cuda.synchronize()
    for st, s in zip(states, systems):
        lo, L = oracle.root_box(st["x"], st["y"], st["z"])
        perm = oracle.stable_sort(oracle.morton_keys(st["x"], st["y"], st["z"], lo, L))
        assert np.array_equal(s.numpy()["id"], perm)


def keyed_order(st):
    lo, L = oracle.root_box(st["x"], st["y"], st["z"])
    return oracle.stable_sort(oracle.morton_keys(st["x"], st["y"], st["z"], lo, L))


def set_positions(s, st):
    for d in "xyz":
        s.t[d].copy_(torch.as_tensor(st[d], device="cuda"))
    torch.cuda.synchronize()


def test_sample_sort_close_to_key_order_with_ties(H):
    # the key sort as it runs from one build to the next: the sample sort takes its splitters from the last
    # build's sorted keys. After a build on a state in key order, the positions move by a small drift and 1000
    # particles spread through the array go to 10 points (equal keys far apart in the current order): the next
    # build takes the sample sort (no fallback) and gives the oracle's stable order and tree.
    n = 300000
    st = ics.plummer(n, 90)
    st = {k: v[keyed_order(st)].copy() for k, v in st.items()}
    P = plummer_params(n, 1, eps=1 / 256)
    ctx = H.Context(P)
    s = H.System(st, precision=1)
    ctx.hybrid_build_tree(s)              # the first build of a context may take the radix sort
    torch.cuda.synchronize()
    f0 = ctx.hybrid_sort_fallbacks()
    assert np.array_equal(s.numpy()["id"], np.arange(n))
    st1 = {k: v.copy() for k, v in st.items()}
    for d in "xyz":
        st1[d] = st1[d] + 1e-3 * st1["v" + d]
    rng = np.random.default_rng(3)
    pick = rng.choice(n, 1000, replace=False)
    pts = rng.normal(size=(10, 3))
    for k, d in enumerate("xyz"):
        st1[d][pick] = pts[np.arange(1000) % 10, k]
    set_positions(s, st1)
    ctx.hybrid_build_tree(s)
    torch.cuda.synchronize()
    assert ctx.hybrid_sort_fallbacks() == f0
    assert np.array_equal(s.numpy()["id"], keyed_order(st1))
    T = oracle.Tree(st1["x"], st1["y"], st1["z"], st1["m"], oparams(P))
    check_tree(T, ctx.tree(n), 1)


def test_sample_sort_overflow_falls_back_to_radix(H):
    # splitters that do not fit the state: after a build on a Plummer sphere (its sorted keys give the next
    # build's splitters, at positions j n / nb, nb = ceil(n / 1024) on a batch of at most 2^20 particles), the
    # particles are replaced by a uniform cube, some of whose buckets hold more than 4096 keys. The build is
    # repeated with the radix sort, which gives the same stable order; the build after it takes the sample sort
    # again.
    n = 100000
    st = ics.plummer(n, 91)
    st = {k: v[keyed_order(st)].copy() for k, v in st.items()}
    P = plummer_params(n, 1)
    ctx = H.Context(P)
    s = H.System(st, precision=1)
    ctx.hybrid_build_tree(s)
    torch.cuda.synchronize()
    f0 = ctx.hybrid_sort_fallbacks()
    cube = {k: v.copy() for k, v in st.items()}
    rng = np.random.default_rng(4)
    for d in "xyz":
        cube[d] = rng.uniform(-1.0, 1.0, n)
    # the precondition, from the splitters' definition: the cube's composites (key, position) against the
    # Plummer sphere's sorted composites at positions j n / nb
    nb = (n + 1023) // 1024
    lo, L = oracle.root_box(st["x"], st["y"], st["z"])
    ka = np.sort(oracle.morton_keys(st["x"], st["y"], st["z"], lo, L))
    pos = (np.arange(1, nb) * n) // nb
    lo, L = oracle.root_box(cube["x"], cube["y"], cube["z"])
    kb = oracle.morton_keys(cube["x"], cube["y"], cube["z"], lo, L)
    comp_a = ka[pos].astype(object) * n + pos
    comp_b = kb.astype(object) * n + np.arange(n)
    bucket = np.searchsorted(np.array(sorted(comp_a), dtype=object), comp_b, side="right")
    assert np.bincount(bucket.astype(np.int64)).max() > 4096
    set_positions(s, cube)
    ctx.hybrid_build_tree(s)
    torch.cuda.synchronize()
    assert ctx.hybrid_sort_fallbacks() == f0 + 1
    assert np.array_equal(s.numpy()["id"], keyed_order(cube))
    T = oracle.Tree(cube["x"], cube["y"], cube["z"], cube["m"], oparams(P))
    check_tree(T, ctx.tree(n), 1)
    ctx.hybrid_build_tree(s)              # now in key order: the sample sort again
    torch.cuda.synchronize()
    assert ctx.hybrid_sort_fallbacks() == f0 + 1
    assert np.array_equal(s.numpy()["id"], keyed_order(cube))


def test_empty_system_refused(H):
    # an empty system (n = 0) is refused with EINVAL before anything is enqueued, alone and inside a batch, and the
    # context then steps a real system normally
    ctx = H.Context(plummer_params(64, 1))
    empty = H.System({k: np.zeros(0) for k in H.System.FIELDS}, precision=1)
    other = H.System(ics.plummer(64, 3), precision=1)
    for call in (lambda: ctx.hybrid_build_tree(empty), lambda: ctx.hybrid_step(empty, 1),
                 lambda: ctx.hybrid_step_batched([other, empty], 1)):
        with pytest.raises(H.HybridError) as err:
            call()
        assert err.value.code == H.EINVAL
    s = H.System(ics.plummer(64, 3), precision=1)
    ctx.hybrid_step(s, 1)
    torch.cuda.synchronize()
    out = s.numpy()
    assert all(np.all(np.isfinite(out[k])) for k in ("x", "vx", "ax_s", "ax_h"))
    ctx.close()


@pytest.mark.parametrize("n", [1, 2, 3, 17, 33])
def test_tiny_and_coincident(H, n):
    st = ics.plummer(max(n, 2), 9)
    st = {k: v[:n].copy() for k, v in st.items()}
    P = plummer_params(n, 1, n_leaf=1, n_crit=2)
    ctx, s, G = gpu_tree(H, st, P)
    T = oracle.Tree(st["x"], st["y"], st["z"], st["m"], oparams(P))
    assert np.array_equal(s.numpy()["id"], T.perm)
    check_tree(T, G, 1)
    st = coincident_state()
    P = plummer_params(len(st["x"]), 0, n_leaf=4, n_crit=8)
    ctx, s, G = gpu_tree(H, st, P)
    T = oracle.Tree(st["x"], st["y"], st["z"], st["m"], oparams(P))
    assert np.array_equal(s.numpy()["id"], T.perm)
    check_tree(T, G, 0)
    assert T.level.max() == 21


def ancestors(T, c):
    out = []
    while c >= 0:
        out.append(c)
        c = T.parent[c]
    return out


def leaf_of(T):
    lf = np.zeros(T.n, dtype=np.int64)
    for c in np.where(T.nchild == 0)[0]:
        lf[T.first[c]:T.first[c] + T.count[c]] = c
    return lf


def near_threshold(T, g, c, hard):
    mo = T.moments
    p = np.array([mo["cx"][c], mo["cy"][c], mo["cz"][c]])
    gap = np.maximum(np.maximum(T.glo[g] - p, 0.0), p - T.ghi[g])
    d = np.sqrt(np.sum(gap * gap))
    hr = T.params.R2 + mo["bmax"][c]
    thr = hr if hard else max(mo["rb"][c], hr)
    return np.isfinite(thr) and abs(d - thr) <= LIST_BAND * thr


def lists_match(T, gl, ol):
    lf = leaf_of(T)
    flips = 0
    for g, (a, b) in enumerate(zip(gl, ol)):
        for k in range(3):
            A, B = set(a[k].tolist()), set(b[k].tolist())
            if A == B:
                continue
            for e in A ^ B:
                node = e if k == 0 else lf[e]
                ok = any(near_threshold(T, g, c, k == 2) for c in ancestors(T, node))
                assert ok, "group %d list %d entry %d differs away from a threshold" % (g, k, e)
                flips += 1
    return flips


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,mk,kw", CASES[:3] + MODE_CASES, ids=[c[0] for c in CASES[:3] + MODE_CASES])
def test_lists_and_forces(H, name, mk, kw, prec):
    st = mk()
    P = plummer_params(len(st["x"]), prec, **kw)
    ctx = H.Context(P)
    s = H.System(st, precision=prec)
    ctx.hybrid_build_tree(s)
    ctx.hybrid_hard_force(s)
    ctx.hybrid_soft_force(s)              # the last walk holds soft lists
    torch.cuda.synchronize()
    out = s.numpy()
    T = oracle.Tree(out["x"], out["y"], out["z"], out["m"], oparams(P))
    assert np.array_equal(T.perm, np.arange(T.n))
    gl = ctx.lists(T.ng)
    ol = T.walk(mode=1)
    flips = lists_match(T, gl, ol)
    if prec == 0:
        assert flips == 0
    a_s, a_h, sc_s, sc_h = T.forces()
    g_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)
    g_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)
    if prec == 0:
        # a pair at r = R2 to the last bit has K ~ 1e-90 on one side and exactly 0 on the other
        floor = 1e-24 * np.max(sc_s)
        assert np.all(np.abs(g_s - a_s) <= 1e-12 * sc_s[:, None] + floor)
        assert np.all(np.abs(g_h - a_h) <= 1e-12 * sc_h[:, None] + floor)
    else:
        es = np.linalg.norm(g_s - a_s, axis=1) / np.linalg.norm(a_s, axis=1)
        assert np.percentile(es, 99) <= 1e-5, np.percentile(es, 99)
        nz = np.linalg.norm(a_h, axis=1) > 0
        if nz.any():
            eh = np.linalg.norm(g_h - a_h, axis=1)[nz] / np.linalg.norm(a_h, axis=1)[nz]
            assert np.percentile(eh, 99) <= 1e-5, np.percentile(eh, 99)
        assert np.all(np.linalg.norm(g_h, axis=1)[~nz] == 0.0)
    far, near = ctx.hybrid_interactions()   # the last evaluation was the soft force
    os_, oh = T.interactions(mode=3)
    assert far + near == os_ or prec == 1
    assert abs(far + near - os_) <= 1e-3 * os_


@pytest.mark.parametrize("n_crit,tpg,depth", [(64, 8, 0), (256, 32, 2), (32, 16, 4), (16, 16, 3), (256, 64, 4)],
                         ids=["ks8", "ks8-ncrit256-depth2", "ks2-depth4", "ks1", "ks4-ncrit256-depth4"])
def test_forces_every_kernel_setting(H, n_crit, tpg, depth):
    # every sinks-per-lane variant (1, 2, 4, 8) and staging depth of the FP32 pair kernels against the oracle
    st = ics.plummer(12000, 61)
    P = plummer_params(12000, 1, n_crit=n_crit, threads_per_group=tpg, tile_depth=depth)
    ctx = H.Context(P)
    s = H.System(st, precision=1)
    ctx.hybrid_build_tree(s)
    ctx.hybrid_hard_force(s)
    ctx.hybrid_soft_force(s)
    torch.cuda.synchronize()
    out = s.numpy()
    T = oracle.Tree(out["x"], out["y"], out["z"], out["m"], oparams(P))
    a_s, a_h, sc_s, sc_h = T.forces()
    g_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)
    g_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)
    es = np.linalg.norm(g_s - a_s, axis=1) / np.linalg.norm(a_s, axis=1)
    assert np.percentile(es, 99) <= 1e-5, np.percentile(es, 99)
    nz = np.linalg.norm(a_h, axis=1) > 0
    eh = np.linalg.norm(g_h - a_h, axis=1)[nz] / np.linalg.norm(a_h, axis=1)[nz]
    assert np.percentile(eh, 99) <= 1e-5, np.percentile(eh, 99)
    assert np.all(np.linalg.norm(g_h, axis=1)[~nz] == 0.0)


def test_hard_lists_and_theta_zero(H):
    st = ics.plummer(3000, 4)
    for prec in (0, 1):
        P = plummer_params(3000, prec, theta=0.0)
        ctx = H.Context(P)
        s = H.System(st, precision=prec)
        ctx.hybrid_build_tree(s)
        ctx.hybrid_soft_force(s)
        ctx.hybrid_hard_force(s)              # the last walk holds hard lists
        out = s.numpy()
        T = oracle.Tree(out["x"], out["y"], out["z"], out["m"], oparams(P))
        gl = ctx.lists(T.ng)
        ol = T.walk(mode=2)
        assert lists_match(T, gl, ol) == 0 or prec == 1
        # theta = 0: soft + hard equals direct summation
        full, sc = oracle.direct(T.x, T.y, T.z, T.m, eps=P.eps)
        g = (np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64) +
             np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64))
        if prec == 0:
            assert np.all(np.abs(g - full) <= 1e-12 * sc[:, None])
        else:
            e = np.linalg.norm(g - full, axis=1) / np.linalg.norm(full, axis=1)
            assert np.percentile(e, 99) <= 1e-5


def test_c1_trajectory_fp64(H):
    # Plummer N = 4096 seed 0, eps 1/64, theta 0.5, R1 = 4 eps, R2 = 8 eps, dt 1/128, n = 4, 16 steps, FP64
    st = ics.plummer(4096, 0)
    st["id"] = np.arange(4096, dtype=np.int64)
    P = plummer_params(4096, 0, dt_soft=1 / 128, n_hard=4)
    ctx = H.Context(P)
    s = H.System(st, precision=0)
    ctx.hybrid_step(s, 16)
    out = s.numpy()
    ost = {k: np.array(v, copy=True) for k, v in st.items()}
    a_s, a_h = oracle.hybrid_steps(ost, oparams(P), 16)
    assert np.array_equal(out["id"], ost["id"])
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        assert np.max(np.abs(out[k] - ost[k])) <= 1e-9, k
    assert np.allclose(np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1), a_s, rtol=0, atol=1e-9)


@pytest.mark.parametrize("kw", [dict(n_hard=4), dict(n_hard=1, R1=0.0, R2=0.0, mac=1, a_err=2.0 ** -8)],
                         ids=["hybrid", "normal_absmac"])
def test_step_fp32_close_to_oracle(H, kw):
    st = ics.plummer(2048, 8)
    st["id"] = np.arange(2048, dtype=np.int64)
    P = plummer_params(2048, 1, dt_soft=1 / 128, **kw)
    ctx = H.Context(P)
    s = H.System(st, precision=1)
    ctx.hybrid_step(s, 2)
    out = s.numpy()
    ost = {k: np.array(v, copy=True) for k, v in st.items()}
    oracle.hybrid_steps(ost, oparams(P), 2)
    o = np.argsort(out["id"])
    q = np.argsort(ost["id"])
    for k in ("x", "y", "z"):
        assert np.max(np.abs(out[k][o] - ost[k][q])) <= 1e-8


@pytest.mark.parametrize("graphs", [False, True], ids=["eager", "graphs"])
@pytest.mark.parametrize("skin", [0.05, 1e-7], ids=["reused", "skin_exceeded_rebuilds"])
def test_reused_lists_follow_the_oracle(H, skin, graphs):
    # skin > 0: hard steps 1..n-1 reuse the tree and the neighbour lists of the last build (an option outside
    # the paper). At theta = 0 the soft force is direct summation whichever lists carry it and the hard force
    # takes every pair within R2, so three soft steps must follow the oracle (which rebuilds at every hard
    # step) to FP32 force rounding. With a skin of 1e-7 the first drift moves particles beyond skin / 2 and the
    # step falls back to rebuilding; with 0.05 the reuse holds and the step launches fewer kernels. On a stream
    # of its own the step replays a captured graph, and a fallback resumes eagerly after the graph.
    n = 2048
    st = ics.plummer(n, 8)
    st["id"] = np.arange(n, dtype=np.int64)
    launches = []
    for sk in (0.0, skin):
        P = plummer_params(n, 1, theta=0.0, dt_soft=1 / 128, n_hard=4, skin=sk)
        ctx = H.Context(P, torch.cuda.Stream() if graphs else None)
        s = H.System(st, precision=1)
        torch.cuda.synchronize()
        ctx.hybrid_step(s, 0)
        l0 = ctx.hybrid_launch_count()
        for _ in range(3):
            ctx.hybrid_step(s, 1)
        torch.cuda.synchronize()
        launches.append(ctx.hybrid_launch_count() - l0)
        out = s.numpy()
        ost = {k: np.array(v, copy=True) for k, v in st.items()}
        oracle.hybrid_steps(ost, oparams(P), 3)
        o, q = np.argsort(out["id"]), np.argsort(ost["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            assert np.max(np.abs(out[k][o] - ost[k][q])) <= 1e-8, (sk, k)
        ctx.close()
    if skin > 1e-3:
        assert launches[1] < launches[0]
    else:
        assert launches[1] >= launches[0]


def test_reused_lists_close_to_rebuilds_at_theta(H):
    # theta = 0.5: the skin changes the tree opening (cells are taken only beyond R2 + skin + b_max), so the
    # soft force differs from the rebuilt one by less than the tree error (~1e-3 rms); over three soft steps of
    # 1/128 that moves positions by far less than 1e-6. The graph path (a stream of its own) replays the reuse.
    n = 6000
    st = ics.plummer(n, 31)
    res = []
    for sk in (0.0, 0.04):
        P = plummer_params(n, 1, dt_soft=1 / 128, n_hard=4, skin=sk)
        ctx = H.Context(P, torch.cuda.Stream())
        s = H.System(st, precision=1)
        torch.cuda.synchronize()
        for _ in range(3):
            ctx.hybrid_step(s, 1)
        torch.cuda.synchronize()
        out = s.numpy()
        res.append({k: out[k][np.argsort(out["id"])] for k in ("x", "y", "z", "vx")})
        ctx.close()
    for k in ("x", "y", "z"):
        assert np.max(np.abs(res[0][k] - res[1][k])) <= 1e-6, k


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_equals_alone(H, prec):
    sizes = [1000, 5003, 2500]
    states = [ics.plummer(n, 20 + k) for k, n in enumerate(sizes)]
    P = plummer_params(1000, prec, n_hard=2)
    per = [H.Params(**{**P.__dict__, "eps": 1 / (4 * n ** (1 / 3)), "R1": 4 / (4 * n ** (1 / 3)),
                       "R2": 8 / (4 * n ** (1 / 3))}) for n in sizes]
    ctx = H.Context(P)
    alone = []
    for st, p in zip(states, per):
        s = H.System(st, precision=prec, params=p)
        ctx.hybrid_step(s, 2)
        alone.append(s.numpy())
    sysb = [H.System(st, precision=prec, params=p) for st, p in zip(states, per)]
    ctx.hybrid_step_batched(sysb, 2)
    for a, s in zip(alone, sysb):
        b = s.numpy()
        if prec == 0:   # FP64: bitwise
            for k in ("x", "y", "z", "vx", "vy", "vz", "ax_s", "ax_h", "id"):
                assert np.array_equal(a[k], b[k]), k
        else:           # FP32: chunked sums are added atomically, so equal to rounding
            assert np.array_equal(a["id"], b["id"])
            for k in ("x", "y", "z"):
                assert np.max(np.abs(a[k] - b[k])) <= 1e-10
            for w in ("s", "h"):
                A = np.stack([a["a%s_%s" % (d, w)] for d in "xyz"], 1).astype(np.float64)
                B = np.stack([b["a%s_%s" % (d, w)] for d in "xyz"], 1).astype(np.float64)
                nz = np.linalg.norm(A, axis=1) > 0
                e = np.linalg.norm(A - B, axis=1)[nz] / np.linalg.norm(A, axis=1)[nz]
                assert np.percentile(e, 99) <= 1e-5


def test_autotune_choice_and_results(H):
    sizes = [3000, 1200, 4100]
    states = [ics.plummer(n, 40 + k) for k, n in enumerate(sizes)]
    P = plummer_params(3000, 1)
    ctx = H.Context(P)
    sysb = [H.System(st, precision=1) for st in states]
    before = [s.numpy() for s in sysb]
    cands = [(32, 8, 0), (64, 16, 3), (64, 32, 2), (128, 32, 4)]
    chosen, ms = ctx.hybrid_autotune(sysb, cands)
    assert chosen in cands and np.all(ms > 0)
    assert ms[cands.index(chosen)] == ms.min()
    assert (ctx.params.n_crit, ctx.params.threads_per_group, ctx.params.tile_depth) == chosen
    for b, s in zip(before, sysb):   # the autotuner only reads the systems
        a = s.numpy()
        for k in ("x", "y", "z", "vx", "vy", "vz", "m", "id"):
            assert np.array_equal(a[k], b[k]), k
    # a step with the tuned context equals one on a fresh context built with the chosen setting
    ctx.hybrid_step_batched(sysb, 1)
    P2 = H.Params(**{**P.__dict__, "n_crit": chosen[0], "threads_per_group": chosen[1], "tile_depth": chosen[2]})
    ref = [H.System(st, precision=1) for st in states]
    H.Context(P2).hybrid_step_batched(ref, 1)
    for s, r in zip(sysb, ref):
        a, b = s.numpy(), r.numpy()
        assert np.array_equal(a["id"], b["id"])
        for w in ("s", "h"):
            A = np.stack([a["a%s_%s" % (d, w)] for d in "xyz"], 1).astype(np.float64)
            B = np.stack([b["a%s_%s" % (d, w)] for d in "xyz"], 1).astype(np.float64)
            nz = np.linalg.norm(B, axis=1) > 0
            e = np.linalg.norm(A - B, axis=1)[nz] / np.linalg.norm(B, axis=1)[nz]
            assert np.percentile(e, 99) <= 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_eager(H, prec):
    # on a stream of its own the library captures each op sequence once (the tree build as a two-branch
    # graph) and replays it; on the legacy default stream it launches eagerly: same results
    st = ics.plummer(6000, 71)
    P = plummer_params(6000, prec, n_hard=2)
    runs = []
    for stream in (None, torch.cuda.Stream()):
        ctx = H.Context(P, stream)
        s = H.System(st, precision=prec)
        torch.cuda.synchronize()               # inputs made on the default stream are ready
        for k in range(3):
            ctx.hybrid_profile(k == 2)         # the last step also records the kernels' times
            ctx.hybrid_step(s, 1)
        torch.cuda.synchronize()
        runs.append(s.numpy())
        for kind in range(5):                  # far, near, walk, build, kicks: timed in both modes
            ms, n = ctx.hybrid_profile_read(kind)
            assert ms > 0.0 and n >= 1, (stream, kind)
        ctx.close()
    a, b = runs
    assert np.array_equal(a["id"], b["id"])
    # FP32 form: groups with several work items add their partial sums with atomics, in an order that differs
    # between runs, so accelerations agree to FP32 rounding of those sums (~1e-6 relative); three soft steps of
    # dt_s = 1/128 carry that into v and x at well below 1e-7
    for k in ("x", "y", "z", "vx", "vy", "vz"):
        if prec == 0:
            assert np.array_equal(a[k], b[k]), k
        else:
            assert np.max(np.abs(a[k] - b[k])) <= 1e-7 * max(1.0, np.max(np.abs(a[k]))), k


def test_bounded_wait_times_out_and_context_survives(H):
    # failure detection without a fault: a device wait on a flag nothing sets gives up after its polls,
    # the host reads HYBRID_ETIMEOUT, and the same context then steps normally
    st = ics.plummer(2000, 81)
    P = plummer_params(2000, 1)
    ctx = H.Context(P)
    assert ctx.hybrid_selftest_wait(1000) == H.ETIMEOUT
    assert ctx.hybrid_selftest_wait(1000) == H.ETIMEOUT      # the status was cleared and is raised again
    s = H.System(st, precision=1)
    ctx.hybrid_step(s, 1)
    ctx.hybrid_sync()
    assert np.all(np.isfinite(s.numpy()["x"]))


def test_kick_drift_calls(H):
    st = ics.plummer(1000, 30)
    P = plummer_params(1000, 0)
    ctx = H.Context(P)
    s = H.System(st, precision=0)
    s.t["ax_s"].fill_(0.5)
    s.t["ay_s"].fill_(-0.25)
    s.t["az_s"].fill_(2.0)
    ctx.hybrid_kick(s, 0, 0.125)
    ctx.hybrid_drift(s, 0.0625)
    out = s.numpy()
    vx = st["vx"] + 0.125 * 0.5
    assert np.array_equal(out["vx"], vx)
    assert np.array_equal(out["x"], st["x"] + 0.0625 * vx)


def test_c2_full_size_sampled(H):
    # Plummer N = 2^17 seed 1, eps 1/128, theta 0.5, R1 = 4 eps, R2 = 8 eps, FP32 pairs (the benchmark workload)
    n = 1 << 17
    st = ics.plummer(n, 1)
    P = plummer_params(n, 1, eps=1 / 128)
    ctx = H.Context(P)
    s = H.System(st, precision=1)
    ctx.hybrid_build_tree(s)
    ctx.hybrid_soft_force(s)
    ctx.hybrid_hard_force(s)
    out = s.numpy()
    T = oracle.Tree(out["x"], out["y"], out["z"], out["m"], oparams(P))
    assert np.array_equal(T.perm, np.arange(n))
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(T.ng, 300, replace=False))
    a_s, a_h, _, _ = T.forces(groups=sel)
    mask = ~np.isnan(a_s[:, 0])
    g_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)[mask]
    g_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)[mask]
    es = np.linalg.norm(g_s - a_s[mask], axis=1) / np.linalg.norm(a_s[mask], axis=1)
    assert np.percentile(es, 99) <= 1e-5
    nz = np.linalg.norm(a_h[mask], axis=1) > 0
    eh = np.linalg.norm(g_h - a_h[mask], axis=1)[nz] / np.linalg.norm(a_h[mask], axis=1)[nz]
    assert np.percentile(eh, 99) <= 1e-5


def sampled_lists_match(T, gl, ol, sel):
    """lists_match on the selected groups: gl maps a group to its GPU lists, ol holds the oracle's for sel."""
    lf = leaf_of(T)
    flips = 0
    for g, b in zip(sel, ol):
        a = gl[g]
        for k in range(3):
            A, B = set(a[k].tolist()), set(b[k].tolist())
            for e in A ^ B:
                node = e if k == 0 else lf[e]
                ok = any(near_threshold(T, g, c, k == 2) for c in ancestors(T, node))
                assert ok, "group %d list %d entry %d differs away from a threshold" % (g, k, e)
                flips += 1
    return flips


def sampled_forces_ok(T, out, sel):
    a_s, a_h, _, _ = T.forces(groups=sel)
    mask = ~np.isnan(a_s[:, 0])
    g_s = np.stack([out["ax_s"], out["ay_s"], out["az_s"]], 1).astype(np.float64)[mask]
    g_h = np.stack([out["ax_h"], out["ay_h"], out["az_h"]], 1).astype(np.float64)[mask]
    es = np.linalg.norm(g_s - a_s[mask], axis=1) / np.linalg.norm(a_s[mask], axis=1)
    assert np.percentile(es, 99) <= 1e-5, np.percentile(es, 99)
    nz = np.linalg.norm(a_h[mask], axis=1) > 0
    eh = np.linalg.norm(g_h - a_h[mask], axis=1)[nz] / np.linalg.norm(a_h[mask], axis=1)[nz]
    assert np.percentile(eh, 99) <= 1e-5, np.percentile(eh, 99)
    assert np.all(np.linalg.norm(g_h, axis=1)[~nz] == 0.0)


def large_params(n):
    eps = 1 / 512
    return plummer_params(n, 1, eps=eps, theta=0.4, R1=3 * eps, R2=6 * eps, n_crit=256)


def test_large_hernquist_tree_lists_forces(H):
    # Hernquist N = 2^21 (seed 2) with the large workload's parameters (eps 1/512, theta 0.4, R1 = 3 eps,
    # R2 = 6 eps, n_crit 256): radix tiles of 2048 keys and the large-batch item lengths. Keys, sort order,
    # topology, groups and group boxes bit-exact over the whole tree; soft and hard lists equal as sets (up to
    # the 1e-6 threshold band) and forces within 1e-5 at p99 on 200 sampled groups
    n = 1 << 21
    st = ics.hernquist(n, 2)
    P = large_params(n)
    ctx, s, G = gpu_tree(H, st, P)
    T = oracle.Tree(st["x"], st["y"], st["z"], st["m"], oparams(P))
    out = s.numpy()
    assert np.array_equal(out["id"], T.perm)
    assert np.array_equal(out["x"], T.x) and np.array_equal(out["m"], T.m)
    check_tree(T, G, 1)
    del G
    rng = np.random.default_rng(1)
    sel = np.sort(rng.choice(T.ng, 200, replace=False))
    ctx.hybrid_hard_force(s)              # a hard walk: the lists hold the hard neighbours
    torch.cuda.synchronize()
    flips_h = sampled_lists_match(T, ctx.lists(T.ng, sel), T.walk(sel, mode=2), sel)
    ctx.hybrid_soft_force(s)              # a soft walk: the lists hold cells and soft particles
    torch.cuda.synchronize()
    gl = ctx.lists(T.ng, sel)
    ol = T.walk(sel, mode=1)
    flips_s = sampled_lists_match(T, gl, ol, sel)
    total = sum(len(b[0]) + len(b[1]) + len(b[2]) for b in ol)
    assert flips_s + flips_h <= 1e-4 * total
    del gl
    sampled_forces_ok(T, s.numpy(), sel)
    ctx.close()


def test_large_workload_full_size_tree(H):
    # the large workload itself: Hernquist N = 2^24 (seed 2). Keys, sort order, topology, groups and group
    # boxes bit-exact against the oracle's tree of all 2^24 particles; forces on 64 sampled groups
    n = 1 << 24
    st = ics.hernquist(n, 2)
    P = large_params(n)
    ctx, s, G = gpu_tree(H, st, P)
    T = oracle.Tree(st["x"], st["y"], st["z"], st["m"], oparams(P))
    assert np.array_equal(s.numpy()["id"], T.perm)
    check_tree(T, G, 1)
    del G, st
    ctx.hybrid_soft_force(s)
    ctx.hybrid_hard_force(s)
    torch.cuda.synchronize()
    rng = np.random.default_rng(2)
    sampled_forces_ok(T, s.numpy(), np.sort(rng.choice(T.ng, 64, replace=False)))
    ctx.close()


def ragged_batch(prec):
    sizes = [1500, 3001, 777, 2048]
    states = [ics.plummer(n, 50 + k) for k, n in enumerate(sizes)]
    for k, st in enumerate(states):
        st["id"] = np.arange(sizes[k], dtype=np.int64)
    per = []
    for n in sizes:
        eps = 1 / (4 * n ** (1 / 3))
        per.append(plummer_params(n, prec, eps=eps, dt_soft=1 / 128, n_hard=4))
    return sizes, states, per


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_follows_the_oracle(H, prec):
    # every system of a ragged batch (its own N and eps, one call per step for all of them) against the
    # oracle run on that system alone, over two soft steps. FP64: positions and velocities within 1e-9. FP32
    # pairs: a force error of 1e-5 of |a| <= ~2 kicked over 2 dt_s = 1/64 moves v by up to ~3e-7 and x by
    # ~100 times less, so velocities within 1e-6 and positions within 1e-8
    sizes, states, per = ragged_batch(prec)
    ctx = H.Context(per[0])
    sysb = [H.System(st, precision=prec, params=p) for st, p in zip(states, per)]
    ctx.hybrid_step_batched(sysb, 2)
    tol_x, tol_v = (1e-9, 1e-9) if prec == 0 else (1e-8, 1e-6)
    for st, p, s in zip(states, per, sysb):
        out = s.numpy()
        ost = {k: np.array(v, copy=True) for k, v in st.items()}
        oracle.hybrid_steps(ost, oparams(p), 2)
        o, q = np.argsort(out["id"]), np.argsort(ost["id"])
        for k in ("x", "y", "z", "vx", "vy", "vz"):
            tol = tol_v if k.startswith("v") else tol_x
            assert np.max(np.abs(out[k][o] - ost[k][q])) <= tol, (len(st["x"]), k)
    ctx.close()
