"""hybrid_energy_noalloc, the allocation-free energy entry point, against
hybrid_energy (the context-owning call) through the C-ABI.

Both sum the same FP64 terms (kinetic 1/2 m v^2, softened pair potential of
Eq. 2 over i != j) in different orders. Every term of each sum has one sign,
so the relative difference is bounded by about n * 2^-53 (n = 20011:
2.2e-12); the tests use 1e-11. The allocation-free call reduces in a fixed
order, so two calls in a row must agree bit for bit.

Kept in a file collected last so that it runs both after every other test and
alone in a fresh process (the scratch set-up happens on its first call here).
"""
import ctypes as C

import numpy as np
import pytest

from paper_1406_6158_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-11


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1406_6158_gb300 import build, hybrid
    build.build()
    hybrid.load()
    return hybrid


def _energy_ctx(H, st, G, eps):
    P = H.Params(G=G, eps=eps, precision=0)
    ctx = H.Context(P)
    s = H.System(st, precision=0, ids=False)
    T, W = ctx.hybrid_energy(s)
    torch.cuda.synchronize()
    return T, W, s


def _args(s):
    return [s.t[k] for k in ("x", "y", "z", "vx", "vy", "vz", "m")]


@pytest.mark.parametrize("n,G,eps", [(20011, 1.0, 1.0 / 128), (257, 0.7, 0.05)])
def test_noalloc_matches_energy_twice(H, n, G, eps):
    st = ics.plummer(n, seed=11 + n)
    T0, W0, s = _energy_ctx(H, st, G, eps)
    T1, W1 = H.hybrid_energy_noalloc(*_args(s), G, eps)
    T2, W2 = H.hybrid_energy_noalloc(*_args(s), G, eps)
    assert abs(T1 - T0) <= RTOL * abs(T0) and abs(W1 - W0) <= RTOL * abs(W0), (T0, W0, T1, W1)
    assert abs(T2 - T0) <= RTOL * abs(T0) and abs(W2 - W0) <= RTOL * abs(W0), (T0, W0, T2, W2)
    assert (T1, W1) == (T2, W2)
    assert W1 < 0.0 < T1


def test_noalloc_on_a_side_stream(H):
    st = ics.plummer(5003, seed=5)
    T0, W0, s = _energy_ctx(H, st, 1.0, 0.01)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        T, W = H.hybrid_energy_noalloc(*_args(s), 1.0, 0.01, stream=side)
        assert abs(T - T0) <= RTOL * abs(T0) and abs(W - W0) <= RTOL * abs(W0)


def test_noalloc_takes_no_device_memory(H):
    # after a first call on the device (set-up: scratch address, kernels loaded), further calls leave the
    # device's free memory and torch's reserved pool exactly where they were
    st = ics.plummer(3001, seed=3)
    _, _, s = _energy_ctx(H, st, 1.0, 0.02)
    H.hybrid_energy_noalloc(*_args(s), 1.0, 0.02)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(2):
        H.hybrid_energy_noalloc(*_args(s), 1.0, 0.02)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_limits(H):
    L = H.load()
    T, W = C.c_double(7.0), C.c_double(7.0)
    # n = 0: set-up only, zeros
    assert L.hybrid_energy_noalloc(0, None, None, None, None, None, None, None, 1.0, 0.0, None,
                                   C.byref(T), C.byref(W)) == H.OK
    assert (T.value, W.value) == (0.0, 0.0)
    # sizes beyond the fixed scratch are refused on the host, before any launch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    assert L.hybrid_energy_noalloc(H.ENERGY_NOALLOC_MAX_N + 1, p, p, p, p, p, p, p, 1.0, 0.0, None,
                                   C.byref(T), C.byref(W)) == H.ETOOLARGE
    assert L.hybrid_energy_noalloc(-1, p, p, p, p, p, p, p, 1.0, 0.0, None, C.byref(T), C.byref(W)) == H.EINVAL
    with pytest.raises(H.HybridError, match="ETOOLARGE"):
        big = torch.zeros(H.ENERGY_NOALLOC_MAX_N + 1, dtype=torch.float64, device="cuda")
        H.hybrid_energy_noalloc(big, big, big, big, big, big, big, 1.0, 0.0)
    np.testing.assert_equal(H.ENERGY_NOALLOC_MAX_N, 4194304)
