"""The C-ABI library builds for sm_103a, loads on a machine without a GPU, and
exports every entry point include/hybrid.h declares. No compute call is made."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1406_6158_gb300 import build, hybrid
    build.build()
    return hybrid.load()


def declared():
    text = open(os.path.join(ROOT, "include", "hybrid.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hybrid_[a-z_]+)\s*\(", text)))


def test_header_declares_the_path():
    names = declared()
    for f in ("hybrid_build_tree", "hybrid_soft_force", "hybrid_hard_force", "hybrid_kick", "hybrid_drift",
              "hybrid_step", "hybrid_step_batched", "hybrid_create", "hybrid_destroy"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1406_6158_gb300 import hybrid
    for name in declared():
        assert hasattr(lib, name), name
    assert sorted(hybrid.EXPORTS) == declared()


def test_library_is_sm103a(lib):
    # the fatbinary carries sm_103a code; checked from the build flags, not by decoding the binary
    from paper_1406_6158_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_invalid_params_rejected_without_gpu(lib):
    from paper_1406_6158_gb300 import hybrid
    bad = [
        dict(eps=-1.0), dict(R1=0.2, R2=0.1), dict(R1=0.1, R2=0.1), dict(n_hard=0), dict(n_leaf=0),
        dict(n_crit=0), dict(precision=2), dict(mac=1, a_err=0.0), dict(theta=-0.1),
        dict(threads_per_group=-1), dict(tile_depth=1), dict(tile_depth=5), dict(skin=-0.1),
        dict(skin=float("inf")), dict(skin=0.01, precision=0, R1=0.1, R2=0.2), dict(skin=0.01, R1=0.0, R2=0.0),
    ]
    for kw in bad:
        p = hybrid.Params(**kw).c()
        h = C.c_void_p()
        assert lib.hybrid_create(C.byref(h), C.byref(p), None) == hybrid.EINVAL, kw
        assert not h.value
    assert lib.hybrid_create(None, None, None) == hybrid.EINVAL
    assert lib.hybrid_autotune(None, None, 0, None, 0, None, None) == hybrid.EINVAL
    assert lib.hybrid_destroy(None) == hybrid.OK
    assert lib.hybrid_launch_count(None) == 0


def test_struct_layout_matches_header():
    # hybrid_params: 7 doubles + 7 int32 (84, padded to 88) + 1 double = 96; hybrid_system: int64 + 14 pointers +
    # pointer + int32
    from paper_1406_6158_gb300 import hybrid
    assert C.sizeof(hybrid.hybrid_params) == 96
    assert hybrid.hybrid_params.skin.offset == 88
    assert C.sizeof(hybrid.hybrid_system) == 8 + 8 * 15 + 8


def test_status_codes_match_header():
    # the binding's status constants are the header's enum values, in order
    from paper_1406_6158_gb300 import hybrid
    text = open(os.path.join(ROOT, "include", "hybrid.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"HYBRID_([A-Z]+)\s*=\s*(\d+)", text))
    for name in ("OK", "EINVAL", "ENOMEM", "ECUDA", "ECAPACITY", "ETIMEOUT", "ETOOLARGE"):
        assert getattr(hybrid, name) == enum[name], name


def test_params_fields_match_header():
    # hybrid_params fields in the header's order (the ctypes struct mirrors it)
    from paper_1406_6158_gb300 import hybrid
    text = open(os.path.join(ROOT, "include", "hybrid.h")).read()
    body = text[text.index("typedef struct {\n    double G"):text.index("} hybrid_params;")]
    names = re.findall(r"(?:double|int32_t)\s+([^;]+);", body)
    fields = [f.strip() for group in names for f in group.split(",")]
    assert fields == [f for f, _ in hybrid.hybrid_params._fields_]


def test_system_fields_match_header():
    from paper_1406_6158_gb300 import hybrid
    text = open(os.path.join(ROOT, "include", "hybrid.h")).read()
    end = text.index("} hybrid_system;")
    body = text[text.rindex("typedef struct {", 0, end):end]
    fields = []
    for decl in re.findall(r"^\s+([^;]+);", body, flags=re.M):
        names = decl.split(None, 1)[1] if not decl.startswith("const") else decl.split(None, 2)[2]
        fields += [f.strip().lstrip("*") for f in names.split(",")]
    assert fields == [f for f, _ in hybrid.hybrid_system._fields_]



def test_noalloc_binding_refuses_foreign_tensors_before_the_call(monkeypatch):
    # the kernels read n doubles through each pointer: float32, CPU or mismatched tensors must never reach them
    torch = pytest.importorskip("torch")
    from paper_1406_6158_gb300 import hybrid

    def no_load():
        raise AssertionError("the library was reached")

    monkeypatch.setattr(hybrid, "load", no_load)
    f64 = [torch.zeros(8, dtype=torch.float64) for _ in range(7)]
    with pytest.raises(ValueError, match="CUDA device"):
        hybrid.hybrid_energy_noalloc(*f64, 1.0, 0.01)
    f32 = [torch.zeros(8, dtype=torch.float32) for _ in range(7)]
    with pytest.raises(ValueError, match="float64"):
        hybrid.hybrid_energy_noalloc(*f32, 1.0, 0.01)
    with pytest.raises(ValueError, match="one length"):
        hybrid.hybrid_energy_noalloc(*f64[:6], torch.zeros(9, dtype=torch.float64), 1.0, 0.01)
