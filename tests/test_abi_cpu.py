"""The C ABI without a GPU: the library builds, loads and exports every symbol
the header declares; its host-side schedule arithmetic agrees with the oracle;
argument checks that need no device reject bad input."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2209_00117_gb300 import build

    build.build()
    from paper_2209_00117_gb300 import _native

    return _native


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vd_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(native):
    lib = native.lib()
    declared = _declared("vd.h")
    assert len(declared) >= 20
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    # the binding declares a signature for every symbol, and nothing else
    assert sorted(native.SIGNATURES) == declared


def test_schedules_match_oracle(native, orc):
    from paper_2209_00117_gb300 import vd

    g = np.random.default_rng(11)
    for _ in range(2000):
        w, h = int(g.integers(1, 32769)), int(g.integers(1, 32769))
        s, d = int(g.integers(1, 1 << 23)), int(g.integers(0, 70))
        vn, ex = int(g.integers(0, 3)), int(g.integers(0, 3))
        assert vd.djfa_schedule(w, h, s, d, vn, ex) == orc.djfa_schedule(w, h, s, d, vn, ex)
        assert vd.jfa_schedule(w, h, ex) == orc.jfa_schedule(w, h, ex)


def test_schedule_argument_errors(native):
    lib = native.lib()
    ks = np.zeros(8, np.int32)
    nbs = np.zeros(8, np.int32)
    p, q = ks.ctypes.data, nbs.ctypes.data
    assert lib.vd_jfa_schedule(0, 5, 0, p, q, 8) == native.VD_EINVAL
    assert lib.vd_jfa_schedule(5, 32769, 0, p, q, 8) == native.VD_EINVAL
    assert lib.vd_jfa_schedule(5, 5, 3, p, q, 8) == native.VD_EINVAL
    assert lib.vd_jfa_schedule(5, 5, 0, None, None, 8) == native.VD_EINVAL
    assert lib.vd_jfa_schedule(5, 5, 0, None, None, 0) == 3
    assert lib.vd_djfa_schedule(5, 5, 0, 1, 2, 0, p, q, 8) == native.VD_EINVAL
    assert lib.vd_djfa_schedule(5, 5, 3, -1, 2, 0, p, q, 8) == native.VD_EINVAL
    assert lib.vd_djfa_schedule(5, 5, 3, 1, -2, 0, p, q, 8) == native.VD_EINVAL
    assert "extra_passes" in native.last_error() or "d_max" in native.last_error()


def test_create_rejects_bad_sizes_without_device(native):
    lib = native.lib()
    for w, h, n in [(0, 4, 1), (4, 0, 1), (32769, 4, 1), (4, 4, 0), (4, 4, -3)]:
        assert not lib.vd_create(w, h, n)
        assert native.last_error()


def test_null_context_is_einval(native):
    lib = native.lib()
    assert lib.vd_jfa(None, 0, 0) == native.VD_EINVAL
    assert lib.vd_djfa_step(None, 1, 2, 0, 0) == native.VD_EINVAL
    assert lib.vd_destroy(None) == native.VD_OK
    assert lib.vd_launch_count(None) == -1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2209_00117_gb300 import _native

    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _native.lib()


def _defines(header):
    """{name: value} of the header's integer #defines (plain or parenthesised)."""
    text = open(os.path.join(ROOT, "include", header)).read()
    out = {}
    for name, val in re.findall(r"^#define (VD_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text, flags=re.M):
        out[name] = int(val)
    return out


def test_binding_constants_match_header(native):
    """The Python binding's option, error, metric and neighbourhood constants
    equal the header's, so a caller of either sees the same numbers."""
    from paper_2209_00117_gb300 import vd

    d = _defines("vd.h")
    opts = {k[len("VD_OPT_"):]: v for k, v in d.items() if k.startswith("VD_OPT_")}
    bopts = {k[len("VD_BOPT_"):]: v for k, v in d.items() if k.startswith("VD_BOPT_")}
    assert opts and bopts
    for name, v in opts.items():
        assert getattr(vd, "OPT_" + name) == v, name
    for name, v in bopts.items():
        assert getattr(vd, "BOPT_" + name) == v, name
    for name in ("VD_OK", "VD_EINVAL", "VD_ENOMEM", "VD_ECUDA", "VD_ETIMEOUT", "VD_EBUSY", "VD_ENOTFOUND"):
        assert getattr(native, name) == d[name], name
    assert (vd.EUCLID, vd.MANHATTAN) == (d["VD_METRIC_EUCLID"], d["VD_METRIC_MANHATTAN"])
    assert (vd.MOORE, vd.VON_NEUMANN) == (d["VD_NB_MOORE"], d["VD_NB_VON_NEUMANN"])
    assert vd.MAX_PASSES == d["VD_MAX_PASSES"]
    assert len(vd.KERNEL_KINDS) == d["VD_KERNEL_KINDS"]
