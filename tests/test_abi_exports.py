"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/prenom.h declares (no compute calls here)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "prenom.h")).read()
    return sorted(set(re.findall(r"^PRENOM_API\s+[\w\s\*]*?\b(prenom_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("prenom_create", "prenom_create_object", "prenom_set_prior_grid", "prenom_train_step",
                 "prenom_render", "prenom_render_backward", "prenom_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2503_01582_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_debug_bounds_build_exports_every_declared_symbol():
    """The bounds-checked debug build (the same sources with PRENOM_DEBUG_BOUNDS)
    compiles and exports the same entry points."""
    from paper_2503_01582_gb300 import build

    path = build.build(debug_bounds=True)
    assert path.endswith("libprenom_debug.so")
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol():
    from paper_2503_01582_gb300 import _abi

    assert sorted(_abi.symbols()) == _declared()
    for n in _declared():
        assert callable(getattr(_abi, n))


def test_package_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2503_01582_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "prenom_oracle" not in text, f


def test_arch_param_count_matches_oracle_layout(orc):
    """Host-only query of the library (no device work): the parameter count of
    an architecture equals the oracle's for the same layout contract."""
    import paper_2503_01582_gb300 as pkg
    from paper_2503_01582_gb300 import build

    build.build()
    cases = [dict(L=8, F=2, log2T=14, n_min=16, n_max=256, width=32, hidden=2),
             dict(L=16, F=2, log2T=19, n_min=16, n_max=2048, width=64, hidden=2),
             dict(L=4, F=2, log2T=12, n_min=16, n_max=64, width=16, hidden=3),
             dict(L=16, F=2, log2T=14, n_min=16, n_max=2048, width=16, hidden=1)]
    for c in cases:
        assert pkg.arch_param_count(pkg.make_arch(**c)) == orc.param_count(orc.Arch(**c)), c
    import pytest

    with pytest.raises(pkg.PrenomError) as e:
        pkg.arch_param_count(pkg.make_arch(width=48))
    assert e.value.code == -1


def test_noalloc_step_refuses_bad_arguments_on_the_host():
    """The allocation-free step checks its arguments before any CUDA call, so
    these refusals run without a GPU (the pointers are never dereferenced):
    moment buffers off a 16-byte boundary (its Adam pass moves four floats at
    a time), flags it cannot honour, out-of-range Adam constants and grids."""
    import pytest

    import paper_2503_01582_gb300 as pkg
    from paper_2503_01582_gb300 import _abi, build

    build.build()
    arch = pkg.make_arch()
    batch = _abi.prenom_ray_batch()
    ok = pkg.make_opts()

    def refused(theta, m, v, opts=ok, grid=0, res=0, what=""):
        with pytest.raises(_abi.PrenomError) as e:
            _abi.prenom_train_step_noalloc(arch, theta, m, v, 0, grid, res, batch, opts)
        assert e.value.code == _abi.PRENOM_ERR_INVALID_ARG
        assert what in _abi.prenom_last_error(None)

    base = 1 << 20  # an aligned fake address
    refused(base + 4, base, base, what="16-byte aligned")
    refused(base, base + 4, base, what="16-byte aligned")
    refused(base, base, base + 8, what="16-byte aligned")
    for flag in (pkg.PRENOM_FLAG_NO_ADAM, pkg.PRENOM_FLAG_CHECK_FINITE, pkg.PRENOM_FLAG_SPLIT):
        refused(base, base, base, opts=pkg.make_opts(flags=flag), what="not supported")
    refused(base, base, base, opts=pkg.make_opts(lr=float("nan")), what="Adam constants")
    refused(base, base, base, opts=pkg.make_opts(escape_eps=float("inf")), what="escape_eps")
    refused(base, base, base, grid=base, res=2048, what="res")


def test_binding_constants_match_the_header():
    """Every numeric constant the header defines (error codes, precisions,
    feature types, flags, state and kernel ids, the allocation-free limit) has
    the same value in the binding."""
    from paper_2503_01582_gb300 import _abi

    src = open(os.path.join(ROOT, "include", "prenom.h")).read()
    defs = re.findall(r"^#define (PRENOM_[A-Z0-9_]+)\s+(\(1u? << [0-9]+\)|\(?-?[0-9]+u?\)?)", src, flags=re.M)
    assert len(defs) >= 30
    for name, text in defs:
        t = text.strip("()").replace("u", "")
        value = (1 << int(t.split("<<")[1])) if "<<" in t else int(t)
        assert getattr(_abi, name) == value, name
