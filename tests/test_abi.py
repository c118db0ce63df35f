"""The C ABI library loads and exports every entry point that include/*.h
declares; argument checks that run before any CUDA call behave (no GPU
needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(qlbm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    from paper_1309_1656_gb300 import _build
    if not _build.up_to_date():
        g.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("qlbm_create", "qlbm_destroy", "qlbm_init_equilibrium", "qlbm_step", "qlbm_moments",
              "qlbm_conserved", "qlbm_get_state", "qlbm_set_state", "qlbm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_1309_1656_gb300 import qlbm
    for kw in (dict(lattice=5, dims=(4, 4, 1)), dict(lattice=2, dims=(4, 4, 2)),
               dict(lattice=3, dims=(0, 4, 4)), dict(lattice=2, dims=(4, 4, 1), tau=-1.0),
               dict(lattice=2, dims=(4, 4, 1), beta0=0.0),
               dict(lattice=2, dims=(4, 4, 1), precision=7),
               # 2^32 sites: beyond the kernels' 32-bit site index (155 GB in
               # FP16 at 2^31 would still fit the device, so this must be caught)
               dict(lattice=2, dims=(65536, 65536, 1), precision=2),
               dict(lattice=3, dims=(1024, 1024, 2048), precision=2)):
        args = dict(tau=0.8, beta0=1.0, dt=1.0, precision=0)
        args.update(kw)
        with pytest.raises(qlbm.QLBMError) as e:
            qlbm.qlbm_create(args["lattice"], args["dims"], args["tau"], args["beta0"], args["dt"],
                             args["precision"])
        assert e.value.code == qlbm.QLBM_ERR_INVALID_ARG
        assert qlbm.qlbm_last_error(None)


def header_constants():
    """Enumerators and #define constants of include/*.h: name -> value."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(QLBM_[A-Z0-9_]+)\s*=\s*(-?\d+)", text):
            out[m.group(1)] = int(m.group(2))
        for m in re.finditer(r"#define\s+(QLBM_[A-Z0-9_]+)\s+(-?\d+)\b", text):
            out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_the_header():
    from paper_1309_1656_gb300 import qlbm
    consts = header_constants()
    for name in ("QLBM_FP64", "QLBM_FP32", "QLBM_FP16_DEV", "QLBM_DF64", "QLBM_FP64_DF",
                 "QLBM_ERR_OOM", "QLBM_ERR_INVALID_ARG", "QLBM_ERR_UNSUPPORTED"):
        assert name in consts, name
    checked = 0
    for name, value in consts.items():
        if hasattr(qlbm, name):
            assert getattr(qlbm, name) == value, name
            checked += 1
    assert checked >= 10
    # every precision the binding names is one the header declares
    precs = {v for k, v in consts.items() if k in ("QLBM_FP64", "QLBM_FP32", "QLBM_FP16_DEV", "QLBM_DF64",
                                                    "QLBM_FP64_DF")}
    assert set(qlbm.PRECISIONS.values()) == precs


def test_create_rejects_the_precision_after_the_last(lib):
    from paper_1309_1656_gb300 import qlbm
    bad = max(qlbm.PRECISIONS.values()) + 1
    with pytest.raises(qlbm.QLBMError) as e:
        qlbm.qlbm_create(2, (4, 4, 1), 0.8, 1.0, 1.0, bad)
    assert e.value.code == qlbm.QLBM_ERR_INVALID_ARG


def test_binding_fails_loudly_without_the_library(tmp_path):
    # no CPU fallback: with the library absent, importing the binding raises
    import subprocess
    import sys
    code = ("import paper_1309_1656_gb300._build as b; b.LIB = %r\n"
            "try:\n"
            "    import paper_1309_1656_gb300.qlbm\n"
            "except ImportError as e:\n"
            "    print('ImportError:', e)\n"
            "else:\n"
            "    print('imported')\n") % str(tmp_path / "missing" / "libqlbm.so")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "ImportError: libqlbm.so is not built" in r.stdout, r.stdout
