"""The C-ABI library builds, loads and exports every call include/otf_md.h
declares; the product code never reaches the oracle (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^OTF_API\s+[\w\s\*]*?\b(\w+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2503_07526_gb300 import build_lib

    return build_lib.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("md_init", "md_step", "corr_push", "corr_read", "gk_integrate"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)$", out, re.M))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_ctypes_loads_and_binds_every_symbol(built_lib):
    import paper_2503_07526_gb300 as pkg

    L = pkg.lib()
    for name in declared_symbols():
        assert hasattr(L, name)
    assert set(pkg.EXPORTS) == set(declared_symbols())


def test_gk_integrate_host_call_matches_closed_form(built_lib):
    """gk_integrate is host code (no GPU): trapezoid of phi^l is a geometric sum."""
    import numpy as np

    import paper_2503_07526_gb300 as pkg

    phi, L, dt = 0.85, 30, 0.1
    t = np.arange(L + 1) * dt
    I, run = pkg.gk_integrate(t, phi ** np.arange(L + 1), prefactor=3.0)
    want = dt * (0.5 + phi * (1 - phi ** L) / (1 - phi) - 0.5 * phi ** L)
    assert I == pytest.approx(3 * want, rel=1e-14)
    Icut, _ = pkg.gk_integrate(t, 1.0 - t, t_cut=0.25)
    assert Icut == pytest.approx(0.25 - 0.25 ** 2 / 2, rel=1e-14)
    with pytest.raises(pkg.MdError):
        pkg.gk_integrate([0.0, 1.0, 0.5], [1.0, 1.0, 1.0])


def test_product_code_never_imports_the_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2503_07526_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), fn
                assert "liboracle" not in src and "oracle.c" not in src, fn
