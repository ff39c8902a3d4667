"""The C ABI library builds for sm_103a, loads, and exports every entry
point that include/pd.h declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pd_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("pd_features", "pd_objective_grad", "pd_hvp", "pd_assign", "pd_fit", "pd_K", "pd_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2605_20816_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in declared_symbols():
        assert re.search(r"\bT %s$" % name, out, flags=re.M), name


def test_pure_host_entry_points():
    # the host-only helpers run without a GPU
    from paper_2605_20816_gb300 import pd
    assert pd.pd_K(2, 4) == 15 and pd.pd_K(3, 3) == 20
    assert pd.pd_alpha(2, 2) == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    assert pd.strerror(pd.PD_ELABEL) == "label outside 0..N-1"
