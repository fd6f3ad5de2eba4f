"""The C-ABI library loads and exports every entry point its header declares
(no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(hb_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2202_12477_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hb_mesh_create", "hb_apply_A", "hb_dot", "hb_cg_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2202_12477_gb300 import hb
    assert set(declared_functions()) <= set(hb.exported_names())


def test_u01_matches_definition_on_host(libpath):
    """hb_u01 runs on the host: compare with a direct SplitMix64 evaluation."""
    from paper_2202_12477_gb300 import hb
    M = 2 ** 64 - 1

    def sm(s):
        z = (s + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    for seed, stream, idx in [(0, 1, 0), (5, 2, 12345), (2 ** 63, 1, 7)]:
        s = ((seed ^ ((stream * 0x9E3779B97F4A7C15) & M)) + idx) & M
        assert hb.hb_u01(seed, stream, idx) == (sm(s) >> 11) * 2.0 ** -53
