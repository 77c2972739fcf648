"""The C-ABI library loads and exports every symbol include/he.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(he_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    import paper_2305_17341_gb300.builder as b
    return b.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = declared_symbols()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols(built):
    from paper_2305_17341_gb300 import _lib
    names = declared_symbols()
    assert sorted(set(_lib.SIGNATURES)) == names
    _lib.lib()  # resolves every signature


def test_pure_host_entry_points(built):
    from paper_2305_17341_gb300 import _lib
    p = _lib.he_params_default(2)
    assert (p.logN, p.n_q, p.n_p) == (16, 21, 2)
    steps = _lib.he_rot_steps_for_matmul(128, 16, 16, 1 << 15)
    # Table 1 MinRotKeys: Z n1+2n2-2 = 30, T n1+n2-2 = 22 (disjoint), plus one replication step
    assert len(steps) == 30 + 22 + 1
    with pytest.raises(_lib.HeError):
        _lib.he_rot_steps_for_matmul(128, 3, 16, 1 << 15)


def test_rot_steps_match_oracle_schedule(built):
    from oracle.hmm import matmul_rot_steps, transpose_rot_steps
    from paper_2305_17341_gb300 import _lib
    for n, n1z, n1t, S in [(32, 8, 8, 8192), (128, 16, 16, 32768), (16, 4, 2, 512), (8, 8, 8, 64)]:
        assert _lib.he_rot_steps_for_matmul(n, n1z, n1t, S) == matmul_rot_steps(n, n1z, n1t, S)
        assert _lib.he_rot_steps_for_transpose(n, n1z, S) == transpose_rot_steps(n, n1z, S)
