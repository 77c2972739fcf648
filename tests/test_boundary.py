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


def test_rot_steps_for_decomposed_schedules_match_oracle(built):
    """The key set of a product with decomposed Z / T (Sec. 4.2) equals the
    oracle's schedule; Table 3's 128x128 settings included."""
    from oracle.hmm import matmul_rot_steps
    from paper_2305_17341_gb300 import _lib
    for n, n1z, n1t, S, dz, dt in [(16, 4, 4, 2048, 8, 8), (16, 4, 4, 2048, 4, 0), (16, 4, 2, 2048, 0, 4),
                                    (32, 8, 8, 8192, 16, 16), (128, 8, 8, 16384, 64, 32), (128, 16, 16, 16384, 32, 64)]:
        assert _lib.he_rot_steps_for_sched(n, n1z, n1t, S, dz, dt) == matmul_rot_steps(n, n1z, n1t, S, dz, dt)
    assert _lib.he_rot_steps_for_sched(16, 4, 4, 2048) == _lib.he_rot_steps_for_matmul(16, 4, 4, 2048)
    import pytest
    with pytest.raises(_lib.HeError):
        _lib.he_rot_steps_for_sched(16, 4, 4, 2048, 6, 0)   # n1 must divide n'


def test_lazy_schedule_host_matches_oracle_and_paper(built):
    """The library's Lazy Normalization simulation (host code) equals the
    oracle's and reproduces the printed averages 14.5 (l_P = 4) and 13.8
    (l_P = 14) of Sec. 7."""
    import numpy as np
    from oracle.pca import lazy_normalization_schedule
    from paper_2305_17341_gb300 import _lib
    for t in (1, 4, 9, 14):
        assert _lib.he_lazy_normalization_schedule(t) == lazy_normalization_schedule(t)
    assert round(np.mean(_lib.he_lazy_normalization_schedule(4)), 1) == 14.5
    assert round(np.mean(_lib.he_lazy_normalization_schedule(14)), 1) == 13.8
    with pytest.raises(_lib.HeError):
        _lib.he_lazy_normalization_schedule(0)


def test_context_options_need_a_context(built):
    """The per-context switches reject a null context without touching the GPU."""
    from paper_2305_17341_gb300 import _lib
    for fn in (_lib.he_ctx_set_newton_composition, _lib.he_ctx_set_packed_refresh, _lib.he_ctx_set_autotune):
        with pytest.raises(_lib.HeError) as e:
            fn(None, True)
        assert e.value.code == _lib.HE_ERR_ARG
    for fn in (_lib.he_ctx_set_multsum_variant, _lib.he_ctx_set_ntt_variant, _lib.he_ctx_set_ntt_chunk):
        with pytest.raises(_lib.HeError) as e:
            fn(None, 4)
        assert e.value.code == _lib.HE_ERR_ARG
