"""CPU checks of the C ABI: the library builds, loads and exports every symbol include/hgf.h
declares; host-only entry points work without a GPU. No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    return hgf.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hgf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgf_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_1803_00005_gb300 import hgf
    decl = declared_symbols()
    assert len(decl) >= 18
    assert sorted(hgf.EXPORTED) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_num_channels_host_only(lib):
    from paper_1803_00005_gb300 import hgf
    from oracle import hgf_oracle as O
    for C in (1, 3):
        for d in (1, 2, 3):
            for basis in ("monomial", "powers"):
                want = O.n_channels(C, d, basis)
                got = hgf.hgf_num_channels(C, d, basis)
                assert got == (want if want <= 19 else 0)
    assert hgf.hgf_num_channels(3, 4) == 0          # n = 34 > 19: unsupported
    assert hgf.hgf_num_channels(1, 9, "powers") == 9


def test_create_fails_cleanly_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.hgf_create(0, ctypes.byref(h)) != 0
    assert lib.hgf_destroy(None) == 0
    assert lib.hgf_guidance_release(None) == 0


def test_null_context_rejected(lib):
    from paper_1803_00005_gb300 import hgf
    assert lib.hgf_aggregate(None, None, None, 0, 1, None, 0, None, None, None) == hgf.HGF_EINVAL
    assert lib.hgf_prepare(None, None, 3, 4, 4, None, None, None) == hgf.HGF_EINVAL
    assert lib.hgf_filter(None, None, None, None, 0, 1, None, 0, None, None, None) == hgf.HGF_EINVAL
