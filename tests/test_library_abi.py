"""The C-ABI library builds, loads and exports every entry point declared in
include/fmm.h; host-side validation rejects bad arguments before any GPU work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmmlib():
    from paper_2511_15269_gb300 import build, fmm
    build.build()
    return fmm


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(fmmlib):
    names = declared_functions()
    assert len(names) >= 12
    assert set(names) == set(fmmlib.ENTRY_POINTS)
    so = C.CDLL(fmmlib.library_path())
    for name in names:
        assert hasattr(so, name), name


def test_num_levels_matches_oracle(fmmlib, orc):
    for n, leaf, s in [(1, 4, 2), (4096, 64, 2), (1 << 20, 128, 2), (1 << 22, 64, 2), (1000, 8, 1),
                       (12345, 16, 3), (131072, 128, 2)]:
        assert fmmlib.fmm_num_levels(n, leaf, s) == orc.num_levels(n, leaf, s)
    assert fmmlib.fmm_num_levels(0, 64, 2) == -1
    assert fmmlib.fmm_num_levels(100, 2, 2) == -1


def test_build_rejects_bad_arguments_without_gpu(fmmlib):
    L = fmmlib.lib()
    prm = fmmlib.fmm_params(4, 64, 2, 0.5, fmmlib.FMM_FP64, 0)
    out = C.c_void_p()
    fake = C.c_void_p(0x1000)  # never dereferenced: validation fails first
    assert L.fmm_build_tree(None, 10, C.byref(prm), None, C.byref(out)) == fmmlib.FMM_ERR_INVALID_ARG
    assert "pos" in fmmlib.fmm_last_error()
    bad = [fmmlib.fmm_params(0, 64, 2, 0.5, 0, 0), fmmlib.fmm_params(11, 64, 2, 0.5, 0, 0),
           fmmlib.fmm_params(4, 3, 2, 0.5, 0, 0), fmmlib.fmm_params(4, 512, 2, 0.5, 0, 0),
           fmmlib.fmm_params(4, 64, 4, 0.5, 0, 0), fmmlib.fmm_params(4, 64, 2, 1.0, 0, 0),
           fmmlib.fmm_params(4, 64, 2, 0.0, 0, 0), fmmlib.fmm_params(4, 64, 2, 0.5, 7, 0),
           fmmlib.fmm_params(4, 64, 2, 0.5, 0, 8)]
    for b in bad:
        assert L.fmm_build_tree(fake, 100, C.byref(b), None, C.byref(out)) == fmmlib.FMM_ERR_INVALID_ARG
        assert out.value is None
    assert L.fmm_build_tree(fake, 0, C.byref(prm), None, C.byref(out)) == fmmlib.FMM_ERR_INVALID_ARG
    assert L.fmm_eval_potential(None, None, None, None) == fmmlib.FMM_ERR_INVALID_ARG
    assert L.fmm_tree_set_precision(None, 0) == fmmlib.FMM_ERR_INVALID_ARG
    L.fmm_tree_free(None)
