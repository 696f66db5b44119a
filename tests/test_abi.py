"""The C-ABI library builds, loads without a GPU and exports what
include/muffin.h declares; its host-built tables match the oracle's
independently derived ones."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_08468_gb300.build import build
    build()
    import paper_1905_08468_gb300 as pkg
    return pkg.library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "muffin.h")).read()
    return sorted(set(re.findall(r"MUFFIN_API\s+[\w\s\*]*?\b(muffin_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    from paper_1905_08468_gb300 import native
    assert set(native.SIGNATURES) == set(names)


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.muffin_version()
    assert lib.muffin_last_error()


def test_filter_taps_match_oracle(lib):
    import paper_1905_08468_gb300 as pkg
    from oracle.daubechies import daubechies_lowpass
    for p in range(1, 9):
        assert np.allclose(pkg.filter_taps(p), daubechies_lowpass(p), atol=1e-13), p


def test_dct_table_matches_oracle(lib):
    import paper_1905_08468_gb300 as pkg
    from oracle.spectral import dct_matrix
    for L in (1, 3, 8, 64):
        assert np.allclose(pkg.dct_table(L), dct_matrix(L), atol=1e-14)


def test_invalid_arguments_are_rejected(lib):
    import paper_1905_08468_gb300 as pkg
    with pytest.raises(pkg.MuffinError) as e:
        pkg.filter_taps(9)
    assert e.value.status == 1
    # bad shapes are rejected before any device work
    psf = np.zeros((2, 6, 6), np.float32)
    with pytest.raises(pkg.MuffinError) as e:
        pkg.Plan(6, 2, psf)
    assert e.value.status == 1 and "power of two" in str(e.value)
    with pytest.raises(pkg.MuffinError) as e:
        pkg.Plan(8, 2, np.zeros((2, 8, 8), np.float32), levels=4)
    assert e.value.status == 1


def test_no_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1905_08468_gb300 as pkg
    with pytest.raises(pkg.MuffinError) as e:
        pkg.Plan(8, 2, np.ones((2, 8, 8), np.float32))
    assert e.value.status == 3
