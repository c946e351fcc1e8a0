"""CPU checks of the C-ABI library: it loads, exports every symbol include/ks.h declares,
and its host-only entry point agrees with the oracle.  No compute call needs a GPU here."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from oracle import ks_oracle as ko
from paper_2106_03872_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ks():
    from paper_2106_03872_gb300 import ks as mod
    if not os.path.exists(mod.LIB_PATH):
        from paper_2106_03872_gb300 import build
        build.build()
    mod.load()
    return mod


def header_symbols():
    text = open(os.path.join(ROOT, "include", "ks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ks_[a-z_0-9]+)\s*\(", text)))


def test_header_symbols_listed_in_binding(ks):
    assert header_symbols() == sorted(ks.EXPORTS)


def test_library_exports_every_declared_symbol(ks):
    lib = ct.CDLL(ks.LIB_PATH)
    for name in header_symbols():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("L,N", [(10.0, 24), (20.0, 64), (30.0, 96), (15.0, 48), (10.0, 32)])
def test_count_gvectors_matches_oracle(ks, L, N):
    cell = ko.Cell(dict(L=L, N=N, ecut=20.0, pos=np.zeros((0, 3)), vloc_depth=0.0, vloc_width=0.8, nproj=1,
                        proj_sigma=0.5, proj_rc=2.0, proj_D=0.5))
    assert ks.count_gvectors(L, N, 20.0) == cell.nG


def test_count_gvectors_rejects_bad_grids(ks):
    for L, N, ecut in [(10.0, 25, 20.0), (10.0, 6, 20.0), (10.0, 256, 20.0), (10.0, 14, 20.0), (40.0, 24, 20.0),
                       (-1.0, 24, 20.0)]:
        with pytest.raises(ks.KsError) as e:
            ks.count_gvectors(L, N, ecut)
        assert e.value.status == ks.KS_ERR_ARG


def test_last_error_is_thread_local_text(ks):
    with pytest.raises(ks.KsError):
        ks.count_gvectors(10.0, 25, 20.0)
    assert b"N=25" in ks.load().ks_last_error()


def test_make_desc_marshals_cell(ks):
    cell = inputs.cell("small")
    d = ks.make_desc(cell, "fp64")
    assert d.N == 24 and d.natoms == 4 and d.nstates == 8 and d.prec == ks.KS_FP64
    assert abs(d.pos[5] - cell["pos"][1, 2]) == 0.0


def test_tensor_core_wait_expiry_reports_cuda_error(ks):
    """The host side of the bounded mbarrier waits: a nonzero error word becomes KS_ERR_CUDA with
    a message; zero is success.  (No kernel is made to time out: the word is what a kernel whose
    wait expired leaves behind.)"""
    lib = ks.load()
    assert lib.ks_tc_status_check(0) == ks.KS_OK
    assert lib.ks_tc_status_check(1) == ks.KS_ERR_CUDA
    assert b"bounded wait expired" in lib.ks_last_error()
