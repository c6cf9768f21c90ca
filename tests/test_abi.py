"""The C-ABI library loads and exports every entry point declared in
include/trs.h (no GPU needed: nothing is called that touches the device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "trs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(trs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_03952_gb300 import build as B
    B.build()
    from paper_1812_03952_gb300 import trs
    return trs.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("trs_bsr_create", "trs_cpr_setup", "trs_fgmres_solve", "trs_solve_adjoint"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_03952_gb300 import trs
    for s in declared_symbols():
        assert hasattr(lib, s), f"{s} not exported"
    assert set(declared_symbols()) == set(trs.EXPORTS)


def test_no_torch_types_in_header():
    text = open(os.path.join(ROOT, "include", "trs.h")).read()
    assert "torch" not in text.replace("torch.", "") or "at::" not in text
    assert "at::Tensor" not in text


def test_build_targets_sm_103a():
    from paper_1812_03952_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-fmad=false" in B.UNITS["k_setup.cu"]


def test_version_and_error_calls_need_no_gpu(lib):
    assert lib.trs_version().decode().startswith("trs")
    assert isinstance(lib.trs_last_error(), bytes)
