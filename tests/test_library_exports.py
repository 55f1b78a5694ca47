"""The C-ABI library builds, loads and exports every entry point declared in include/qttpdip.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qttpdip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("ccp_assemble", "newton_apply", "qtt_compress", "qtt_inverse", "qtt_apply", "newton_solve",
              "pdip_step", "qtt_round"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1808_02558_gb300 import binding, build

    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    lib = binding.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.SYMBOLS) == set(declared_functions())
