"""Host-side checks of the C-ABI library: it builds, loads, and exports every symbol that
include/ls.h declares (no compute call: these run without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_1408_4495_gb300 import build as B
from paper_1408_4495_gb300 import ls as LS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ls.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:ls_status|void|const char\*)\s+(ls_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(LS.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_structs_match_header_sizes():
    # ls_grid: 6 ints; ls_info: int, int, double, int (padded to 24);
    # ls_nd_stats: 3 ints (+pad) + int64 + 6 doubles
    assert ctypes.sizeof(LS.LsGrid) == 24
    assert ctypes.sizeof(LS.LsInfo) == 24
    assert ctypes.sizeof(LS.LsNdStats) == 72


def test_binding_refuses_without_library(tmp_path):
    saved = LS._lib
    LS._lib = None
    try:
        with pytest.raises(RuntimeError):
            LS.load(str(tmp_path / "missing.so"))
    finally:
        LS._lib = saved
