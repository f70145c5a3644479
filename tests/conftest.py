import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libls")
    config.addinivalue_line("markers", "late(rank): runs after every unmarked test, in increasing rank, so "
                                       "that a run stopping at its first failure has run the others first")


def pytest_collection_modifyitems(session, config, items):
    def key(item):
        # the allocation-free entry point's file comes after everything else, late ones included
        if os.path.basename(str(item.fspath)).startswith("test_zz_"):
            return (2, 0)
        mk = item.get_closest_marker("late")
        if mk is None:
            return (0, 0)
        return (1, mk.args[0] if mk.args else 0)
    items.sort(key=key)  # stable: file and definition order within a group
