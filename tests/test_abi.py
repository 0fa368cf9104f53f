"""The C-ABI library builds, loads, and exports every symbol that
include/*.h declares; argument validation that happens before any device
work behaves as documented (no GPU needed)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rdsplit_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def librd():
    from paper_1512_03126_gb300 import build
    build.build()
    from paper_1512_03126_gb300 import rdsplit
    return rdsplit


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["rdsplit_mesh_create", "rdsplit_set_model", "rdsplit_run", "rdsplit_get_counts"]:
        assert n in names


def test_library_exports_every_declared_symbol(librd):
    L = ctypes.CDLL(librd.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_has_the_same_names(librd):
    missing = [n for n in declared_functions() if not hasattr(librd, n)]
    assert not missing, missing


def test_host_validation_without_device_work(librd):
    with pytest.raises(librd.RdsplitError) as e:
        librd.rdsplit_mesh_create(0, np.zeros((0, 4)), np.zeros(0), np.zeros((0, 4)), np.zeros((0, 4)))
    assert e.value.code == librd.RDSPLIT_EINVAL
    assert "n_tets" in librd.rdsplit_last_error()
    with pytest.raises(librd.RdsplitError) as e:
        librd.rdsplit_run(None, 1.0, 1)
    assert e.value.code == librd.RDSPLIT_EINVAL
    rc = librd.lib().rdsplit_set_model(None, 1, None, 0, None, None, None, None, 1.0)
    assert rc == librd.RDSPLIT_EINVAL
