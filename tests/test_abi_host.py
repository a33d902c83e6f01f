"""Host-side checks of the C-ABI library that need no GPU: it builds, loads
and exports every entry point include/lbm.h declares; its Table 2 rates agree
with the oracle's; argument validation rejects bad inputs before any device
work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def L():
    from paper_1902_11193_gb300 import _build, lbm

    _build.build_lbm()
    return lbm


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = _declared("lbm.h")
    assert "lbm_create" in names and "lbm_run_to_convergence" in names
    so = C.CDLL(L._build.LBM_SO)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


@pytest.mark.parametrize("st", ["A", "B", "C", "D", "E", "SRT"])
@pytest.mark.parametrize("tau", [0.55, 0.8, 1.0, 1.6, 2.0])
def test_rates_match_oracle(L, ora, st, tau):
    for lam in (1 / 64, 3 / 16, 3 / 8, 1.0):
        assert np.array_equal(L.rates(st, tau, lam), ora.rates(st, tau, lam))


def test_create_rejects_bad_arguments(L):
    m = np.zeros((4, 4, 4), np.uint8)
    with pytest.raises(L.LBMError) as e:
        L.LBMSolver(m, "B", tau=0.5)
    assert e.value.code == -1
    with pytest.raises(L.LBMError):
        L.LBMSolver(m, "E", tau=1.0, Lambda=0.0)
    bad = m.copy()
    bad[0, 0, 0] = 2
    with pytest.raises(L.LBMError):
        L.LBMSolver(bad, "B", tau=1.0)
    # the mask check runs in blocks of 65536 voxels: bad values on either side
    # of a block boundary and in the ragged last block are all caught
    big = np.zeros((35, 40, 50), np.uint8)  # 70,000 voxels
    for flat, val in ((65535, 2), (65536, 255), (big.size - 1, 3)):
        bad = big.copy()
        bad.reshape(-1)[flat] = val
        with pytest.raises(L.LBMError) as e:
            L.LBMSolver(bad, "B", tau=1.0)
        assert e.value.code == -1
    # masks of 2^24 voxels and more are scanned by several host threads:
    # bad values at the start, across the split and at the end are caught
    huge = np.zeros((256, 256, 256), np.uint8)
    for flat in (0, huge.size // 2 - 1, huge.size // 2, huge.size - 1):
        bad = huge.copy()
        bad.reshape(-1)[flat] = 2
        with pytest.raises(L.LBMError) as e:
            L.LBMSolver(bad, "B", tau=1.0)
        assert e.value.code == -1
    with pytest.raises(L.LBMError):
        L.LBMSolver(m, "B", tau=1.0, block_size=48)
    s = L.rates("B", 1.0)
    s[4] = 2.5
    with pytest.raises(L.LBMError):
        L.LBMSolver(m, rates_=s)
    s = L.rates("B", 1.0)
    s[6] = 0.9  # one rate per moment group
    with pytest.raises(L.LBMError):
        L.LBMSolver(m, rates_=s)


def test_null_handles_are_rejected(L):
    """Calls that need no device reject a null context before touching it."""
    import ctypes as C

    lib = L.lib()
    n = C.c_int64(7)
    assert lib.lbm_convergence_history(None, None, 0, C.byref(n)) == -1 and n.value == 7
    f = C.c_int32(0)
    assert lib.lbm_device_flags(None, C.byref(f)) == -1
    sw, pe = C.c_int64(0), C.c_int64(0)
    assert lib.lbm_batch_schedule_counts(None, C.byref(sw), C.byref(pe)) == -1


def test_strerror_covers_codes(L):
    lib = L.lib()
    for code in range(0, -9, -1):
        assert lib.lbm_strerror(code).decode() != "unknown error"
