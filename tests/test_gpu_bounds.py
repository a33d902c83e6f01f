"""The bounds-check build (-DLBM_BOUNDS_CHECK): every computed offset into
the population, index-record, row-word and row-start arrays is checked
before the access, and a miss raises bit 1 of the context's device flag
instead of touching memory.  It stands in for a memory checker on the
streaming of eq. (LBE) over voxel images (Sec. 2.1): tiny ragged lattices
with fluid on every face go through every kernel family
(tests/bounds_cases.py), the flag must stay clear, and every result must be
bitwise that of the normal build (the checks change no arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checked(tmp_path_factory):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import _build

    so = _build.build_bounds_check()
    out = str(tmp_path_factory.mktemp("bounds") / "checked.npz")
    subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), so, out], check=True,
                   timeout=1200)
    return dict(np.load(out))


def test_bounds_flag_stays_clear(checked):
    flags = {k[len("flags__"):]: int(v) for k, v in checked.items() if k.startswith("flags__")}
    assert len(flags) > 100
    bad = {k: v for k, v in flags.items() if v & 2}
    assert not bad, bad
    assert not any(v & 1 for v in flags.values())


def test_checked_build_matches_normal_build(checked):
    sys.path.insert(0, HERE)
    import bounds_cases

    res, flags = bounds_cases.run_cases()
    assert not any(flags.values())
    assert set(res) == {k for k in checked if not k.startswith("flags__")}
    for k, v in res.items():
        assert np.array_equal(v, checked[k], equal_nan=True), k
