"""lbm_mean_velocity_noalloc: the mean velocity of caller-held populations
with no device allocation (for callers whose device memory belongs to
another allocator, or who cannot take cudaMalloc's synchronisation), checked
against lbm_mean_velocity of a context holding the same state.

Collected last on purpose: a failure here leaves every other result of a
stop-at-first-failure run in place.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_11193_gb300 import geometry, lbm

    lbm.lib()
    return torch, lbm, geometry


def _call(lib, torch, g, mask_dev, dims, F, U_dev):
    rc = lib.lbm_mean_velocity_noalloc(g.data_ptr(), mask_dev.data_ptr(), dims,
                                       np.ascontiguousarray(F, np.float64), U_dev.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return U_dev.cpu().numpy().copy()


def test_noalloc_mean_velocity_matches_context(env):
    torch, lbm, geometry = env
    lib = lbm.lib()
    mask = geometry.sphere_array(24, "bcc", c=0.3)
    F = (1e-5, -2e-6, 3e-6)
    dims = np.array(mask.shape[::-1], np.int32)
    S = lbm.LBMSolver(mask, "D", 0.9, force=F, precision="fp64", layout="ab")
    mask_dev = torch.from_numpy(mask).cuda()
    U_dev = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (25, 40):  # two calls in a row, on two different states
        S.step(steps)
        f = S.get_populations()
        g = torch.from_numpy(np.ascontiguousarray(f - W[:, None, None, None])).cuda()
        got = _call(lib, torch, g, mask_dev, dims, F, U_dev)
        want = S.mean_velocity()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_noalloc_mean_velocity_many_blocks(env):
    """A 100 x 96 x 96 Boolean medium: 3,600 blocks of partials, so the
    finalising block's strided loop over more than 1,024 partials runs."""
    torch, lbm, geometry = env
    lib = lbm.lib()
    mask = geometry.boolean((100, 96, 96), 5, 0.45, seed=77)[0]
    F = (2e-6, 1e-6, -1e-6)
    dims = np.array(mask.shape[::-1], np.int32)
    S = lbm.LBMSolver(mask, "B", 1.0, force=F, precision="fp64", layout="ab")
    mask_dev = torch.from_numpy(mask).cuda()
    U_dev = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (7, 12):
        S.step(steps)
        f = S.get_populations()
        g = torch.from_numpy(np.ascontiguousarray(f - W[:, None, None, None])).cuda()
        got = _call(lib, torch, g, mask_dev, dims, F, U_dev)
        want = S.mean_velocity()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    S.close()


@pytest.mark.parametrize("dims", [(257, 256, 256), (2**31 - 1, 2**31 - 1, 2**31 - 1),
                                  (2**31 - 1, 2**20, 1), (1, 1, 2**24 + 1)])
def test_noalloc_rejects_oversized_lattice(env, dims):
    """Just over 2^24 nodes, and edges whose product would overflow 64 bits
    if it were formed before the check."""
    torch, lbm, _ = env
    lib = lbm.lib()
    dims = np.array(dims, np.int32)
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    m = torch.zeros(1, dtype=torch.uint8, device="cuda")
    rc = lib.lbm_mean_velocity_noalloc(one.data_ptr(), m.data_ptr(), dims,
                                       np.zeros(3), one.data_ptr(), None)
    assert rc == -1
