"""Neighbour lists from the GPU equal the oracle's sets bit for bit (reading X10)."""
import numpy as np
import pytest

import scenes
from oracle import neighbors as onb
from sph_testutil import SCENES_SMALL, lib_build, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", sorted(SCENES_SMALL))
def test_lists_equal_oracle(name):
    s = SCENES_SMALL[name]()
    nb, _ = lib_build(s)
    off, idx = nb.export()
    off_o, idx_o = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    n, nnz, mc = nb.info()
    assert n == s.n and nnz == len(idx_o) and mc == np.diff(off_o).max()


def test_lists_equal_oracle_slope_subset():
    s = scenes.slope_subset(1, nx=24, ny=12, nz=24)
    nb, _ = lib_build(s)
    off, idx = nb.export()
    off_o, idx_o = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)


def test_pairs_on_the_float_band_edge():
    # pairs whose float32 r^2 lands inside the filter band are decided in float64:
    # build a set with separations straddling 2h at the float32 resolution
    torch_cuda()
    h = np.float32(0.013)
    base = np.float32(0.2)
    seps = np.float32(2 * h) + np.arange(-6, 7, dtype=np.float32) * np.spacing(np.float32(2 * h))
    pos = np.zeros((2 * len(seps), 4), np.float32)
    for k, d in enumerate(seps):
        pos[2 * k, :3] = (base, base + 0.05 * k, base)
        pos[2 * k + 1, :3] = (np.float32(base + d), base + 0.05 * k, base)
    pos[:, 3] = 1e-3
    s = scenes.random_box(0, nf=4)
    s.pos = pos
    s.rho = np.full(len(pos), 1000.0, np.float32)
    s.mu = np.ones(len(pos), np.float32)
    s.ptype = np.zeros(len(pos), np.uint8)
    s.lo, s.hi, s.periodic, s.h = np.zeros(3), np.full(3, 1.0), np.array([0, 0, 0], np.int32), float(h)
    nb, _ = lib_build(s)
    off, idx = nb.export()
    off_o, idx_o = onb.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    assert 0 < len(idx_o) < len(pos)


def test_single_particle_and_errors():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.periodic_lattice(8)
    one = s.copy()
    for k in ("pos", "rho", "mu", "ptype"):
        setattr(one, k, getattr(s, k)[:1].copy())
    nb, _ = lib_build(one)
    off, idx = nb.export()
    assert off.cpu().tolist() == [0, 0] and idx.numel() == 0
    # capacity: 80 lattice neighbours against a cap of 40
    with pytest.raises(binding.SphError) as e:
        lib_build(s, max_neighbors=40)
    assert e.value.status == 3
    # non-finite position
    bad = s.copy()
    bad.pos[5, 1] = np.nan
    with pytest.raises(binding.SphError) as e:
        lib_build(bad)
    assert e.value.status == 4
    # periodic axis shorter than three cells
    short = s.copy()
    short.hi = s.lo + np.array([0.05, 0.08, 0.08])
    with pytest.raises(binding.SphError) as e:
        lib_build(short)
    assert e.value.status == 1
    torch.cuda.synchronize()
