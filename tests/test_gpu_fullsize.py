"""Parity at the full bench size (box workload, 1,157,308 particles), on sampled rows.

The oracle cannot assemble the whole matrix in seconds, so it recomputes sampled
rows one by one (O(N) each): neighbour sets bit for bit, the float32 apply, and
the float64 residual of the GPU solution; the solve runs with the bench's options.
"""
import numpy as np
import pytest

import scenes
from oracle import neighbors as onb, operator as oop
from sph_testutil import lib_build, params_for, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def box():
    torch = torch_cuda()
    s = scenes.lava_box(0, n=100)
    nb, _ = lib_build(s)
    rng = np.random.default_rng(11)
    fl = np.flatnonzero(s.ptype == scenes.FLUID)
    wl = np.flatnonzero(s.ptype == scenes.WALL)
    rows = np.concatenate([rng.choice(fl, 48, replace=False), rng.choice(wl, 16, replace=False),
                           [0, s.n - 1]]).astype(np.int64)
    nbr_rows = onb.rows_for(s, rows)
    return s, nb, rows, nbr_rows


def test_sampled_neighbour_rows_bit_exact(box):
    s, nb, rows, nbr_rows = box
    off, idx = nb.export()
    off = off.cpu().numpy()
    idx = idx.cpu().numpy()
    for b, ref in zip(rows, nbr_rows):
        np.testing.assert_array_equal(idx[off[b]:off[b + 1]], ref)


def test_sampled_apply_rows(box):
    torch = torch_cuda()
    s, nb, rows, nbr_rows = box
    v = np.zeros((s.n, 4), np.float32)
    v[:, :3] = np.random.default_rng(5).normal(size=(s.n, 3))
    vt = torch.from_numpy(v).cuda()
    yt = torch.empty_like(vt)
    nb.apply(params_for(s), vt, yt)
    y = yt.cpu().numpy()[rows, :3].astype(np.float64)
    ref = oop.rows_apply(s, rows, nbr_rows, v[:, :3].astype(np.float64))
    assert np.linalg.norm(y - ref) <= 1e-5 * np.linalg.norm(ref)


def test_full_size_solve_residual_on_sampled_rows(box):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s, nb, rows, nbr_rows = box
    b = torch.from_numpy(s.b).cuda()
    x = torch.from_numpy(s.x0).cuda()
    rep = nb.solve(params_for(s), binding.solve_opts(), b, x)
    assert rep["status"] == 0 and rep["true_rel_res"] <= 1e-6, rep
    xg = x.cpu().numpy()
    r_ref = s.b[rows] - oop.rows_apply(s, rows, nbr_rows, xg)
    rt = torch.empty_like(x)
    nb.residual(params_for(s), x, b, rt)
    r_gpu = rt.cpu().numpy()[rows]
    scale = np.abs(s.b[rows]).sum() + np.abs(oop.rows_apply(s, rows, nbr_rows, np.abs(xg))).sum()
    assert np.abs(r_gpu - r_ref).max() <= 1e-13 * scale
    # the sampled rows carry the same small residual as the whole system
    assert np.linalg.norm(r_ref) / np.linalg.norm(s.b[rows]) <= 2e-5
