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


def _partial_csr(n, rows, nbr_rows):
    """CSR with only the sampled rows' neighbour lists (the other rows empty)."""
    counts = np.zeros(n, np.int64)
    order = np.argsort(rows)
    for k in order:
        counts[rows[k]] = len(nbr_rows[k])
    offsets = np.zeros(n + 1, np.int64)
    offsets[1:] = np.cumsum(counts)
    idx = np.concatenate([nbr_rows[k] for k in order]).astype(np.int32)
    return offsets, idx


def test_slope_full_size_mu_pass_and_solve_on_sampled_rows():
    """The 4.12M-particle Papanastasiou slope (the precision study's scene) at full size:
    the mu pass on sampled fluid rows against the oracle's rheology, the mixed solve with
    the bench's options, and its float64 residual on sampled rows against the oracle's
    row-by-row operator built on the GPU's viscosities."""
    torch = torch_cuda()
    from oracle import rheology as orh
    from paper_2206_14780_gb300 import binding

    s = scenes.slope(0)
    nb, t = lib_build(s)
    vel = torch.from_numpy(s.vel).cuda()
    wv = torch.from_numpy(s.wall_vel).cuda()
    mu = torch.empty(s.n, dtype=torch.float32, device="cuda")
    nb.mu_papanastasiou(vel, wv, *s.rheology, mu, set_handle=True)
    mu_g = mu.cpu().numpy()
    rng = np.random.default_rng(17)
    fl = np.flatnonzero(s.ptype == scenes.FLUID)
    wl = np.flatnonzero(s.ptype == scenes.WALL)
    rows = np.unique(np.concatenate([rng.choice(fl, 40, replace=False), rng.choice(wl, 8, replace=False)]))
    nbr_rows = onb.rows_for(s, rows)
    off, idx = _partial_csr(s.n, rows, nbr_rows)
    mu_ref, _ = orh.mu_pass(s, off, idx)
    rf = rows[s.ptype[rows] == scenes.FLUID]
    assert np.abs(mu_g[rf] - mu_ref[rf]).max() <= 1e-4 * np.abs(mu_ref[rf]).max()
    b = torch.from_numpy(s.b).cuda()
    x = torch.from_numpy(s.x0).cuda()
    p = params_for(s)
    rep = nb.solve(p, binding.solve_opts(), b, x)
    assert rep["status"] == 0 and rep["true_rel_res"] <= 1e-6, rep
    xg = x.cpu().numpy()
    mu64 = mu_g.astype(np.float64)
    r_ref = s.b[rows] - oop.rows_apply(s, rows, nbr_rows, xg, mu=mu64)
    rt = torch.empty_like(x)
    nb.residual(p, x, b, rt)
    r_gpu = rt.cpu().numpy()[rows]
    scale = np.abs(s.b[rows]).sum() + np.abs(oop.rows_apply(s, rows, nbr_rows, np.abs(xg), mu=mu64)).sum()
    assert np.abs(r_gpu - r_ref).max() <= 1e-12 * scale


def test_ensemble_full_size_batched_on_sampled_rows():
    """The 64-scene ensemble (about 9M particles) in one batched solve with the bench's
    options; on the largest, the smallest and a middle scene, sampled rows of b - A x from
    the oracle's row-by-row operator agree with the reported residual level."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    ens = scenes.ensemble(0)
    nbs, bs, xs, ps, ts = [], [], [], [], []
    for s in ens:
        nb, t = lib_build(s)
        t["vel"] = torch.from_numpy(s.vel).cuda()
        nbs.append(nb)
        ts.append(t)
        bs.append(torch.from_numpy(s.b).cuda())
        xs.append(torch.empty_like(bs[-1]))
        ps.append(params_for(s))
    for nb, p, t, b, x in zip(nbs, ps, ts, bs, xs):
        binding.warm_start(nb, p, None, t["vel"], t["ptype"], b, x)
    batch = binding.Batch(nbs, ps)
    st, reps = batch.solve(binding.solve_opts(), bs, xs)
    assert st == 0 and all(r["status"] == 0 and r["true_rel_res"] <= 1e-6 for r in reps), reps
    sizes = np.array([s.n for s in ens])
    pick = [int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2])]
    rng = np.random.default_rng(23)
    for k in pick:
        s = ens[k]
        rows = np.unique(rng.choice(s.n, 16, replace=False))
        nbr_rows = onb.rows_for(s, rows)
        xg = xs[k].cpu().numpy()
        r = s.b[rows] - oop.rows_apply(s, rows, nbr_rows, xg)
        # sampled rows of a solution at a 1e-6 joint residual: no row far above that level
        assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(s.b[rows]) + 1e-12, (k, np.linalg.norm(r))
    batch.close()
