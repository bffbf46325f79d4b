"""Batched ensemble solve: every scene matches its own oracle solve and the single-scene path."""
import numpy as np
import pytest

import scenes
from oracle import operator as oop, solvers as osv
from sph_testutil import lib_build, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _small_ensemble():
    # uneven sizes, different nu and dt, both boundary models and both means
    out = [scenes.couette(0), scenes.lava_box(1, n=10, nu=3.0, dt=2e-4), scenes.random_box(2, nf=400, mu_spread=8.0),
           scenes.couette(3, nx=24, ny=8, nz=12, nu=30.0, dt=3e-4, boundary=scenes.BC_DYNAMIC),
           scenes.lava_box(4, n=14), scenes.periodic_lattice(9, jitter=0.1, seed=5, mu_spread=2.0)]
    out[2].mean = scenes.MEAN_ARITHMETIC
    return out


def test_batch_matches_oracle_per_scene():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    ens = _small_ensemble()
    nbs = [lib_build(s)[0] for s in ens]
    batch = binding.Batch(nbs, [params_for(s) for s in ens])
    bs = [torch.from_numpy(s.b).cuda() for s in ens]
    xs = [torch.from_numpy(s.x0).cuda() for s in ens]
    st, reps = batch.solve(binding.solve_opts(), bs, xs)
    assert st == 0, reps
    info = batch.info()
    assert 0 <= info["variant"] < 8 and info["grid"] > 0 and len(info["tune_ms"]) == 8
    # the whole solve runs as one graph launch (its passes in a conditional WHILE node)
    assert info["graph_mode"] == 2
    # the tuned tile length is one of the candidates, timed for each, and the tile
    # table covers every scene's slices
    assert info["tile_candidates"] == [16, 32, 64] and info["tile_slices"] in info["tile_candidates"]
    assert all(t > 0 for t in info["tile_tune_ms"])
    nsl = [-(-nb.info()[0] // 32) for nb in nbs]
    assert info["ntiles"] == sum(-(-k // info["tile_slices"]) for k in nsl)
    for s, x, rep in zip(ens, xs, reps):
        off, idx, A = oracle_system(s)
        xg = x.cpu().numpy()
        res, _ = oop.true_residual(A, xg, s.b)
        assert rep["status"] == 0 and res <= 1e-6, (s.name, res, rep)
        assert abs(rep["true_rel_res"] - res) <= 1e-9 + 1e-2 * res
    # a second solve from the same guesses reuses the graph and gives the same answer
    xs2 = [torch.from_numpy(s.x0).cuda() for s in ens]
    st2, reps2 = batch.solve(binding.solve_opts(), bs, xs2)
    assert st2 == 0
    for x, x2 in zip(xs, xs2):
        np.testing.assert_array_equal(x.cpu().numpy(), x2.cpu().numpy())
    # the 1e-5 distance to the oracle's solution on a solve to a 1e-7 true residual (a
    # 1e-6 residual bounds the error only to ~kappa * 1e-6 on the stiff boxes)
    xs7 = [torch.from_numpy(s.x0).cuda() for s in ens]
    st7, reps7 = batch.solve(binding.solve_opts(rtol=1e-7), bs, xs7)
    assert st7 == 0, reps7
    for s, x7 in zip(ens, xs7):
        off, idx, A = oracle_system(s)
        x_ref = osv.reference_solution(A, s.b, s.x0)
        assert rel_l2(x7.cpu().numpy(), x_ref) <= 1e-5, s.name
    batch.close()


def test_batch_scene_already_converged_and_zero_rhs():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    ens = [scenes.couette(7), scenes.lava_box(8, n=10)]
    nbs = [lib_build(s)[0] for s in ens]
    batch = binding.Batch(nbs, [params_for(s) for s in ens])
    off, idx, A = oracle_system(ens[0])
    x_exact = osv.reference_solution(A, ens[0].b, ens[0].x0, rtol=1e-14)
    z = np.zeros_like(ens[1].b)
    bs = [torch.from_numpy(ens[0].b).cuda(), torch.from_numpy(z).cuda()]
    xs = [torch.from_numpy(x_exact).cuda(), torch.from_numpy(z).cuda()]
    st, reps = batch.solve(binding.solve_opts(), bs, xs)
    assert st == 0
    assert reps[0]["iters"] == 0 and reps[1]["iters"] == 0
    np.testing.assert_array_equal(xs[1].cpu().numpy(), 0.0)
    batch.close()


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batch_each_tile_length_matches_oracle(tile):
    """A tile length fixed by sph_batch_set_tile (the tuner then keeps it): every scene
    still reaches the 1e-6 true residual the oracle computes, and the batch reports it."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    ens = _small_ensemble()
    nbs = [lib_build(s)[0] for s in ens]
    batch = binding.Batch(nbs, [params_for(s) for s in ens])
    batch.set_tile(tile)
    bs = [torch.from_numpy(s.b).cuda() for s in ens]
    xs = [torch.from_numpy(s.x0).cuda() for s in ens]
    st, reps = batch.solve(binding.solve_opts(), bs, xs)
    assert st == 0, reps
    info = batch.info()
    assert info["tile_slices"] == tile
    for s, x, rep in zip(ens, xs, reps):
        off, idx, A = oracle_system(s)
        res, _ = oop.true_residual(A, x.cpu().numpy(), s.b)
        assert rep["status"] == 0 and res <= 1e-6, (s.name, tile, res, rep)
    lib = binding.load()
    assert lib.sph_batch_set_tile(batch.handle, 24, None) == 1          # not a candidate: invalid
    assert batch.info()["tile_slices"] == tile
    batch.close()

