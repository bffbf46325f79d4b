"""The seeded input generators: the particle counts, layouts and right-hand sides the
workloads are stated with, and their determinism (CPU only)."""
import numpy as np
import pytest

import scenes


def _on_lattice_offsets(p, dx, origin):
    """Offset of each position from the nearest cell centre (i + 1/2) dx + origin."""
    q = (p - origin) / dx - 0.5
    return (q - np.rint(q)) * dx


def test_couette_counts_and_rhs():
    s = scenes.couette(0)
    assert (s.n, s.n_fluid) == (3200, 2000)
    nf = s.n_fluid
    assert np.all(s.ptype[:nf] == scenes.FLUID) and np.all(s.ptype[nf:] == scenes.WALL)
    # dummy walls: b = 2 u_w; the top wall moves at (1, 0, 0), the bottom one rests
    top = s.pos[nf:, 1] > s.meta["H"]
    assert top.sum() == 600
    np.testing.assert_array_equal(s.b[nf:][top], np.tile([2.0, 0.0, 0.0], (600, 1)))
    np.testing.assert_array_equal(s.b[nf:][~top], 0.0)
    np.testing.assert_array_equal(s.b[:nf], s.vel[:nf, :3].astype(np.float64))
    d = scenes.couette(0, boundary=scenes.BC_DYNAMIC)
    np.testing.assert_array_equal(d.b[nf:][top], np.tile([1.0, 0.0, 0.0], (600, 1)))
    # linear profile plus at most 1% noise
    prof = s.pos[:nf, 1].astype(np.float64) / s.meta["H"]
    assert np.max(np.abs(s.vel[:nf, 0] - prof)) <= 0.01 + 1e-6
    assert s.h == pytest.approx(0.013, rel=1e-6) and s.pos[0, 3] == np.float32(1000.0 * 0.01 ** 3)


def test_box_counts_jitter_and_walls():
    assert scenes._box_count(100) == 1157308
    s = scenes.lava_box(0, n=12)
    assert s.n == scenes._box_count(12) and s.n_fluid == 12 ** 3
    nf = s.n_fluid
    off_f = _on_lattice_offsets(s.pos[:nf, :3].astype(np.float64), s.dx, 0.0)
    assert np.max(np.abs(off_f)) <= 0.1 * s.dx * (1 + 1e-5)
    assert np.max(np.abs(off_f)) > 0.09 * s.dx               # jittered, up to +-0.1 dx
    off_w = _on_lattice_offsets(s.pos[nf:, :3].astype(np.float64), s.dx, 0.0)
    assert np.max(np.abs(off_w)) <= 1e-6                     # walls never jittered
    # walls at rest, b = v on fluid rows
    np.testing.assert_array_equal(s.b[nf:], 0.0)
    assert abs(float(np.std(s.vel[:nf, :3])) - 0.1) < 0.01


def test_slope_counts_and_viscosity_profile():
    s = scenes.slope_subset(0)
    assert s.n == 50 * 20 * 50 + 50 * 3 * 50 == 57500
    assert 200 * 100 * 200 + 200 * 3 * 200 == 4120000      # the full slope by the same rule
    tau0, mu0, m = s.rheology
    assert (tau0, mu0, m) == (100.0, 1e3, 1000.0)
    nf = s.n_fluid
    # plug above y0 moves rigidly at U (to the noise), sheared layer below
    y = s.pos[:nf, 1].astype(np.float64)
    plug = y > s.meta["y0"] + s.dx
    assert plug.any() and (~plug).any()
    np.testing.assert_allclose(s.vel[:nf][plug, 0], 0.1, rtol=1e-4)
    assert np.all(s.vel[:nf][~plug, 0] <= 0.1 * (1 + 1e-4))
    np.testing.assert_array_equal(s.periodic, [1, 0, 1])


def test_generators_are_seeded():
    a, b, c = scenes.lava_box(3, n=8), scenes.lava_box(3, n=8), scenes.lava_box(4, n=8)
    for f in ("pos", "vel", "b", "x0"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.pos, c.pos) and not np.array_equal(a.vel, c.vel)
    e1 = scenes.ensemble(2, S=4, n_hi=2e4)
    e2 = scenes.ensemble(2, S=4, n_hi=2e4)
    assert [s.n for s in e1] == [s.n for s in e2]
    for s1, s2 in zip(e1, e2):
        np.testing.assert_array_equal(s1.pos, s2.pos)


def test_ensemble_draws():
    ens = scenes.ensemble(1, S=8, n_lo=1e4, n_hi=3e4)
    assert len(ens) == 8
    for k, s in enumerate(ens):
        assert ("couette" if k % 2 == 0 else "lava_box") in s.name
        assert 1.0 <= s.meta["nu"] <= 1e3 and 1e-4 <= s.dt <= 5e-4
        assert 1e4 <= s.meta["target"] <= 3e4
        # the lattice whose total is nearest the drawn count
        if k % 2 == 0:
            ny = int(round(s.meta["H"] / s.dx))
            assert s.n == scenes._couette_count(ny)
            assert all(abs(scenes._couette_count(ny) - s.meta["target"])
                       <= abs(scenes._couette_count(j) - s.meta["target"]) for j in (ny - 1, ny + 1))
        else:
            n = s.meta["n"]
            assert s.n == scenes._box_count(n)
            assert all(abs(scenes._box_count(n) - s.meta["target"])
                       <= abs(scenes._box_count(j) - s.meta["target"]) for j in (n - 1, n + 1))
        np.testing.assert_allclose(s.mu[:s.n_fluid], 1000.0 * s.meta["nu"], rtol=1e-6)
