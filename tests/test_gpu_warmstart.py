"""Warm start on the GPU: the dummy-wall closure and the residual training targets
against the float64 oracle, and the trained network's gain over the previous-step
start on held-out problems."""
import json
import os

import numpy as np
import pytest

import scenes
from oracle import mlp as omlp, neighbors as onb, operator as oop, warmstart as ows
from sph_testutil import lib_build, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

SCENES = [lambda: scenes.lava_box(3, n=10), lambda: scenes.couette(2),
          lambda: scenes.couette(5, boundary=scenes.BC_DYNAMIC), lambda: scenes.slope_subset(1, nx=12, ny=8, nz=12)]


def _rough(s, seed):
    rng = np.random.default_rng(seed)
    v = np.array(s.vel, np.float32, copy=True)
    fl = s.ptype == scenes.FLUID
    v[fl, :3] += (0.2 * np.abs(v[fl, :3]).max() + 0.05) * rng.standard_normal((int(fl.sum()), 3)).astype(np.float32)
    return v


def _net_params(seed):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    p["W4"] = p["W4"] * 5.0
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(scale=0.05, size=p[k].shape)
    return omlp.flatten(p).astype(np.float32)


@pytest.mark.parametrize("make", SCENES)
def test_wall_closure_matches_oracle(make):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = make()
    nb, t = lib_build(s)
    v = _rough(s, 1)
    b = torch.from_numpy(s.b).cuda()
    x0 = torch.empty_like(b)
    binding.warm_start(nb, params_for(s), None, torch.from_numpy(v).cuda(), t["ptype"], b, x0)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = oop.assemble(s, off, idx)
    ref = ows.start(A, s.b, v, None, s.ptype, 1.0)
    got = x0.cpu().numpy()
    fl = s.ptype == scenes.FLUID
    np.testing.assert_array_equal(got[fl], v[fl, :3].astype(np.float64))
    assert rel_l2(got[~fl], ref[~fl]) <= 1e-5
    r = s.b - A @ got
    assert np.abs(r[~fl]).max() <= 1e-5 * np.abs(s.b).max() + 1e-5 * np.abs(got).max()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("flags", [2, 3, 0, 1])
@pytest.mark.parametrize("make", SCENES[:2] + SCENES[3:])
def test_residual_targets_match_oracle(make, flags, mode):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = make()
    nb, t = lib_build(s)
    v = _rough(s, 2)
    vt = torch.from_numpy(v).cuda()
    b = torch.from_numpy(s.b).cuda()
    net = binding.Mlp(_net_params(3))
    net.set_mode(mode)
    p = params_for(s)
    feats = torch.empty((s.n, 16), dtype=torch.int16, device="cuda")
    tg = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    mask = torch.empty(s.n, dtype=torch.uint8, device="cuda")
    L = binding.mlp_residual_targets(nb, p, net, vt, t["ptype"], b, feats, tg, mask, flags)
    y = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    net.forward(feats, y)
    f2 = torch.empty_like(feats)
    U = binding.mlp_features(nb, p, vt, f2)
    torch.cuda.synchronize()
    yg = y.cpu().numpy().astype(np.float64)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = oop.assemble(s, off, idx)
    jac, lg = bool(flags & binding.RLOSS_JACOBI), bool(flags & binding.RLOSS_LOG)
    S = ows.shepard_matrix(s, off, idx) if mode else None
    t_ref, _, L_ref = ows.residual_targets(A, s.b, v, yg, s.ptype, U, jac, lg, S)
    fl = s.ptype == scenes.FLUID
    np.testing.assert_array_equal(mask.cpu().numpy(), fl.astype(np.uint8))
    step = tg.cpu().numpy()[:, :3].astype(np.float64) - yg[:, :3]
    step_ref = t_ref - yg[:, :3]
    assert rel_l2(step[fl], step_ref[fl]) <= 2e-3, rel_l2(step[fl], step_ref[fl])
    np.testing.assert_array_equal(tg.cpu().numpy()[~fl], 0.0)
    if lg:
        assert abs(L - L_ref) <= 2e-3, (L, L_ref)
    else:
        assert abs(L - L_ref) <= 2e-3 * abs(L_ref), (L, L_ref)


@pytest.mark.parametrize("make", SCENES)
def test_highpass_start_matches_oracle(make):
    """x0 = v + U (y - S y) on fluid rows (Shepard average S), walls closed."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = make()
    nb, t = lib_build(s)
    v = _rough(s, 4)
    vt = torch.from_numpy(v).cuda()
    b = torch.from_numpy(s.b).cuda()
    net = binding.Mlp(_net_params(5))
    net.set_mode(binding.MLP_HIGHPASS)
    x0 = torch.empty_like(b)
    p = params_for(s)
    binding.warm_start(nb, p, net, vt, t["ptype"], b, x0)
    feats = torch.empty((s.n, 16), dtype=torch.int16, device="cuda")
    U = binding.mlp_features(nb, p, vt, feats)
    y = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    net.forward(feats, y)
    torch.cuda.synchronize()
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = oop.assemble(s, off, idx)
    S = ows.shepard_matrix(s, off, idx)
    ref = ows.start(A, s.b, v, y.cpu().numpy().astype(np.float64), s.ptype, U, S)
    got = x0.cpu().numpy()
    fl = s.ptype == scenes.FLUID
    corr, corr_ref = got[fl] - v[fl, :3], ref[fl] - v[fl, :3]
    assert rel_l2(corr, corr_ref) <= 1e-4, rel_l2(corr, corr_ref)
    assert rel_l2(got[~fl], ref[~fl]) <= 1e-5
    with pytest.raises(binding.SphError):
        net.set_mode(2)


def test_residual_targets_reject_unknown_flags():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(0)
    nb, t = lib_build(s)
    vt = torch.from_numpy(s.vel).cuda()
    b = torch.from_numpy(s.b).cuda()
    feats = torch.empty((s.n, 16), dtype=torch.int16, device="cuda")
    tg = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    mask = torch.empty(s.n, dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.SphError):
        binding.mlp_residual_targets(nb, params_for(s), binding.Mlp(_net_params(0)), vt, t["ptype"], b, feats, tg,
                                     mask, 4)


def test_trained_network_beats_previous_step_start():
    """Held-out problems of the training families (seeds the training never drew):
    fewer BiCGSTAB iterations to the same 1e-6 true residual than x0 = v^n."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding
    from paper_2206_14780_gb300 import train_warmstart as tw

    assert os.path.exists(tw.DEFAULT_WEIGHTS)
    z = np.load(tw.DEFAULT_WEIGHTS)
    net = binding.Mlp(z["params"])
    net.set_mode(int(json.loads(str(z["meta"])).get("mode", 0)) if "meta" in z else 0)
    dev = torch.device("cuda", 0)
    fams = [tw.Family(k, 2000 + j, dev) for j, k in enumerate(["couette", "slope", "box"])]
    rng = np.random.default_rng(2024)
    opts = binding.solve_opts()
    its = {"vn": [], "learned": []}
    for k in range(60):
        fam = fams[k % 3]
        p, vel, bb = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(bb).to(dev)
        x_vn = tw._fluid_x0(fam, bt, vt, "vn")
        x_l = torch.empty_like(bt)
        binding.warm_start(fam.nb, p, net, vt, fam.t["ptype"], bt, x_l)
        for key, x in (("vn", x_vn), ("learned", x_l)):
            rep = fam.nb.solve(p, opts, bt, x)
            assert rep["status"] == 0 and rep["true_rel_res"] <= 1e-6, (key, rep)
            its[key].append(rep["iters"])
    gain = np.mean(its["vn"]) - np.mean(its["learned"])
    assert gain > 0.5, (np.mean(its["vn"]), np.mean(its["learned"]))


def test_learned_start_on_an_unseen_million_particle_box(record_property):
    """The c5 evaluation scale: an unseen 1.16M-particle lava box (seed 11, never drawn in
    training).  Every start reaches the 1e-6 true residual; the iterations from the
    learned start, from v^n and from v^n with the dummy-wall closure are recorded (in
    the test's properties) whatever their order.  What the start is measured to do at
    this scale: it does NOT beat v^n with the wall closure on these boxes (the bench's
    learned leg reports the same comparison on three seeds and the ensemble), so the
    assertion bounds it instead: within 25% of the closure start's iterations."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding
    from paper_2206_14780_gb300 import train_warmstart as tw

    z = np.load(tw.DEFAULT_WEIGHTS)
    net = binding.Mlp(z["params"])
    net.set_mode(int(json.loads(str(z["meta"])).get("mode", 0)) if "meta" in z else 0)
    s = scenes.lava_box(11, n=100)
    nb, t = lib_build(s)
    p = params_for(s)
    vel = torch.from_numpy(s.vel).cuda()
    b = torch.from_numpy(s.b).cuda()
    its = {}
    for key in ("vn", "vn_walls", "learned"):
        x = torch.from_numpy(s.x0).cuda()
        if key == "vn_walls":
            binding.warm_start(nb, p, None, vel, t["ptype"], b, x)
        elif key == "learned":
            binding.warm_start(nb, p, net, vel, t["ptype"], b, x)
        rep = nb.solve(p, binding.solve_opts(), b, x)
        assert rep["status"] == 0 and rep["true_rel_res"] <= 1e-6, (key, rep)
        its[key] = rep["iters"]
        record_property(f"iters_{key}", rep["iters"])
    print("unseen 1.16M box, iterations:", its)
    assert its["learned"] <= 1.25 * its["vn_walls"], its
