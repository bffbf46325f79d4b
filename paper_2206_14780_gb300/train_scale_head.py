"""Trains the learned preconditioner scale (GPU): the warm-start network's
architecture, evaluated on the same 16 per-particle features, predicting the log of
each dummy-wall row's scale on top of the Jacobi diagonal.

    python -m paper_2206_14780_gb300.train_scale_head --out scale_head_mlp.npz

Target: the closed-form wall scale norm2^-p of sph_wall_row_scale, norm2 = the
squared norm of the row of D^-1 A.  The exponent p is chosen first by solves the
method itself generates: random problems of the training geometries are solved
from v^n (with the dummy-wall closure) under each candidate p, and the p with the
fewest mean iterations is kept.  Then the network is fitted (mean squared error on
the wall rows, Adam, sph_mlp_train_step) to the logs of that scale over many
random draws (viscosity, dt and velocity field redrawn; the wall rows' targets
depend on the geometry, the features on the draw as well).  Everything numeric runs
in the library; this script draws the random problems and moves tensors.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2206_14780_gb300.train_warmstart import Family, _init_params  # noqa: E402

DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "scale_head_mlp.npz")
# training geometries: (family, seed); sizes from 3.2k to 40k particles
GEOMETRIES = [("couette", 0), ("couette", 1), ("couette_big", 2), ("box", 3), ("box", 4), ("box_big", 5),
              ("box_big", 6), ("slope", 7), ("slope_big", 8)]


def _closure_x0(fam, p, vt, bt):
    import torch

    from paper_2206_14780_gb300 import binding

    x = torch.empty_like(bt)
    binding.warm_start(fam.nb, p, None, vt, fam.t["ptype"], bt, x)
    return x


def select_power(fams, powers, draws, seed, dev, log=print):
    """Mean iterations to a 1e-6 true residual under each candidate p (and Jacobi
    alone) over `draws` random problems of the training geometries."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    opts = binding.solve_opts()
    its = {p: [] for p in (0.0,) + tuple(powers)}
    for k in range(draws):
        fam = fams[k % len(fams)]
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(b).to(dev)
        sc = torch.empty(fam.scene.n, dtype=torch.float32, device=dev)
        for pw in its:
            fam.nb.wall_row_scale(p, pw, sc)
            fam.nb.set_row_scale(sc)
            x = _closure_x0(fam, p, vt, bt)
            rep = fam.nb.solve(p, opts, bt, x)
            its[pw].append(rep["iters"] if rep["status"] == 0 else 10 ** 6)
        fam.nb.set_row_scale(None)
    mean = {pw: float(np.mean(v)) for pw, v in its.items()}
    best = min(powers, key=lambda pw: mean[pw])
    log(f"  mean iterations by power: {mean}; chosen p = {best}")
    return best, mean


def generate(fams, power, draws, per_draw, seed, dev, log=print):
    """Features and targets (log s, 0, 0, 0) of per_draw random wall rows of each of
    `draws` random problems."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    F, T = [], []
    t0 = time.time()
    for k in range(draws):
        fam = fams[k % len(fams)]
        s = fam.scene
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        feats = torch.empty((s.n, 16), dtype=torch.int16, device=dev)
        binding.mlp_features(fam.nb, p, vt, feats)
        tgt = torch.empty((s.n, 4), dtype=torch.float32, device=dev)
        mask = torch.empty(s.n, dtype=torch.uint8, device=dev)
        binding.mlp_scale_targets(fam.nb, p, power, tgt, mask)
        walls = torch.nonzero(mask, as_tuple=False).flatten()
        sel = walls[torch.from_numpy(rng.integers(0, walls.numel(), size=per_draw)).to(dev)]
        F.append(feats[sel])
        T.append(tgt[sel])
    log(f"  {draws} draws, {time.time() - t0:.1f} s")
    return torch.cat(F), torch.cat(T), dict(draws=draws, per_draw=per_draw, gen_seconds=time.time() - t0)


def train(feats, targets, steps, batch, lr0, seed, init_seed=0, log=print):
    """Adam on the mean squared error between the network's outputs and (log s, 0, 0)."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    net = binding.Mlp(_init_params(init_seed))
    M = feats.shape[0]
    ones = torch.ones(batch, dtype=torch.uint8, device=feats.device)
    base = float(targets[:, 0].pow(2).mean())
    hist = []
    t0 = time.time()
    for k in range(steps):
        lr = lr0 * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * k / steps)))
        idx = torch.from_numpy(rng.integers(0, M, size=batch)).to(feats.device)
        hist.append(net.train_step(feats[idx].contiguous(), targets[idx].contiguous(), ones, batch, lr))
        if (k + 1) % 1000 == 0:
            log(f"  step {k + 1}: loss {np.mean(hist[-100:]):.4e} (zero-prediction loss {base:.4e})")
    return net, dict(steps=steps, batch=batch, lr0=lr0, final_loss=float(np.mean(hist[-100:])),
                     zero_prediction_loss=base, train_seconds=time.time() - t0)


def evaluate(net, power, n, seed, dev):
    """Held-out geometries (other seeds, a larger box): mean iterations from v^n with the
    dummy-wall closure under Jacobi alone, the closed-form scale and the learned scale."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    fams = [Family(k, 100 + j + seed, dev) for j, k in enumerate(["couette", "box_big", "slope_big"])]
    opts = binding.solve_opts()
    keys = ("jacobi", "closed_form", "learned")
    its = {k: [] for k in keys}
    err = []
    for j in range(n):
        fam = fams[j % len(fams)]
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(b).to(dev)
        sc_c = torch.empty(fam.scene.n, dtype=torch.float32, device=dev)
        sc_l = torch.empty_like(sc_c)
        fam.nb.wall_row_scale(p, power, sc_c)
        binding.mlp_row_scale(fam.nb, p, net, vt, sc_l)
        wall = torch.from_numpy(fam.scene.ptype != 0).to(dev)
        err.append(float((sc_l[wall].log() - sc_c[wall].log()).abs().mean()))
        for key, sc in (("jacobi", None), ("closed_form", sc_c), ("learned", sc_l)):
            fam.nb.set_row_scale(sc)
            x = _closure_x0(fam, p, vt, bt)
            rep = fam.nb.solve(p, opts, bt, x)
            its[key].append(rep["iters"])
        fam.nb.set_row_scale(None)
    return dict(mean_iters={k: float(np.mean(v)) for k, v in its.items()}, mean_abs_log_error=float(np.mean(err)),
                problems=n)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--powers", default="2,3,4")
    ap.add_argument("--select-draws", type=int, default=90)
    ap.add_argument("--draws", type=int, default=2000)
    ap.add_argument("--per-draw", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=32768)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval", type=int, default=60)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args(argv)
    import torch

    from paper_2206_14780_gb300 import binding

    binding.load()
    dev = torch.device("cuda", 0)
    fams = [Family(k, sd, dev) for k, sd in GEOMETRIES]
    powers = tuple(float(x) for x in args.powers.split(","))
    print("choosing the exponent by solves ...", flush=True)
    power, by_power = select_power(fams, powers, args.select_draws, args.seed, dev)
    print(f"generating {args.draws} draws ...", flush=True)
    feats, targets, gstats = generate(fams, power, args.draws, args.per_draw, args.seed + 1, dev)
    print(f"{feats.shape[0]} samples; training {args.steps} steps ...", flush=True)
    net, tstats = train(feats, targets, args.steps, args.batch, args.lr, args.seed + 2)
    ev = evaluate(net, power, args.eval, args.seed, dev)
    print("held-out:", json.dumps(ev), flush=True)
    meta = dict(power=power, iterations_by_power={str(k): v for k, v in by_power.items()},
                generation=gstats, train=tstats, heldout=ev, geometries=GEOMETRIES, seed=args.seed)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, params=net.params(), meta=json.dumps(meta))
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
