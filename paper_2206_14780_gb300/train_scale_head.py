"""Trains the learned preconditioner scale (GPU): the warm-start network's
architecture, evaluated on the same 16 per-particle features, predicting the log of
each dummy-wall row's scale on top of the Jacobi diagonal.

    python -m paper_2206_14780_gb300.train_scale_head --out scale_head_mlp.npz

Weighting the dummy-wall rows down against the Jacobi-scaled fluid rows shortens the
inner iteration on stiff systems and lengthens it on mild ones, so the best weight
depends on the problem.  The targets come from solves the method itself generates:
each random problem of the training geometries (viscosity, dt and velocity field
redrawn, so the stiffness dt sum c spans several decades) is solved from v^n with the
dummy-wall closure under each candidate constant wall scale c, and the c with the
fewest iterations becomes the target log c of that problem's wall rows
(sph_mlp_scale_targets).  The network is then fitted to those targets (mean squared
error on the wall rows, Adam through sph_mlp_train_step); feature 10 gives a wall row
the stiffness of its fluid neighbours.  Everything numeric runs in the library; this
script draws the random problems and moves tensors.
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
# training geometries: (family, seed); sizes from 3.2k to 45k particles; _gauss: the truncated
# Gaussian kernel with 4 dummy layers
GEOMETRIES = [("couette", 0), ("couette", 1), ("couette_big", 2), ("box", 3), ("box", 4), ("box_big", 5),
              ("box_big", 6), ("slope", 7), ("slope_big", 8), ("couette_gauss", 9), ("box_gauss", 10),
              ("box_big_gauss", 11)]


def _closure_x0(fam, p, vt, bt):
    import torch

    from paper_2206_14780_gb300 import binding

    x = torch.empty_like(bt)
    binding.warm_start(fam.nb, p, None, vt, fam.t["ptype"], bt, x)
    return x


def generate(fams, cands, draws, per_draw, seed, dev, log=print):
    """For `draws` random problems: iterations under each constant wall scale in cands,
    the best one as the target of per_draw random wall rows (features, targets)."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    opts = binding.solve_opts()
    F, T = [], []
    its = {c: [] for c in cands}
    best_its, chosen = [], []
    t0 = time.time()
    for k in range(draws):
        fam = fams[k % len(fams)]
        s = fam.scene
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(b).to(dev)
        sc = torch.empty(s.n, dtype=torch.float32, device=dev)
        row = {}
        for c in cands:
            fam.nb.wall_row_scale(p, c, 0.0, sc)
            fam.nb.set_row_scale(sc)
            x = _closure_x0(fam, p, vt, bt)
            rep = fam.nb.solve(p, opts, bt, x)
            row[c] = rep["iters"] if rep["status"] == 0 else 10 ** 6
            its[c].append(row[c])
        fam.nb.set_row_scale(None)
        c_best = min(cands, key=lambda c: (row[c], -c))
        best_its.append(row[c_best])
        chosen.append(c_best)
        feats = torch.empty((s.n, 16), dtype=torch.int16, device=dev)
        binding.mlp_features(fam.nb, p, vt, feats)
        tgt = torch.empty((s.n, 4), dtype=torch.float32, device=dev)
        mask = torch.empty(s.n, dtype=torch.uint8, device=dev)
        binding.mlp_scale_targets(fam.nb, p, c_best, 0.0, tgt, mask)
        walls = torch.nonzero(mask, as_tuple=False).flatten()
        sel = walls[torch.from_numpy(rng.integers(0, walls.numel(), size=per_draw)).to(dev)]
        F.append(feats[sel])
        T.append(tgt[sel])
        if (k + 1) % 200 == 0:
            log(f"  {k + 1} problems, {time.time() - t0:.1f} s")
    stats = dict(draws=draws, per_draw=per_draw, solves=draws * len(cands), gen_seconds=time.time() - t0,
                 mean_iters_by_scale={str(c): float(np.mean(v)) for c, v in its.items()},
                 mean_iters_best=float(np.mean(best_its)),
                 chosen={str(c): int(sum(1 for x in chosen if x == c)) for c in cands})
    log(f"  mean iterations by constant wall scale: {stats['mean_iters_by_scale']}; per-problem best "
        f"{stats['mean_iters_best']:.2f}; chosen {stats['chosen']}")
    return torch.cat(F), torch.cat(T), stats


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


def evaluate(net, n, seed, dev, fixed=((1.0, 3.0), (0.125, 0.0))):
    """Held-out geometries (other seeds, a larger box): mean iterations from v^n with the
    dummy-wall closure under Jacobi alone, fixed closed-form wall scales (factor, power)
    and the learned scale."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    fams = [Family(k, 100 + j + seed, dev) for j, k in enumerate(["couette", "box_big", "slope_big", "box",
                                                                   "box_gauss"])]
    opts = binding.solve_opts()
    keys = ["jacobi"] + [f"c{f:g}_p{pw:g}" for f, pw in fixed] + ["learned"]
    its = {k: [] for k in keys}
    for j in range(n):
        fam = fams[j % len(fams)]
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(b).to(dev)
        scales = {"jacobi": None}
        for f, pw in fixed:
            sc = torch.empty(fam.scene.n, dtype=torch.float32, device=dev)
            fam.nb.wall_row_scale(p, f, pw, sc)
            scales[f"c{f:g}_p{pw:g}"] = sc
        sl = torch.empty(fam.scene.n, dtype=torch.float32, device=dev)
        binding.mlp_row_scale(fam.nb, p, net, vt, sl)
        scales["learned"] = sl
        for key, sc in scales.items():
            fam.nb.set_row_scale(sc)
            x = _closure_x0(fam, p, vt, bt)
            rep = fam.nb.solve(p, opts, bt, x)
            its[key].append(rep["iters"])
        fam.nb.set_row_scale(None)
    return dict(mean_iters={k: float(np.mean(v)) for k, v in its.items()}, problems=n)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scales", default="1,0.5,0.25,0.125,0.0625")
    ap.add_argument("--draws", type=int, default=600)
    ap.add_argument("--per-draw", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=32768)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval", type=int, default=80)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args(argv)
    import torch

    from paper_2206_14780_gb300 import binding

    binding.load()
    dev = torch.device("cuda", 0)
    fams = [Family(k, sd, dev) for k, sd in GEOMETRIES]
    cands = tuple(float(x) for x in args.scales.split(","))
    print(f"solving {args.draws} problems under {len(cands)} wall scales ...", flush=True)
    feats, targets, gstats = generate(fams, cands, args.draws, args.per_draw, args.seed, dev)
    print(f"{feats.shape[0]} samples; training {args.steps} steps ...", flush=True)
    net, tstats = train(feats, targets, args.steps, args.batch, args.lr, args.seed + 2)
    ev = evaluate(net, args.eval, args.seed, dev)
    print("held-out:", json.dumps(ev), flush=True)
    meta = dict(target="per-problem best constant wall scale", candidates=list(cands), generation=gstats,
                train=tstats, heldout=ev, geometries=GEOMETRIES, seed=args.seed)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, params=net.params(), meta=json.dumps(meta))
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
