"""Trains the warm-start network on problems of the viscous step itself (GPU).

    python -m paper_2206_14780_gb300.train_warmstart --steps 4000 --out warmstart_mlp.npz

Data: three small geometries redrawn every step with random parameters:
plane-Couette slabs, Papanastasiou-slope slabs (viscosity from the mu pass) and
open lava boxes with a mix of smooth and white-noise velocity; viscosity, time
step, amplitude and roughness are drawn log-uniformly over several decades.

Loss: the Jacobi-scaled starting residual the solver would see,
by default log(sum |b - A x0|^2 / sum |b|^2) over the fluid rows of each
problem, x0 = v + U net with the dummy-wall closure (see
sph_mlp_residual_targets for the weighted and linear variants).  Fitting the
solution x* pointwise (mean squared error on x* - v) lowers that error but
leaves its rough part, which A amplifies by up to 1 + 2 dt sum c, so it does
not shorten the solve; the number of iterations to a relative residual grows
with log |r0| / |b|, which is what the default loss measures.  sph_mlp_residual_targets turns L into pseudo-targets
whose mean-squared-error gradient is dL/dparameters, so sph_mlp_train_step
(Adam) does the update.  Everything numeric runs in the library; this script
only draws the random scenes and moves tensors.
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

DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart_mlp.npz")


def _loguniform(rng, lo, hi):
    return math.exp(rng.uniform(math.log(lo), math.log(hi)))


class Family:
    """One fixed geometry whose viscosity, dt and velocity field are redrawn per solve."""

    def __init__(self, kind, seed, dev):
        import torch

        import scenes
        from paper_2206_14780_gb300 import binding

        self.kind = kind
        gauss = kind.endswith("_gauss")      # the truncated Gaussian kernel (4 dummy layers)
        kind = kind[:-6] if gauss else kind
        big = kind.endswith("_big")
        kind = kind[:-4] if big else kind
        self.kind = kind
        kw = dict(kernel=scenes.KERNEL_GAUSSIAN, layers=4) if gauss else {}
        if kind == "couette":
            if gauss:
                self.scene = scenes.couette(seed, nx=40 if big else 20, ny=20 if big else 10, nz=40 if big else 16, **kw)
            else:
                self.scene = scenes.couette(seed, nx=40, ny=20, nz=40) if big else scenes.couette(seed)
        elif kind == "slope":
            self.scene = scenes.slope(seed, nx=32, ny=20, nz=32) if big else scenes.slope(seed, nx=16, ny=10, nz=16)
        else:
            self.scene = scenes.lava_box(seed, n=32 if big else 16, **kw)
        s = self.scene
        self.t = binding.scene_tensors(s, dev)
        self.nb = binding.build_neighbors(self.t["pos"], self.t["rho"], self.t["mu"], self.t["ptype"], s.lo, s.hi,
                                          s.periodic, s.h, max_neighbors=512 if gauss else 128, kernel=s.kernel)
        self.dev = dev
        self.fl = np.flatnonzero(s.ptype == scenes.FLUID)
        self.fl_t = torch.from_numpy(self.fl).to(dev)
        self.torch = torch

    def draw(self, rng):
        """Random right-hand side problem on this geometry: (params, vel[n,4] f32, b[n,3] f64)."""
        import scenes
        from paper_2206_14780_gb300 import binding

        torch = self.torch
        s = self.scene
        P = s.pos[:, :3].astype(np.float64)
        vel = np.zeros((s.n, 4), np.float32)
        if self.kind == "couette":
            nu = _loguniform(rng, 0.1, 1000.0)
            dt = _loguniform(rng, 5e-5, 1e-3)
            U = rng.uniform(0.1, 2.0)
            rough = _loguniform(rng, 1e-3, 1.0)
            H = s.meta["H"]
            vel[:, 0] = U * P[:, 1] / H
            vel[:, :3] += (U * rough * rng.uniform(-1, 1, size=(s.n, 3))).astype(np.float32)
            mu = np.full(s.n, 1000.0 * nu, np.float32)
            self.nb.set_viscosity(torch.from_numpy(mu).to(self.dev))
        elif self.kind == "box":
            nu = _loguniform(rng, 0.1, 100.0)
            dt = _loguniform(rng, 1e-4, 1e-3)
            sigma = _loguniform(rng, 1e-2, 1.0)
            white = rng.uniform(0.0, 1.0)
            L = s.meta["n"] * s.dx
            k = rng.integers(1, 4, size=3) * math.pi / max(L, 1e-9)
            ph = rng.uniform(0, 2 * math.pi, size=3)
            smooth = np.stack([np.sin(k[a] * P[:, (a + 1) % 3] + ph[a]) for a in range(3)], axis=1)
            vel[:, :3] = (sigma * ((1 - white) * smooth + white * rng.standard_normal((s.n, 3)))).astype(np.float32)
            mu = np.full(s.n, 1000.0 * nu, np.float32)
            self.nb.set_viscosity(torch.from_numpy(mu).to(self.dev))
        else:
            dt = _loguniform(rng, 1e-4, 1e-3)
            U = rng.uniform(0.02, 0.2)
            plug = rng.uniform(0.1, 0.5)
            noise = _loguniform(rng, 1e-5, 1e-1)
            H = s.meta["H"]
            y0 = (1 - plug) * H
            yy = np.clip(P[:, 1], 0.0, y0)
            vel[:, 0] = U * (1 - (1 - yy / y0) ** 2) * (1 + noise * rng.standard_normal(s.n))
            vel[:, 1:3] = noise * U * rng.standard_normal((s.n, 2))
            tau0, mu0 = _loguniform(rng, 10.0, 300.0), _loguniform(rng, 1.0, 1e3)
            vt = torch.from_numpy(vel).to(self.dev)
            mu = torch.empty(s.n, dtype=torch.float32, device=self.dev)
            self.nb.mu_papanastasiou(vt, torch.from_numpy(s.wall_vel).to(self.dev), tau0, mu0, 1000.0, mu,
                                     set_handle=True)
        vel[s.ptype != scenes.FLUID, :3] = s.wall_vel[s.ptype != scenes.FLUID, :3]
        b = np.zeros((s.n, 3))
        b[:] = vel[:, :3]
        wall = s.ptype != scenes.FLUID
        b[wall] = 2.0 * s.wall_vel[wall, :3]
        return binding.visc_params(dt, s.boundary, s.mean), vel, b


def _fluid_x0(fam, bt, vt, kind):
    """x0 = 0 or v^n on fluid rows, b on wall rows."""
    fl = fam.fl_t
    x = bt.clone()
    x[fl] = 0.0 if kind == "zero" else vt[fl, :3].double()
    return x


def generate(n_solves, seed, dev, per_solve=256, log=print, families=None):
    """Solve n_solves random problems from v^n to a 1e-6 true residual; keep the
    features and the targets (x* - v^n) / U of per_solve random fluid particles
    of each.  Returns device tensors feats [M,16] (bf16 bits), targets [M,4]."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    fams = [Family(k, j, dev) for j, k in enumerate(families or FAMILIES)]
    opts = binding.solve_opts()
    F, T, its = [], [], []
    t0 = time.time()
    for k in range(n_solves):
        fam = fams[k % len(fams)]
        s = fam.scene
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(b).to(dev)
        x = _fluid_x0(fam, bt, vt, "vn")
        rep = fam.nb.solve(p, opts, bt, x)
        if rep["status"] != 0:
            continue
        its.append(rep["iters"])
        feats = torch.empty((s.n, 16), dtype=torch.int16, device=dev)
        binding.mlp_features(fam.nb, p, vt, feats)
        tgt = torch.empty((s.n, 4), dtype=torch.float32, device=dev)
        mask = torch.empty(s.n, dtype=torch.uint8, device=dev)
        binding.mlp_targets(fam.nb, vt, x, fam.t["ptype"], tgt, mask)
        sel = torch.from_numpy(rng.choice(fam.fl, size=min(per_solve, len(fam.fl)), replace=False)).to(dev)
        F.append(feats[sel])
        T.append(tgt[sel])
        if (k + 1) % 2000 == 0:
            log(f"  {k + 1} solves, {time.time() - t0:.1f} s, mean iterations {np.mean(its):.1f}")
    return torch.cat(F), torch.cat(T), dict(solves=len(its), mean_iters_from_vn=float(np.mean(its)),
                                             gen_seconds=time.time() - t0)


def train_mse(feats, targets, steps, batch, lr0, seed, init_seed=0, log=print):
    """Adam on the mean squared error to (x* - v^n) / U over the generated samples."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    net = binding.Mlp(_init_params(init_seed))
    M = feats.shape[0]
    ones = torch.ones(batch, dtype=torch.uint8, device=feats.device)
    base = float(targets[:, :3].pow(2).sum(1).mean())
    hist = []
    t0 = time.time()
    for k in range(steps):
        lr = lr0 * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * k / steps)))
        idx = torch.from_numpy(rng.integers(0, M, size=batch)).to(feats.device)
        hist.append(net.train_step(feats[idx].contiguous(), targets[idx].contiguous(), ones, batch, lr))
        if (k + 1) % 500 == 0:
            log(f"  step {k + 1}: loss {np.mean(hist[-100:]):.4e} (zero-correction loss {base:.4e})")
    return net, dict(steps=steps, batch=batch, lr0=lr0, loss="mse", final_loss=float(np.mean(hist[-100:])),
                     zero_correction_loss=base, train_seconds=time.time() - t0)


FAMILIES = ["couette", "slope", "box", "couette_big", "slope_big", "box_big"]


def train(steps, scenes_per_step, lr0, seed, init_seed=0, log=print, dev=None, flags=2, mse_data=None,
          mse_batch=32768, mode=0):
    """Adam on the residual loss over freshly drawn problems; with mse_data =
    (feats, targets) every other step is a mean-squared-error step on (x* - v) / U
    instead.  Returns (net, stats)."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    fams = [Family(k, j, dev) for j, k in enumerate(FAMILIES)]
    net = binding.Mlp(_init_params(init_seed))
    net.set_mode(mode)
    ones = torch.ones(mse_batch, dtype=torch.uint8, device=dev)
    bufs = []
    for fam in fams:
        n = fam.scene.n
        bufs.append((torch.empty((n, 16), dtype=torch.int16, device=dev),
                     torch.empty((n, 4), dtype=torch.float32, device=dev),
                     torch.empty(n, dtype=torch.uint8, device=dev)))
    hist, base = [], []
    t0 = time.time()
    for k in range(steps):
        lr = lr0 * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * k / steps)))
        if mse_data is not None and k % 2 == 1:
            idx = torch.from_numpy(rng.integers(0, mse_data[0].shape[0], size=mse_batch)).to(dev)
            net.train_step(mse_data[0][idx].contiguous(), mse_data[1][idx].contiguous(), ones, mse_batch, lr)
            continue
        F, T, M, Ls = [], [], [], []
        for j in rng.choice(len(fams), size=scenes_per_step, replace=True):
            fam = fams[j]
            p, vel, b = fam.draw(rng)
            vt = torch.from_numpy(vel).to(dev)
            bt = torch.from_numpy(b).to(dev)
            f, t, m = bufs[j]
            Ls.append(binding.mlp_residual_targets(fam.nb, p, net, vt, fam.t["ptype"], bt, f, t, m, flags))
            F.append(f.clone())
            T.append(t.clone())
            M.append(m.clone())
        F, T, M = torch.cat(F), torch.cat(T), torch.cat(M)
        net.train_step(F, T, M, int(M.sum()), lr)
        hist.append(float(np.mean(Ls)))
        if (k + 1) % 500 == 0:
            log(f"  step {k + 1}: residual loss {np.mean(hist[-100:]):.4e} ({time.time() - t0:.1f} s)")
    return net, dict(steps=steps, scenes_per_step=scenes_per_step, lr0=lr0, loss_flags=flags, mode=mode,
                     mixed_mse=mse_data is not None,
                     first_loss=float(np.mean(hist[:50])), final_loss=float(np.mean(hist[-100:])),
                     train_seconds=time.time() - t0)


def evaluate(net, n, seed, dev):
    """Held-out problems from the same families (other seeds): mean iterations to a
    1e-6 true residual and mean log10 of the starting residual |b - A x0| / |b|
    from x0 = 0, x0 = v^n (walls b), x0 = v^n with the dummy-wall closure and the
    learned x0 (identical right-hand sides)."""
    import torch

    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(seed)
    fams = [Family(k, 100 + j + seed, dev) for j, k in enumerate(["couette", "slope", "box"])]
    opts = binding.solve_opts()
    keys = ("zero", "vn", "vn_walls", "learned")
    its = {k: [] for k in keys}
    r0 = {k: [] for k in keys}
    per = {f.kind: {k: [] for k in keys} for f in fams}
    per_r0 = {f.kind: {k: [] for k in keys} for f in fams}
    for j in range(n):
        fam = fams[j % len(fams)]
        p, vel, b = fam.draw(rng)
        vt = torch.from_numpy(vel).to(dev)
        bt = torch.from_numpy(b).to(dev)
        x0s = {"zero": _fluid_x0(fam, bt, vt, "zero"), "vn": _fluid_x0(fam, bt, vt, "vn")}
        xw = torch.empty_like(bt)
        binding.warm_start(fam.nb, p, None, vt, fam.t["ptype"], bt, xw)
        x0s["vn_walls"] = xw
        xl = torch.empty_like(bt)
        binding.warm_start(fam.nb, p, net, vt, fam.t["ptype"], bt, xl)
        x0s["learned"] = xl
        nb_ = float(bt.norm())
        for key, x0 in x0s.items():
            r = torch.empty_like(bt)
            fam.nb.residual(p, x0, bt, r)
            r0[key].append(math.log10(max(float(r.norm()) / nb_, 1e-300)))
            per_r0[fam.kind][key].append(r0[key][-1])
            x = x0.clone()
            rep = fam.nb.solve(p, opts, bt, x)
            its[key].append(rep["iters"])
            per[fam.kind][key].append(rep["iters"])
    return dict(mean_iters={k: float(np.mean(v)) for k, v in its.items()},
                mean_log10_r0={k: float(np.mean(v)) for k, v in r0.items()},
                mean_iters_by_family={f: {k: float(np.mean(v)) for k, v in d.items()} for f, d in per.items()},
                mean_log10_r0_by_family={f: {k: round(float(np.mean(v)), 3) for k, v in d.items()}
                                         for f, d in per_r0.items()},
                problems=n)


def _init_params(seed):
    """He-uniform hidden layers, a small output layer, zero biases (flat float32, 9,603 values)."""
    rng = np.random.default_rng(seed)
    parts = []
    for (o, i) in ((64, 16), (64, 64), (64, 64), (3, 64)):
        lim = math.sqrt(3.0 / i) * (0.1 if o == 3 else 1.0)
        parts.append(rng.uniform(-lim, lim, size=(o, i)).ravel())
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--scenes-per-step", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--eval", type=int, default=300)
    ap.add_argument("--loss", choices=["mse", "log", "log-jacobi", "plain", "jacobi", "log-jacobi+mse"],
                    default="mse")
    ap.add_argument("--solves", type=int, default=20000, help="generated solves (mse loss)")
    ap.add_argument("--per-solve", type=int, default=256)
    ap.add_argument("--batch", type=int, default=32768)
    ap.add_argument("--highpass", action="store_true", help="x0 correction y - S y (SPH_MLP_HIGHPASS)")
    ap.add_argument("--families", default=",".join(FAMILIES),
                    help="comma-separated training geometries (couette, slope, box, each optionally _big)")
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args(argv)
    import torch

    from paper_2206_14780_gb300 import binding

    binding.load()
    dev = torch.device("cuda", 0)
    if args.loss == "mse":
        print(f"generating {args.solves} solves ...", flush=True)
        feats, targets, gstats = generate(args.solves, args.seed, dev, args.per_solve,
                                          families=args.families.split(","))
        gstats["families"] = args.families
        print(f"{feats.shape[0]} samples; training {args.steps} steps ...", flush=True)
        net, tstats = train_mse(feats, targets, args.steps, args.batch, args.lr, args.seed + 1)
        tstats["generation"] = gstats
    else:
        mse_data, gstats = None, None
        loss = args.loss
        if loss.endswith("+mse"):
            loss = loss[:-4]
            print(f"generating {args.solves} solves ...", flush=True)
            f, t, gstats = generate(args.solves, args.seed, dev, args.per_solve)
            mse_data = (f, t)
        flags = {"plain": 0, "jacobi": binding.RLOSS_JACOBI, "log": binding.RLOSS_LOG,
                 "log-jacobi": binding.RLOSS_LOG | binding.RLOSS_JACOBI}[loss]
        net, tstats = train(args.steps, args.scenes_per_step, args.lr, args.seed, dev=dev, flags=flags,
                            mse_data=mse_data, mse_batch=args.batch,
                            mode=binding.MLP_HIGHPASS if args.highpass else 0)
        if gstats:
            tstats["generation"] = gstats
    ev = evaluate(net, args.eval, 7, dev)
    print("held-out:", json.dumps(ev), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    meta = dict(train=tstats, seed=args.seed, heldout=ev, mode=int(tstats.get("mode", 0)))
    np.savez(args.out, params=net.params(), meta=json.dumps(meta))
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
