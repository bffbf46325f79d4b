"""Shared helpers of the GPU parity tests: scene -> device tensors -> library calls.

Inputs come from the seeded ``scenes`` generators; expected values only from
``oracle`` (float64, CPU).  Nothing here computes any part of the method.
"""
import numpy as np

import scenes
from oracle import neighbors as onb, operator as oop, solvers as osv


def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def lib_build(scene, max_neighbors=128):
    from paper_2206_14780_gb300 import binding

    return binding.build_for_scene(scene, max_neighbors=max_neighbors)


def params_for(scene, dt=None):
    from paper_2206_14780_gb300 import binding

    return binding.visc_params(scene.dt if dt is None else dt, scene.boundary, scene.mean)


def oracle_system(scene, method="auto"):
    off, idx = onb.build(scene.pos, scene.lo, scene.hi, scene.periodic, scene.h, method,
                         kernel_id=getattr(scene, "kernel", 0))
    return off, idx, oop.assemble(scene, off, idx)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def gpu_solve(nb, scene, opts=None, b=None, x0=None):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    b = scene.b if b is None else b
    x0 = scene.x0 if x0 is None else x0
    bt = torch.from_numpy(np.ascontiguousarray(b, np.float64)).cuda()
    xt = torch.from_numpy(np.ascontiguousarray(x0, np.float64)).cuda()
    rep = nb.solve(params_for(scene), opts or binding.solve_opts(), bt, xt)
    torch.cuda.synchronize()
    return xt.cpu().numpy(), rep


SCENES_SMALL = {
    "couette_dummy": lambda: scenes.couette(0),
    "couette_dynamic": lambda: scenes.couette(1, boundary=scenes.BC_DYNAMIC),
    "random_box_mu_mass": lambda: scenes.random_box(3, nf=400, mu_spread=20.0, mass_spread=0.3),
    "random_box_arith_open": lambda: scenes.random_box(4, nf=300, periodic=(0, 0, 0), mean=scenes.MEAN_ARITHMETIC,
                                                       mu_spread=5.0),
    "lava_box_12": lambda: scenes.lava_box(2, n=12),
    "periodic_lattice": lambda: scenes.periodic_lattice(9, jitter=0.1, mu_spread=3.0, seed=3),
}
