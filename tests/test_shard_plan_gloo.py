"""The sharded solve's host side on CPU, with two real processes (gloo, world size 2).

sph_shard_plan (host code of the library, no GPU) partitions the rows of a system
into layer-ordered, slice-padded sub-domains (paper Sec. 7).  Each process here
takes its sub-domain of the oracle's assembled A, finds its halo (the rows
outside it that its own rows reference: the outer edge of Sec. 7.1), receives
the halo values of a vector from the other process, applies its rows of A, and
reduces a dot product as per-layer partials all-gathered and summed in layer
order.  Every owned row of A v and the reduced dot must equal, bit for bit, the
same computation done by one process over the whole system: the partition, the
exchange lists and the combine order are what make the sharded GPU solve
independent of the number of sub-domains.
"""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp

import scenes
from oracle import neighbors as onb, operator as oop

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SLICE = 32


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    s = scenes.couette(3, nx=24, ny=8, nz=8)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = oop.assemble(s, off, idx).tocsr()
    axis = int(np.argmax(np.asarray(s.hi) - np.asarray(s.lo)))
    L = float(s.hi[axis] - s.lo[axis])
    nlayers = int(L // (2.0 * float(s.h)))                  # layers at least 2h thick
    width = L / nlayers
    layer = np.clip(np.floor((s.pos[:, axis].astype(np.float64) - s.lo[axis]) / width), 0, nlayers - 1).astype(np.int32)
    v = np.random.default_rng(7).normal(size=s.n)
    return s, A, layer, nlayers, v


def _plan(layer, nlayers, ranks):
    from paper_2206_14780_gb300 import binding

    return binding.shard_plan(layer, nlayers, ranks)


def _slice_layer_dot(y, virt, layer_first_virt, rows_virt_range):
    """y.y over the virtual rows of [v0, v1): per slice of 32 rows in order, per layer
    the slices in order; returns {layer: partial} for the layers inside the range."""
    v0, v1 = rows_virt_range
    yv = np.zeros(v1 - v0)
    sel = (virt >= v0) & (virt < v1)
    yv[virt[sel] - v0] = y[sel]
    out = {}
    for l in range(len(layer_first_virt) - 1):
        a, b = layer_first_virt[l], layer_first_virt[l + 1]
        if a < v0 or b > v1:
            continue
        slices = [float(np.sum(yv[k - v0:k - v0 + SLICE] ** 2)) for k in range(a, b, SLICE)]
        acc = 0.0
        for sv in slices:
            acc += sv
        out[l] = acc
    return out


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, A, layer, nlayers, v = _system()
        virt, rfl, lfv = _plan(layer, nlayers, world)
        v0, v1 = lfv[rfl[rank]], lfv[rfl[rank + 1]]
        mine = np.flatnonzero((virt >= v0) & (virt < v1))          # original row numbers
        owner_of_row = np.searchsorted(lfv[rfl[1:]], virt, side="right")
        # halo: the non-owned columns of the owned rows
        sub = A[mine]
        cols = np.unique(sub.indices)
        halo = cols[owner_of_row[cols] != rank]
        # what the other rank needs from me: its halo rows that I own (both sides compute it)
        other = 1 - rank
        theirs = np.flatnonzero(owner_of_row == other)
        sub_o = A[theirs]
        cols_o = np.unique(sub_o.indices)
        to_send = cols_o[owner_of_row[cols_o] == rank]
        # the exchange: my owned values of the rows the other rank needs, in row order
        local = np.full(s.n, np.nan)
        local[mine] = v[mine]
        send = torch.from_numpy(np.ascontiguousarray(v[to_send]))
        recv = torch.empty(len(halo), dtype=torch.float64)
        if rank == 0:
            dist.send(send, 1)
            dist.recv(recv, 1)
        else:
            dist.recv(recv, 0)
            dist.send(send, 0)
        local[halo] = recv.numpy()
        assert np.all(np.isfinite(local[cols])), "a referenced column was neither owned nor received"
        y_mine = sub @ np.nan_to_num(local, nan=0.0)
        y = np.zeros(s.n)
        y[mine] = y_mine
        parts = _slice_layer_dot(y, virt, lfv, (v0, v1))
        layer_part = np.zeros(nlayers)
        for l, val in parts.items():
            layer_part[l] = val
        gathered = [torch.zeros(nlayers, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(layer_part))
        allp = np.zeros(nlayers)
        for r in range(world):
            lo_l, hi_l = rfl[r], rfl[r + 1]
            allp[lo_l:hi_l] = gathered[r].numpy()[lo_l:hi_l]
        dot = 0.0
        for l in range(nlayers):                                   # layer order
            dot += allp[l]
        q.put(dict(rank=rank, rows=mine, y=y_mine, dot=dot, halo=halo, owned_layers=(int(rfl[rank]), int(rfl[rank + 1])),
                   v0=int(v0), v1=int(v1)))
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
def test_two_process_apply_and_dot_equal_one_process():
    import multiprocessing as mp

    from paper_2206_14780_gb300 import binding

    binding.load()
    s, A, layer, nlayers, v = _system()
    virt, rfl, lfv = _plan(layer, nlayers, 2)
    # plan invariants: a permutation into padded layers, contiguous layer runs per rank
    assert len(np.unique(virt)) == s.n
    for l in range(nlayers):
        rows = np.flatnonzero(layer == l)
        assert np.array_equal(np.sort(virt[rows]), lfv[l] + np.arange(len(rows)))   # order kept, from the layer start
        assert (lfv[l + 1] - lfv[l]) % SLICE == 0 and lfv[l + 1] - lfv[l] - len(rows) < SLICE
        assert np.all(np.diff(virt[rows]) > 0)
    assert rfl[0] == 0 and rfl[-1] == nlayers and np.all(np.diff(rfl) >= 1)
    n0 = lfv[rfl[1]]
    assert abs(int(np.count_nonzero(virt < n0)) - s.n / 2) <= np.bincount(layer).max()   # balanced to a layer
    # one process: the same rows, the same slice/layer order
    y1 = A @ v
    parts = _slice_layer_dot(y1, virt, lfv, (0, lfv[-1]))
    dot1 = 0.0
    for l in range(nlayers):
        dot1 += parts[l]
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((qu.get(timeout=180) for _ in procs), key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rows = np.concatenate([o["rows"] for o in out])
    assert np.array_equal(np.sort(rows), np.arange(s.n))                # every row owned exactly once
    for o in out:
        np.testing.assert_array_equal(o["y"], y1[o["rows"]])           # bit for bit
        assert o["dot"] == dot1
        assert len(o["halo"]) > 0
        # halo rows sit in the layers next to the rank's own (periodic wrap on x)
        hl = set(layer[o["halo"]].tolist())
        lo_l, hi_l = o["owned_layers"]
        assert hl <= {(lo_l - 1) % nlayers, hi_l % nlayers}


def test_plan_rejects_bad_arguments():
    from paper_2206_14780_gb300 import binding

    binding.load()
    with pytest.raises(binding.SphError):
        binding.shard_plan(np.array([0, 1, 2], np.int32), 3, 4)          # more ranks than layers
    with pytest.raises(binding.SphError):
        binding.shard_plan(np.array([0, 5], np.int32), 3, 1)             # layer out of range
    virt, rfl, lfv = binding.shard_plan(np.array([2, 0, 0, 1], np.int32), 3, 3)
    assert virt.tolist() == [64, 0, 1, 32] and rfl.tolist() == [0, 1, 2, 3] and lfv.tolist() == [0, 32, 64, 96]
