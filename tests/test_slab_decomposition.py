"""Slab decomposition of the method on CPU ranks (gloo, world size 2).

The lattice is cut into two x slabs.  Each rank steps the FP64 oracle on
its slab plus H halo layers on each side (the box inside the global
periodic lattice is given by the oracle's origin / global_shape), and after
every step the ranks swap the H interior layers next to each cut (the full
state: h, g and f, or T for the finite-difference solvers).  One step at a
cell reads the state within two cells for the LB solvers (pull streaming
one cell, the phase-field gradient one more) and within five for RK4 (four
stages of one stencil cell each, on velocities whose forcing needs the
gradient one cell further), so H = 5 keeps every interior cell exact.  The
only collective besides the halo swap is the FP64 sum of the diagnostics.

The gathered interior state must equal the undecomposed oracle run bit for
bit (the per-cell arithmetic is the same elementwise sequence either way),
and the all-reduced phi mass and first moments must match its diagnostics.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

H = 5          # halo layers per side
STEPS = 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _workload(thermal):
    from harness import ragged_workload
    return ragged_workload(thermal, 15, walls=True)


def _state_keys(o):
    return ("h", "g", "f") if o.lb_thermal else ("h", "g", "T")


def _swap_halos(o, width, rank, world):
    """Send the H interior layers next to each cut to the neighbour owning
    the other side and fill this slab's halos from what comes back."""
    import torch
    import torch.distributed as dist
    left, right = (rank - 1) % world, (rank + 1) % world
    for k in _state_keys(o):
        a = getattr(o, k)                                    # [..., nz, ny, nx_box], x last
        to_left = torch.from_numpy(np.ascontiguousarray(a[..., H:2 * H]))
        to_right = torch.from_numpy(np.ascontiguousarray(a[..., width:width + H]))
        from_right = torch.empty_like(to_left)
        from_left = torch.empty_like(to_right)
        reqs = [dist.isend(to_left, left, tag=1), dist.isend(to_right, right, tag=2)]
        dist.recv(from_right, right, tag=1)                  # right neighbour's left-edge layers
        dist.recv(from_left, left, tag=2)                    # left neighbour's right-edge layers
        for r in reqs:
            r.wait()
        a[..., width + H:width + 2 * H] = from_right.numpy()
        a[..., 0:H] = from_left.numpy()


def _rank(rank, world, port, thermal, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import model as om
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload(thermal)
        width = w.nx // world
        x0 = rank * width
        o = om.build(w, origin=(x0 - H, 0, 0), shape=(width + 2 * H, w.ny, w.nz))
        for _ in range(STEPS):
            o.step(1)
            _swap_halos(o, width, rank, world)
        inner = {k: getattr(o, k)[..., H:H + width].copy() for k in _state_keys(o)}
        m = o.macro()
        phi = m["phi"][..., H:H + width]
        X, Y, Z = (c[..., H:H + width] for c in (o.X, o.Y, o.Z))
        sums = torch.tensor([phi.sum(), (phi * X).sum(), (phi * Y).sum(), (phi * Z).sum()],
                            dtype=torch.float64)
        dist.all_reduce(sums)
        q.put((rank, x0, inner, sums.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("thermal", ["D3Q7", "RK4"])
def test_two_slabs_equal_the_undecomposed_oracle(thermal):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    from oracle import model as om
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, thermal, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0

    w = _workload(thermal)
    full = om.build(w)
    full.step(STEPS)
    width = w.nx // 2
    for rank, x0, inner, _ in out:
        for k, v in inner.items():
            ref = getattr(full, k)[..., x0:x0 + width]
            assert np.array_equal(v, ref), (thermal, rank, k, float(np.abs(v - ref).max()))
    d = full.diagnostics()
    for _, _, _, sums in out:
        for got, key in zip(sums, ("mass", "mx", "my", "mz")):
            assert abs(got - d[key]) <= 1e-12 * abs(d[key]), (key, got, d[key])
