"""Worker of the x-slab decomposition test: one process per slab, all on
cuda:0, halo columns exchanged after every step through the library's pack /
unpack kernels, carried between the processes by gloo (host staging).

Each slab is a domain of its own columns plus H halo columns per side,
declared a sub-domain of the whole lattice (lbm_set_subdomain) so that every
position-dependent term sees global positions, and started from the whole
lattice's initial state (lbm_get_pdfs / lbm_set_pdfs).  After every step the
H columns next to each cut go to the neighbour, whose halo they refresh.
Rank 0 also steps the whole lattice and compares the gathered slabs with it.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))


def case_workload(name):
    import workloads as W
    from harness import ragged_workload
    if name == "d3q7_walls_moving":
        w = ragged_workload("D3Q7", 15, walls=True)
        return w.replace(params=W.Params(**dict(w.params.__dict__, wall_u_top=(0.02, -0.01),
                                                theta_bottom=70.0))), 2, "generic"
    if name == "rk4_periodic":
        return ragged_workload("RK4", 15, walls=False), 5, "generic"
    if name == "d3q19_wide_tiled":
        return ragged_workload("D3Q19", 15, walls=True, shape=(160, 24, 13)), 2, "skew"
    raise KeyError(name)


# FP64 slabs against the whole lattice: rounding only (observed <= 5e-16 of
# the field's magnitude after the test's steps)
TOL = 1e-12


def state_names(w):
    return ["h", "g", "f"] if w.thermal.startswith("D3Q") else ["h", "g", "T"]


def run(rank, world, port, name, steps, out_path):
    import numpy as np
    import torch
    import torch.distributed as dist
    from harness import gpu_domain, gpu_fields, relerr
    from paper_2401_03041_gb300 import lbm

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    w, H, kernel = case_workload(name)
    if kernel == "generic":
        os.environ["LBM_KERNEL"] = "generic"
    NX = w.nx
    nown = NX // world
    xoff = rank * nown
    nloc = nown + 2 * H
    whole = gpu_domain(w, kernel=None)
    init = {k: whole.get_pdfs(k) for k in state_names(w)}
    whole.close()
    cols = [(xoff - H + j) % NX for j in range(nloc)]
    loc = lbm.Domain(nloc, w.ny, w.nz, w.precision, w.thermal, w.q_phase)
    loc.set_subdomain(xoff - H, NX)
    loc.set_params(w.params)
    if w.sources:
        loc.set_heat_sources(w.sources)
    for k, v in init.items():
        loc.set_pdfs(k, np.ascontiguousarray(v[..., cols]))
    nb = loc.halo_bytes(H)
    dev = torch.device("cuda", 0)
    send_l = torch.empty(nb, dtype=torch.uint8, device=dev)
    send_r = torch.empty(nb, dtype=torch.uint8, device=dev)
    recv_l = torch.empty(nb, dtype=torch.uint8)
    recv_r = torch.empty(nb, dtype=torch.uint8)
    left, right = (rank - 1) % world, (rank + 1) % world
    for _ in range(steps):
        loc.step(1)
        loc.pack_halo_x(H, H, send_l)            # my first own columns -> left neighbour's right halo
        loc.pack_halo_x(nown, H, send_r)         # my last own columns -> right neighbour's left halo
        torch.cuda.synchronize(dev)
        sl, sr = send_l.cpu(), send_r.cpu()
        reqs = [dist.isend(sl, left, tag=1), dist.isend(sr, right, tag=2),
                dist.irecv(recv_r, right, tag=1), dist.irecv(recv_l, left, tag=2)]
        for q in reqs:
            q.wait()
        loc.unpack_halo_x(nown + H, H, recv_r.to(dev))
        loc.unpack_halo_x(0, H, recv_l.to(dev))
    f = gpu_fields(loc)
    mine = {k: (v[..., H:H + nown] if v.ndim == 3 else v[..., H:H + nown]) for k, v in f.items()}
    for k in state_names(w):
        mine["pdf_" + k] = loc.get_pdfs(k)[..., H:H + nown]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        ref = gpu_domain(w, kernel=None)
        ref.step(steps)
        rf = gpu_fields(ref)
        for k in state_names(w):
            rf["pdf_" + k] = ref.get_pdfs(k)
        # the slabs run the position-aware kernel variant and the whole
        # lattice the default one: the compiler contracts their products into
        # FMAs differently, so they agree to rounding, not bit for bit
        bad = []
        for key, v in rf.items():
            got = np.concatenate([g[key] for g in gathered], axis=-1)
            e = relerr(got, v)
            if not e <= TOL:
                bad.append((key, e))
        with open(out_path, "w") as fh:
            fh.write("ok\n" if not bad else f"mismatch {bad}\n")
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    r, wsz, port, name, steps, out = sys.argv[1:7]
    run(int(r), int(wsz), int(port), name, int(steps), out)
