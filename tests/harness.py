"""Shared set-up for the GPU parity tests: the same seeded workload on the
CUDA path (through the C ABI binding) and on the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import model as om
from oracle.stencils import stencil as ostencil


def relerr(a, b, floor=1e-6):
    """||a - b||_inf / max(||b||_inf, floor) (vector fields: over all
    components).  The floor keeps fields that vanish identically (p* or u of
    a uniform lattice, where both sides hold rounding noise of 1e-20) from
    dividing noise by noise; every field of a meaningful run exceeds it."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(float(np.abs(b).max()), floor)
    return float(np.abs(a - b).max() / den)


def gpu_domain(w: W.Workload, precision=None, kernel=None):
    """kernel: None (library's choice), 'generic' or 'bulk' (forced through
    LBM_KERNEL), 'skew' (asserted to be the library's choice), 'aa' (the
    in-place PDF layout on the generic tiles, forced) or 'aa_tiled' (the
    in-place layout on the skewed kernel's tiles, asserted)."""
    import os
    from paper_2401_03041_gb300 import lbm
    old = os.environ.pop("LBM_KERNEL", None)
    if kernel in ("generic", "bulk", "aa"):
        os.environ["LBM_KERNEL"] = "generic" if kernel == "aa" else kernel
    try:
        d = lbm.Domain(w.nx, w.ny, w.nz, precision or w.precision, w.thermal, w.q_phase,
                       layout="aa" if kernel in ("aa", "aa_tiled") else "two_grid")
    finally:
        os.environ.pop("LBM_KERNEL", None)
        if old is not None:
            os.environ["LBM_KERNEL"] = old
    d.set_params(w.params)
    if kernel is not None:
        assert d.kernel_info()["kernel"] == kernel, d.kernel_info()
    if w.sources:
        d.set_heat_sources(w.sources)
    if w.patches is not None:
        p = w.patches
        d.set_heater_patches(p.z, p.sx, p.sy, p.x0, p.y0, p.intensity)
    d.init_droplets(w.droplets)
    return d


def perm_to_oracle(Q):
    """perm[i_lib] = oracle index of the library's direction i."""
    from paper_2401_03041_gb300 import lbm
    c_lib, w_lib = lbm.stencil(Q)
    S = ostencil(Q)
    idx = [next(j for j in range(Q) if tuple(int(v) for v in S.c[j]) == c) for c in c_lib]
    assert np.allclose(np.array(w_lib), S.w[idx], rtol=0, atol=1e-16)
    return np.array(idx)


def gpu_state_in_oracle_order(d, w):
    out = {"h": d.get_pdfs("h")[np.argsort(perm_to_oracle(w.q_phase))],
           "g": d.get_pdfs("g")[np.argsort(perm_to_oracle(27))]}
    if w.thermal.startswith("D3Q"):
        Q = int(w.thermal[3:])
        out["f"] = d.get_pdfs("f")[np.argsort(perm_to_oracle(Q))]
    else:
        out["T"] = d.get_pdfs("T")[0]
    return out


def load_state_into_gpu(d, w, state):
    """Upload an oracle-ordered state (dict h, g, f|T) to the GPU domain."""
    d.set_pdfs("h", state["h"][perm_to_oracle(w.q_phase)])
    d.set_pdfs("g", state["g"][perm_to_oracle(27)])
    if "f" in state:
        d.set_pdfs("f", state["f"][perm_to_oracle(int(w.thermal[3:]))])
    else:
        d.set_pdfs("T", state["T"][None])


def gpu_fields(d):
    f = d.fields(dtype="f64")
    return {k: v.detach().cpu().numpy() for k, v in f.items()}


def ragged_workload(thermal="D3Q7", q_phase=15, walls=True, precision="fp64", shape=(40, 20, 13)):
    """A lattice that spans several 32 x 8 tiles with ragged tails in x and y,
    two moving droplets, heaters, walls at z (or periodic)."""
    p = W.Params(nu_L=0.08, nu_H=0.12, mobility=0.03, xi=4.0, sigma_ref=4e-3,
                 sigma_T=-6e-4, T_ref=0.1, alpha_L=0.04, alpha_H=0.04,
                 walls_z=walls, T_bottom=-0.3, T_top=0.4,
                 grad_T=(0.0, 2e-3, 0.0) if not walls else (1e-3, 0.0, 0.0),
                 grad_T_origin=(20.0, 10.0, 6.0), gravity=(0.0, 0.0, -1e-6))
    drops = [W.Droplet(12.3, 9.1, 6.4, 5.0, 2e-3, -1e-3, 5e-4),
             W.Droplet(33.0, 14.5, 7.0, 4.2, -1e-3, 0.0, 0.0)]
    src = [W.HeatSource(20.0, 5.0, 0.0, 0.05, 6.0), W.HeatSource(35.0, 15.0, 3.0, 0.02, 4.0, 5.0)]
    nx, ny, nz = shape
    return W.Workload(f"ragged_{nx}x{ny}x{nz}", nx, ny, nz, 20, p, drops, src, q_phase=q_phase,
                      thermal=thermal, precision=precision)


def bulk_fits(precision, q_phase, thermal):
    """Whether one of the bulk kernel's shared-memory layouts (three h/f box
    stages, one or two g stages, (phi, T) planes, the role exchange) fits in
    227 KB for this combination: tiles of four rows, else of two."""
    qf = int(thermal[3:]) if thermal.startswith("D3Q") else 0
    nhf = q_phase + qf
    s = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    cols = 32 if s == 8 else 64
    W = cols + 2 * (16 // s)
    rs = 8 if s == 8 else 4
    for rows in (4, 2):
        hfb = -(-W * (rows + 2) * s // 128) * 128
        gb = -(-W * rows * s // 128) * 128
        fixed = 3 * nhf * hfb + 6 * (cols + 2) * (rows + 2) * rs + 8 * cols * rows * rs + 64 + 128
        ring = 2 if fixed + 2 * 27 * gb <= 232448 else 1      # g ring of two stages, else one
        if fixed + ring * 27 * gb <= 232448:
            return True
    return False


def _bulk_rows(precision, q_phase, thermal):
    qf = int(thermal[3:]) if thermal.startswith("D3Q") else 0
    nhf = q_phase + qf
    s = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    cols = 32 if s == 8 else 64
    W = cols + 2 * (16 // s)
    rs = 8 if s == 8 else 4
    for rows in (4, 2):
        hfb = -(-W * (rows + 2) * s // 128) * 128
        gb = -(-W * rows * s // 128) * 128
        fixed = 3 * nhf * hfb + 6 * (cols + 2) * (rows + 2) * rs + 8 * cols * rows * rs + 64 + 128
        ring = 2 if fixed + 2 * 27 * gb <= 232448 else 1
        if fixed + ring * 27 * gb <= 232448:
            return rows, nhf, s, cols, W, rs
    return None


def skew_fits(precision, q_phase, thermal):
    """Whether the skewed kernel's layout (three h/f stages, one or two g
    stages, (phi, T) planes, an exchange of two planes) fits at the bulk
    kernel's tile height."""
    r = _bulk_rows(precision, q_phase, thermal)
    if r is None:
        return False
    rows, nhf, s, cols, W, rs = r
    hfb = -(-W * (rows + 2) * s // 128) * 128
    gb = -(-W * rows * s // 128) * 128
    fixed = 3 * nhf * hfb + 6 * (cols + 2) * (rows + 2) * rs + 16 * cols * rows * rs + 64 + 128
    return fixed + 27 * gb <= 232448


def oracle_for(w):
    return om.build(w)


def droplet_centroids(phi, periodic_xy=True):
    """Per-droplet centroids (sorted), the droplet-tracking rule of the
    design: connected components of phi > 1/2 (merged across the periodic x
    and y faces), phi-weighted means, circular means on the periodic axes,
    cell-centred coordinates.  phi: (nz, ny, nx) array."""
    ndimage = pytest.importorskip("scipy.ndimage")
    lab, n = ndimage.label(phi > 0.5)
    nz, ny, nx = phi.shape
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    if periodic_xy:
        pairs = list(zip(lab[:, :, 0].ravel(), lab[:, :, -1].ravel()))
        pairs += list(zip(lab[:, 0, :].ravel(), lab[:, -1, :].ravel()))
        for a, b in pairs:
            if a and b and find(a) != find(b):
                parent[find(a)] = find(b)
    roots = sorted({find(a) for a in range(1, n + 1)})
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    out = []
    for r in roots:
        mask = np.isin(lab, [a for a in range(1, n + 1) if find(a) == r])
        wgt = phi[mask]
        c = []
        for coord, L in ((x, nx), (y, ny)):
            if periodic_xy:
                th = 2 * np.pi * coord[mask] / L
                ang = np.arctan2((wgt * np.sin(th)).sum(), (wgt * np.cos(th)).sum())
                c.append((ang % (2 * np.pi)) * L / (2 * np.pi))
            else:
                c.append((wgt * coord[mask]).sum() / wgt.sum())
        c.append((wgt * z[mask]).sum() / wgt.sum())
        out.append(c)
    return np.array(sorted(out))
