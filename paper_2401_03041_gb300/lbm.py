"""ctypes binding of ``liblbm.so`` (declared in ``include/lbm.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies the device workspace and the CUDA stream.
If the library is missing the import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Iterable, Optional, Sequence

from . import build as _build

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
          -4: "LBM_ERR_STATE", -5: "LBM_ERR_NONFINITE", -6: "LBM_ERR_TIMEOUT",
          -7: "LBM_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "fp16": 2}
THERMAL = {"D3Q7": 0, "D3Q15": 1, "D3Q19": 2, "D3Q27": 3, "RK2": 4, "RK4": 5}
FIELD_PHI, FIELD_U, FIELD_P, FIELD_T = 1, 2, 4, 8
LAYOUT = {"two_grid": 0, "aa": 1}

# Every symbol include/lbm.h declares.
SYMBOLS = ("lbm_default_params", "lbm_workspace_bytes", "lbm_create_domain",
           "lbm_workspace_bytes_layout", "lbm_create_domain_layout",
           "lbm_halo_bytes", "lbm_pack_halo_x", "lbm_unpack_halo_x", "lbm_set_subdomain",
           "lbm_destroy_domain", "lbm_set_params", "lbm_set_heat_sources",
           "lbm_set_heater_patches", "lbm_set_heater_field", "lbm_init_droplets", "lbm_step",
           "lbm_step_diagnostics", "lbm_get_diagnostics", "lbm_get_fields",
           "lbm_get_pdfs", "lbm_set_pdfs", "lbm_get_level", "lbm_synchronize",
           "lbm_stencil", "lbm_kernel_info", "lbm_profile_steps", "lbm_profile_read",
           "lbm_field_moments", "lbm_adjoint_run", "lbm_adjoint_step",
           "lbm_state_bytes", "lbm_save_state", "lbm_load_state",
           "lbm_last_error", "lbm_version")


class Params(ctypes.Structure):
    _fields_ = [("nu_L", ctypes.c_double), ("nu_H", ctypes.c_double),
                ("rho_L", ctypes.c_double), ("rho_H", ctypes.c_double),
                ("mobility", ctypes.c_double), ("xi", ctypes.c_double),
                ("sigma_ref", ctypes.c_double), ("sigma_T", ctypes.c_double),
                ("T_ref", ctypes.c_double), ("alpha_L", ctypes.c_double),
                ("alpha_H", ctypes.c_double), ("gravity", ctypes.c_double * 3),
                ("walls_z", ctypes.c_int32), ("T_bottom", ctypes.c_double),
                ("T_top", ctypes.c_double), ("grad_T", ctypes.c_double * 3),
                ("grad_T_origin", ctypes.c_double * 3), ("eps_n", ctypes.c_double),
                ("omega_high", ctypes.c_double), ("rk_isotropic_fd", ctypes.c_int32),
                ("T_bottom_amp", ctypes.c_double), ("T_bottom_waves", ctypes.c_int32),
                ("wall_u_bottom", ctypes.c_double * 2), ("wall_u_top", ctypes.c_double * 2),
                ("theta_bottom", ctypes.c_double), ("theta_top", ctypes.c_double),
                ("cp_L", ctypes.c_double), ("cp_H", ctypes.c_double)]


class HeatSource(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("x", "y", "z", "Q", "w", "d")]


class Droplet(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("cx", "cy", "cz", "R", "ux", "uy", "uz")]


class Diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("heat", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("mx", ctypes.c_double),
                ("my", ctypes.c_double), ("mz", ctypes.c_double),
                ("level", ctypes.c_int64), ("nonfinite", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k in ("mass", "heat", "kinetic", "mx", "my", "mz", "level")}
        d["nonfinite"] = bool(self.nonfinite)
        m = self.mass
        d["centroid"] = (self.mx / m, self.my / m, self.mz / m) if m else (0.0, 0.0, 0.0)
        return d


class LBMError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} -> {STATUS.get(status, status)}: {msg}")
        self.status = status


_LIB = None


def library_path() -> str:
    """The in-tree library, or the file named by LBM_LIBRARY (an alternative
    build of the same sources)."""
    return os.environ.get("LBM_LIBRARY") or _build.LIB


def lib():
    """Load liblbm.so (built in-tree by ``build.build()``); raise if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2401_03041_gb300.build.build()")
    L = ctypes.CDLL(path)
    c_int, c_dbl, vp, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "lbm_default_params": (None, [P(Params)]),
        "lbm_workspace_bytes": (sz, [c_int, c_int, c_int, c_int, c_int, c_int]),
        "lbm_create_domain": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, vp, vp, sz, P(vp)]),
        "lbm_workspace_bytes_layout": (sz, [c_int, c_int, c_int, c_int, c_int, c_int, c_int]),
        "lbm_halo_bytes": (sz, [vp, c_int]),
        "lbm_set_subdomain": (c_int, [vp, c_int, c_int]),
        "lbm_pack_halo_x": (c_int, [vp, c_int, c_int, vp]),
        "lbm_unpack_halo_x": (c_int, [vp, c_int, c_int, vp]),
        "lbm_create_domain_layout": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, c_int, vp, vp, sz,
                                             P(vp)]),
        "lbm_destroy_domain": (c_int, [vp]),
        "lbm_set_params": (c_int, [vp, P(Params)]),
        "lbm_set_heat_sources": (c_int, [vp, c_int, P(HeatSource)]),
        "lbm_set_heater_patches": (c_int, [vp, c_int, c_int, c_int, c_int, P(ctypes.c_int32),
                                           P(ctypes.c_int32), P(c_dbl)]),
        "lbm_set_heater_field": (c_int, [vp, vp, c_int]),
        "lbm_init_droplets": (c_int, [vp, c_int, P(Droplet)]),
        "lbm_step": (c_int, [vp, c_int]),
        "lbm_step_diagnostics": (c_int, [vp, c_int, P(Diag)]),
        "lbm_get_diagnostics": (c_int, [vp, P(Diag)]),
        "lbm_get_fields": (c_int, [vp, ctypes.c_uint, vp, c_int, c_int]),
        "lbm_get_pdfs": (c_int, [vp, c_int, vp]),
        "lbm_set_pdfs": (c_int, [vp, c_int, vp]),
        "lbm_get_level": (c_int, [vp, P(ctypes.c_int64)]),
        "lbm_synchronize": (c_int, [vp, c_int]),
        "lbm_stencil": (c_int, [c_int, P(ctypes.c_int32), P(c_dbl)]),
        "lbm_kernel_info": (c_int, [vp, P(ctypes.c_int32)]),
        "lbm_profile_steps": (c_int, [vp, c_int]),
        "lbm_profile_read": (c_int, [vp, P(c_dbl), P(ctypes.c_int32)]),
        "lbm_field_moments": (c_int, [vp, c_int, c_int, c_int, c_int, vp, P(c_dbl)]),
        "lbm_adjoint_run": (c_int, [vp, c_int, c_int, P(c_dbl), c_dbl, P(c_dbl), P(c_dbl)]),
        "lbm_adjoint_step": (c_int, [vp, vp, vp, c_dbl]),
        "lbm_state_bytes": (sz, [vp]),
        "lbm_save_state": (c_int, [vp, vp, sz]),
        "lbm_load_state": (c_int, [vp, vp, sz]),
        "lbm_last_error": (ctypes.c_char_p, []),
        "lbm_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _check(fn: str, status: int):
    if status != LBM_OK:
        raise LBMError(fn, status, lib().lbm_last_error().decode())


def default_params() -> Params:
    p = Params()
    lib().lbm_default_params(ctypes.byref(p))
    return p


def make_params(src=None, **kw) -> Params:
    """Params from the library defaults, overridden by the attributes of
    ``src`` (any object with matching attribute names) and by keywords."""
    p = default_params()
    items = {}
    if src is not None:
        for name, _ in Params._fields_:
            if hasattr(src, name):
                items[name] = getattr(src, name)
    items.update(kw)
    for name, val in items.items():
        if name in ("gravity", "grad_T", "grad_T_origin", "wall_u_bottom", "wall_u_top"):
            getattr(p, name)[:] = [float(v) for v in val]
        elif name in ("walls_z", "rk_isotropic_fd"):
            setattr(p, name, int(bool(val)))
        elif name == "T_bottom_waves":
            setattr(p, name, int(val))
        else:
            setattr(p, name, float(val))
    return p


def field_moments(field, stream=None):
    """FP64 (sum psi, sum psi x, sum psi y, sum psi z) of one contiguous CUDA
    tensor shaped [nz, ny, nx] (leading dimensions of size 1 allowed; float64
    or float32), through the allocation-free entry point; ``stream`` is a
    torch stream on the field's device (default: that device's current
    stream).  The call runs with the field's device current."""
    import torch
    if not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous CUDA tensor")
    if field.dtype not in (torch.float64, torch.float32):
        raise ValueError("field must be float64 or float32")
    if field.dim() < 3 or any(s != 1 for s in field.shape[:-3]):
        raise ValueError("field must be shaped [nz, ny, nx] (leading dimensions of size 1 only)")
    nz, ny, nx = field.shape[-3:]
    with torch.cuda.device(field.device):
        st = stream if stream is not None else torch.cuda.current_stream(field.device)
        if st.device != field.device:
            raise ValueError("stream must belong to the field's device")
        out = (ctypes.c_double * 4)()
        _check("lbm_field_moments", lib().lbm_field_moments(
            ctypes.c_void_p(field.data_ptr()), 0 if field.dtype == torch.float64 else 1,
            int(nx), int(ny), int(nz), ctypes.c_void_p(st.cuda_stream), out))
    return tuple(out)


def stencil(Q: int):
    """(c, w) of the library's stencil Q: lists of (cx, cy, cz) and weights."""
    c = (ctypes.c_int32 * (3 * Q))()
    w = (ctypes.c_double * Q)()
    _check("lbm_stencil", lib().lbm_stencil(Q, c, w))
    return [tuple(c[3 * i:3 * i + 3]) for i in range(Q)], list(w)


class Domain:
    """One lattice on the current CUDA device (see include/lbm.h).

    The device workspace is a torch uint8 tensor; kernels run on ``stream``
    (default: torch's current stream)."""

    def __init__(self, nx, ny, nz, precision="fp64", thermal="D3Q7", q_phase=15,
                 stream=None, device=None, layout="two_grid"):
        import torch
        L = lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.precision, self.thermal, self.q_phase = precision, thermal, int(q_phase)
        self.layout = layout
        lay = LAYOUT[layout]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = L.lbm_workspace_bytes_layout(self.nx, self.ny, self.nz, PRECISION[precision],
                                              THERMAL[thermal], self.q_phase, lay)
        if nbytes == 0:
            raise LBMError("lbm_workspace_bytes", -1, "invalid domain description")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check("lbm_create_domain_layout",
               L.lbm_create_domain_layout(self.nx, self.ny, self.nz, PRECISION[precision],
                                          THERMAL[thermal], self.q_phase, lay,
                                          ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                          ctypes.byref(h)))
        self._h = h
        self._npatch = 0

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check("lbm_destroy_domain", lib().lbm_destroy_domain(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- setup
    def set_params(self, src=None, **kw):
        p = make_params(src, **kw)
        _check("lbm_set_params", lib().lbm_set_params(self._h, ctypes.byref(p)))

    def set_heat_sources(self, sources: Sequence):
        arr = (HeatSource * max(1, len(sources)))()
        for k, s in enumerate(sources):
            d = getattr(s, "d", math.inf)
            arr[k] = HeatSource(s.x, s.y, s.z, s.Q, s.w, -1.0 if not math.isfinite(d) else d)
        _check("lbm_set_heat_sources", lib().lbm_set_heat_sources(self._h, len(sources), arr))

    def set_heater_patches(self, z, sx, sy, x0, y0, intensity):
        n = len(intensity)
        X = (ctypes.c_int32 * max(1, n))(*x0)
        Y = (ctypes.c_int32 * max(1, n))(*y0)
        I = (ctypes.c_double * max(1, n))(*[float(v) for v in intensity])
        _check("lbm_set_heater_patches",
               lib().lbm_set_heater_patches(self._h, int(z), int(sx), int(sy), n, X, Y, I))
        self._npatch = n

    def set_heater_field(self, q):
        """Per-cell heat-source density added to q_T: a contiguous float64 or
        float32 CUDA tensor of nx * ny * nz elements ([z][y][x]), or None to
        remove it.  The domain keeps a reference, so the tensor stays alive
        while steps read it; change it only between synchronised steps."""
        import torch
        if q is None:
            _check("lbm_set_heater_field", lib().lbm_set_heater_field(self._h, None, 0))
            self._qfield = None
            return
        if not q.is_cuda or not q.is_contiguous() or q.numel() != self.nx * self.ny * self.nz:
            raise ValueError("heater field must be a contiguous CUDA tensor of nx*ny*nz elements")
        dt = {torch.float64: 0, torch.float32: 1}.get(q.dtype)
        if dt is None:
            raise ValueError("heater field must be float64 or float32")
        _check("lbm_set_heater_field", lib().lbm_set_heater_field(self._h, ctypes.c_void_p(q.data_ptr()), dt))
        self._qfield = q

    def init_droplets(self, droplets: Iterable):
        ds = list(droplets)
        arr = (Droplet * max(1, len(ds)))()
        for k, d in enumerate(ds):
            arr[k] = Droplet(d.cx, d.cy, d.cz, d.R, getattr(d, "ux", 0.0),
                             getattr(d, "uy", 0.0), getattr(d, "uz", 0.0))
        _check("lbm_init_droplets", lib().lbm_init_droplets(self._h, len(ds), arr))

    # -------------------------------------------------------------- run
    def step(self, n: int = 1):
        _check("lbm_step", lib().lbm_step(self._h, int(n)))

    def step_diagnostics(self, n: int = 1) -> dict:
        d = Diag()
        _check("lbm_step_diagnostics", lib().lbm_step_diagnostics(self._h, int(n), ctypes.byref(d)))
        return d.as_dict()

    def diagnostics(self) -> dict:
        d = Diag()
        _check("lbm_get_diagnostics", lib().lbm_get_diagnostics(self._h, ctypes.byref(d)))
        return d.as_dict()

    def level(self) -> int:
        v = ctypes.c_int64()
        _check("lbm_get_level", lib().lbm_get_level(self._h, ctypes.byref(v)))
        return v.value

    def kernel_info(self) -> dict:
        v = (ctypes.c_int32 * 6)()
        _check("lbm_kernel_info", lib().lbm_kernel_info(self._h, v))
        return {"kernel": {0: "generic", 1: "bulk", 2: "skew", 3: "aa", 4: "aa_tiled"}.get(v[0], str(v[0])),
                "grid": (v[1], v[2], v[3]), "zchunk": v[4], "smem_bytes": v[5]}

    def adjoint_run(self, steps: int, ckpt_every: int, target, normal_cap: float = 0.0):
        """Run ``steps`` steps from the current state and return (J, dJ/dI) for
        J = |centroid - target|^2 at the end, I = heater-patch intensities
        (numpy array, one value per patch), by the discrete adjoint
        (``normal_cap`` <= 0: exact; > 0: see lbm_adjoint_run)."""
        import numpy as np
        tgt = (ctypes.c_double * 3)(*[float(v) for v in target])
        J = ctypes.c_double()
        npatch = self._npatch
        g = np.zeros(max(npatch, 1), dtype=np.float64)
        _check("lbm_adjoint_run", lib().lbm_adjoint_run(
            self._h, int(steps), int(ckpt_every), tgt, float(normal_cap), ctypes.byref(J),
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return J.value, g[:npatch]

    def adjoint_step(self, lam, normal_cap: float = 0.0):
        """(d step / d state)^T lam for the current state; lam is a float64
        array of (q_phase + 27 + Q_f) * N values in get_pdfs order (h, g,
        then f for the thermal LB, or the T field, Q_f = 1, for RK2 / RK4)."""
        import numpy as np
        lam_in = np.ascontiguousarray(lam, dtype=np.float64).ravel()
        qf = 1 if self.thermal.startswith("RK") else int(self.thermal[3:])
        want = (self.q_phase + 27 + qf) * self.nx * self.ny * self.nz
        if lam_in.size != want:
            raise ValueError(f"adjoint_step: lam has {lam_in.size} values, the state has {want}")
        out = np.empty_like(lam_in)
        _check("lbm_adjoint_step", lib().lbm_adjoint_step(self._h, ctypes.c_void_p(lam_in.ctypes.data),
                                                          ctypes.c_void_p(out.ctypes.data),
                                                          float(normal_cap)))
        return out

    def set_subdomain(self, x_offset: int, nx_global: int):
        """Local column x is global column (x + x_offset) mod nx_global."""
        _check("lbm_set_subdomain", lib().lbm_set_subdomain(self._h, int(x_offset), int(nx_global)))

    def halo_bytes(self, width: int) -> int:
        """Bytes of the halo buffer of `width` columns (lbm_halo_bytes)."""
        return int(lib().lbm_halo_bytes(self._h, int(width)))

    def pack_halo_x(self, x0: int, width: int, buf):
        """Columns [x0, x0 + width) of the current state into `buf` (a CUDA
        uint8 tensor of halo_bytes(width) bytes), on the domain's stream."""
        if not buf.is_cuda or buf.numel() * buf.element_size() < self.halo_bytes(width):
            raise ValueError("halo buffer must be a CUDA tensor of halo_bytes(width) bytes")
        _check("lbm_pack_halo_x", lib().lbm_pack_halo_x(self._h, int(x0), int(width),
                                                        ctypes.c_void_p(buf.data_ptr())))

    def unpack_halo_x(self, x0: int, width: int, buf):
        """`buf` (as written by pack_halo_x) into columns [x0, x0 + width)."""
        if not buf.is_cuda or buf.numel() * buf.element_size() < self.halo_bytes(width):
            raise ValueError("halo buffer must be a CUDA tensor of halo_bytes(width) bytes")
        _check("lbm_unpack_halo_x", lib().lbm_unpack_halo_x(self._h, int(x0), int(width),
                                                            ctypes.c_void_p(buf.data_ptr())))

    def save_state(self) -> bytes:
        """The current state (PDFs, RK temperature, time level) as bytes."""
        n = lib().lbm_state_bytes(self._h)
        buf = ctypes.create_string_buffer(n)
        _check("lbm_save_state", lib().lbm_save_state(self._h, buf, n))
        return buf.raw

    def load_state(self, state: bytes):
        """Restore a state returned by save_state of a domain of the same kind."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check("lbm_load_state", lib().lbm_load_state(self._h, buf, len(state)))

    def profile_steps(self, enable: bool = True):
        """Bracket each step-kernel launch with CUDA events on the domain's stream."""
        _check("lbm_profile_steps", lib().lbm_profile_steps(self._h, 1 if enable else 0))

    def profile_read(self):
        """(summed step-kernel milliseconds, timed launches) since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_int32()
        _check("lbm_profile_read", lib().lbm_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def synchronize(self, timeout_ms: int = 60000):
        _check("lbm_synchronize", lib().lbm_synchronize(self._h, int(timeout_ms)))

    # -------------------------------------------------------------- output
    def fields(self, mask=FIELD_PHI | FIELD_U | FIELD_P | FIELD_T, dtype="f64", out=None):
        """Macroscopic fields of the current level as a dict of torch tensors
        (device tensors if ``out`` is None: written by the kernel directly)."""
        import torch
        tdt = torch.float64 if dtype == "f64" else torch.float32
        comps = [(FIELD_PHI, "phi", 1), (FIELD_U, "u", 3), (FIELD_P, "p", 1), (FIELD_T, "T", 1)]
        n = sum(c for bit, _, c in comps if mask & bit)
        buf = out if out is not None else torch.empty((n, self.nz, self.ny, self.nx), dtype=tdt,
                                                      device=self.device)
        on_dev = int(buf.is_cuda)
        _check("lbm_get_fields", lib().lbm_get_fields(self._h, mask, ctypes.c_void_p(buf.data_ptr()),
                                                      on_dev, 0 if dtype == "f64" else 1))
        res, k = {}, 0
        for bit, name, c in comps:
            if mask & bit:
                res[name] = buf[k] if c == 1 else buf[k:k + c]
                k += c
        return res

    def get_pdfs(self, which: str):
        """One PDF set as a (Q, nz, ny, nx) float64 numpy array (un-shifted)."""
        import numpy as np
        idx = {"h": 0, "g": 1, "f": 2, "T": 3}[which]
        Q = {"h": self.q_phase, "g": 27, "T": 1}.get(which)
        if which == "f":
            Q = int(self.thermal[3:])
        arr = np.empty((Q, self.nz, self.ny, self.nx), dtype=np.float64)
        _check("lbm_get_pdfs", lib().lbm_get_pdfs(self._h, idx, ctypes.c_void_p(arr.ctypes.data)))
        return arr

    def set_pdfs(self, which: str, values):
        import numpy as np
        idx = {"h": 0, "g": 1, "f": 2, "T": 3}[which]
        arr = np.ascontiguousarray(values, dtype=np.float64)
        _check("lbm_set_pdfs", lib().lbm_set_pdfs(self._h, idx, ctypes.c_void_p(arr.ctypes.data)))


_CAPTURE_FN = None


def capture_objective(intensities, setup, steps: int, ckpt_every: int, target,
                      normal_cap: float = 0.0):
    """J(I) = |droplet centroid after ``steps`` steps - target|^2 as a
    differentiable function of the heater-patch intensities I (a 1-D tensor).

    ``setup(I)`` must return an initialised FP64 :class:`Domain` whose
    heater patches carry the intensities ``I`` (a list of floats).  The
    forward pass runs the steps through ``Domain.adjoint_run``, which also
    computes dJ/dI with the adjoint kernels; backward returns it scaled by the
    incoming gradient.
    """
    import torch
    global _CAPTURE_FN
    if _CAPTURE_FN is None:
        class _Capture(torch.autograd.Function):
            @staticmethod
            def forward(ctx, I, setup_, steps_, ckpt_, target_, cap_):
                d = setup_([float(v) for v in I.detach().cpu().tolist()])
                try:
                    J, g = d.adjoint_run(steps_, ckpt_, target_, cap_)
                finally:
                    d.close()
                ctx.save_for_backward(torch.as_tensor(g, dtype=torch.float64))
                ctx.in_dtype, ctx.in_device = I.dtype, I.device
                return torch.tensor(J, dtype=torch.float64)

            @staticmethod
            def backward(ctx, gJ):
                (g,) = ctx.saved_tensors
                grad = (gJ.detach().to("cpu", torch.float64) * g).to(ctx.in_device, ctx.in_dtype)
                return grad, None, None, None, None, None

        _CAPTURE_FN = _Capture
    return _CAPTURE_FN.apply(intensities, setup, int(steps), int(ckpt_every), tuple(target),
                             float(normal_cap))
