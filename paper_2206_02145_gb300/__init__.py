"""Python binding of liblbpf.so — the coupled lattice-Boltzmann phase-field
crystal-growth step (Sec. 2 of Tan et al., "Mandelic acid single-crystal
growth: experiments vs numerical simulations") on one GB300.

The functions here carry the C ABI names of ``include/lbpf.h`` and only
marshal arguments through ctypes; every step of the method runs in the CUDA
kernels of the library.  There is no CPU fallback: importing the package
without the built library raises.  Build it with
``python -c "import __graft_entry__ as g; g.build()"``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LBPF_LIB") or os.path.join(_HERE, "_build", "liblbpf.so")

OK, EINVAL, ECUDA, ENOMEM, ESTATE, ENONFINITE, ETIMEDOUT = 0, -1, -2, -3, -4, -5, -6
BC_PERIODIC, BC_INLET_OUTLET, BC_WALL = 0, 1, 2
FP32, FP64, FP16_SHIFTED, BF16_SHIFTED = 0, 1, 2, 3
COLL_BGK, COLL_CHM = 0, 1
FIELD_PHI, FIELD_U, FIELD_RHO, FIELD_UX, FIELD_UY, FIELD_UZ, FIELD_PHI_PREV = (
    1, 2, 4, 8, 16, 32, 64)
FIELD_STATE = 256
NOALLOC_MAX_BLOCKS = 4096
NOALLOC_MAX_NODES = NOALLOC_MAX_BLOCKS * 256 * 64
FIELD_NAMES = ("phi", "U", "rho", "ux", "uy", "uz", "phi_prev")
_STATUS = {OK: "OK", EINVAL: "EINVAL", ECUDA: "ECUDA", ENOMEM: "ENOMEM", ESTATE: "ESTATE",
           ENONFINITE: "ENONFINITE", ETIMEDOUT: "ETIMEDOUT"}


class LbpfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class lbpf_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("flow", ctypes.c_int), ("storage", ctypes.c_int),
        ("fold", ctypes.c_int), ("aniso_literal", ctypes.c_int),
        ("tau_phi0", ctypes.c_double), ("tau_u_liquid", ctypes.c_double),
        ("tau_f", ctypes.c_double), ("w0", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("eps_aniso", ctypes.c_double), ("theta0", ctypes.c_double),
        ("h_drag", ctypes.c_double), ("u_inlet", ctypes.c_double),
        ("u0_inlet", ctypes.c_double), ("body_force", ctypes.c_double * 3),
        ("collision", ctypes.c_int), ("chm_omega_bulk", ctypes.c_double),
        ("chm_omega_high", ctypes.c_double),
    ]


class lbpf_seed(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
                ("radius", ctypes.c_double), ("u0", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("seed", ctypes.c_uint64)]


MAX_FACETS = 12


class lbpf_polygon_seed(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("nfacets", ctypes.c_int),
                ("nx", ctypes.c_double * MAX_FACETS), ("ny", ctypes.c_double * MAX_FACETS),
                ("dist", ctypes.c_double * MAX_FACETS), ("u0", ctypes.c_double),
                ("noise_amp", ctypes.c_double), ("seed", ctypes.c_uint64)]


class lbpf_facets(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("nfacets", ctypes.c_int),
                ("support", ctypes.c_double * MAX_FACETS),
                ("side_cx", ctypes.c_double * MAX_FACETS),
                ("side_cy", ctypes.c_double * MAX_FACETS), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("L", ctypes.c_double * MAX_FACETS),
                ("L_avg", ctypes.c_double), ("Q", ctypes.c_double), ("width", ctypes.c_double),
                ("height", ctypes.c_double), ("aspect", ctypes.c_double)]


class lbpf_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("solute_total", ctypes.c_double),
                ("solute_drift_rel", ctypes.c_double), ("mass_total", ctypes.c_double),
                ("solid_volume", ctypes.c_double), ("r_eq", ctypes.c_double),
                ("iface_pos", ctypes.c_double * 6), ("max_u", ctypes.c_double),
                ("nonfinite", ctypes.c_int64)]


class lbpf_unet_cfg(ctypes.Structure):
    _fields_ = [("in_ch", ctypes.c_int), ("out_ch", ctypes.c_int), ("base_ch", ctypes.c_int),
                ("levels", ctypes.c_int), ("batch", ctypes.c_int), ("height", ctypes.c_int),
                ("width", ctypes.c_int), ("seed", ctypes.c_uint64)]


class lbpf_surrogate_cfg(ctypes.Structure):
    _fields_ = [("steps_per_block", ctypes.c_int), ("judge_every", ctypes.c_int),
                ("drift_tol", ctypes.c_double), ("iface_tol", ctypes.c_double),
                ("iface_budget", ctypes.c_double), ("iface_rel_tol", ctypes.c_double),
                ("shift", ctypes.c_float * 4), ("scale", ctypes.c_float * 4),
                ("res_scale", ctypes.c_float * 4)]


class lbpf_surrogate_report(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_int64), ("surrogate_blocks", ctypes.c_int64),
                ("judged_blocks", ctypes.c_int64), ("fallback_blocks", ctypes.c_int64),
                ("max_drift", ctypes.c_double), ("max_iface_err", ctypes.c_double),
                ("max_iface_est", ctypes.c_double), ("iface_acc", ctypes.c_double),
                ("max_drift_committed", ctypes.c_double)]


EXPORTED = ("lbpf_params_default", "lbpf_create", "lbpf_init_seed", "lbpf_init_fields",
            "lbpf_step", "lbpf_read_fields", "lbpf_state_bytes", "lbpf_write_state",
            "lbpf_diagnostics", "lbpf_set_stream", "lbpf_device_bytes", "lbpf_last_error",
            "lbpf_destroy", "lbpf_field_sums_noalloc", "lbpf_batch_create", "lbpf_batch_step",
            "lbpf_batch_diagnostics", "lbpf_batch_instance", "lbpf_batch_count",
            "lbpf_batch_tuning", "lbpf_batch_last_error", "lbpf_batch_destroy",
            "lbpf_unet_create", "lbpf_unet_forward", "lbpf_unet_grad", "lbpf_unet_train_step",
            "lbpf_unet_param_count", "lbpf_unet_params", "lbpf_unet_device_bytes",
            "lbpf_unet_last_error", "lbpf_unet_destroy", "lbpf_unet_set_tensor_path",
            "lbpf_unet_status", "lbpf_surrogate_sample", "lbpf_surrogate_train",
            "lbpf_surrogate_target", "lbpf_surrogate_advance", "lbpf_init_polygon",
            "lbpf_measure_facets", "lbpf_growth_fit", "lbpf_facets_enqueue",
            "lbpf_facets_collect", "lbpf_set_solid")


def _load_library():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"liblbpf.so is not built ({LIB_PATH}); run __graft_entry__.build() first — "
            "there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    P = ctypes.POINTER(lbpf_params)
    lib.lbpf_params_default.argtypes = [P]
    lib.lbpf_create.argtypes = [P, vp, ctypes.POINTER(vp)]
    lib.lbpf_init_seed.argtypes = [vp, ctypes.POINTER(lbpf_seed)]
    lib.lbpf_init_fields.argtypes = [vp, dp, dp, dp, dp, dp, dp]
    lib.lbpf_step.argtypes = [vp, ctypes.c_int]
    lib.lbpf_read_fields.argtypes = [vp, ctypes.c_uint, vp, sz, ctypes.c_int]
    lib.lbpf_state_bytes.argtypes = [vp]
    lib.lbpf_state_bytes.restype = sz
    lib.lbpf_write_state.argtypes = [vp, vp, sz]
    lib.lbpf_diagnostics.argtypes = [vp, ctypes.POINTER(lbpf_diag)]
    lib.lbpf_set_stream.argtypes = [vp, vp]
    lib.lbpf_device_bytes.argtypes = [vp]
    lib.lbpf_device_bytes.restype = sz
    lib.lbpf_last_error.argtypes = [vp]
    lib.lbpf_last_error.restype = ctypes.c_char_p
    lib.lbpf_destroy.argtypes = [vp]
    lib.lbpf_destroy.restype = None
    lib.lbpf_field_sums_noalloc.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int, vp, vp]
    lib.lbpf_batch_create.argtypes = [P, ctypes.POINTER(lbpf_seed), ctypes.c_int, vp,
                                      ctypes.POINTER(vp)]
    lib.lbpf_batch_step.argtypes = [vp, ctypes.c_int]
    lib.lbpf_batch_diagnostics.argtypes = [vp, ctypes.POINTER(lbpf_diag)]
    lib.lbpf_batch_instance.argtypes = [vp, ctypes.c_int]
    lib.lbpf_batch_instance.restype = vp
    lib.lbpf_batch_count.argtypes = [vp]
    ip, fp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)
    lib.lbpf_batch_tuning.argtypes = [vp, ip, ip, fp, ip]
    lib.lbpf_batch_last_error.argtypes = [vp]
    lib.lbpf_batch_last_error.restype = ctypes.c_char_p
    lib.lbpf_batch_destroy.argtypes = [vp]
    lib.lbpf_batch_destroy.restype = None
    lib.lbpf_unet_create.argtypes = [ctypes.POINTER(lbpf_unet_cfg), vp, ctypes.POINTER(vp)]
    lib.lbpf_unet_forward.argtypes = [vp, vp, vp]
    lib.lbpf_unet_grad.argtypes = [vp, vp, vp, fp]
    lib.lbpf_unet_train_step.argtypes = [vp, vp, vp, ctypes.c_float, vp]
    lib.lbpf_unet_param_count.argtypes = [vp]
    lib.lbpf_unet_param_count.restype = sz
    lib.lbpf_unet_params.argtypes = [vp, ctypes.c_int, fp, sz, ctypes.c_int]
    lib.lbpf_unet_device_bytes.argtypes = [vp]
    lib.lbpf_unet_device_bytes.restype = sz
    lib.lbpf_unet_last_error.argtypes = [vp]
    lib.lbpf_unet_last_error.restype = ctypes.c_char_p
    lib.lbpf_unet_destroy.argtypes = [vp]
    lib.lbpf_unet_destroy.restype = None
    lib.lbpf_unet_set_tensor_path.argtypes = [vp, ctypes.c_int]
    lib.lbpf_unet_status.argtypes = [vp]
    lib.lbpf_surrogate_sample.argtypes = [vp, ctypes.POINTER(lbpf_surrogate_cfg), vp]
    lib.lbpf_surrogate_train.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int, vp, vp, vp,
                                         ctypes.c_int, vp]
    lib.lbpf_surrogate_target.argtypes = [ctypes.POINTER(lbpf_surrogate_cfg), vp, vp,
                                          ctypes.c_int64, vp, vp]
    lib.lbpf_surrogate_advance.argtypes = [vp, vp, ctypes.POINTER(lbpf_surrogate_cfg),
                                           ctypes.c_int, ctypes.POINTER(lbpf_surrogate_report)]
    lib.lbpf_init_polygon.argtypes = [vp, ctypes.POINTER(lbpf_polygon_seed)]
    lib.lbpf_measure_facets.argtypes = [vp, ctypes.c_int, dp, dp, ctypes.POINTER(lbpf_facets)]
    lib.lbpf_growth_fit.argtypes = [dp, dp, ctypes.c_int, dp, dp, dp]
    lib.lbpf_facets_enqueue.argtypes = [vp, ctypes.c_int, dp, dp]
    lib.lbpf_facets_collect.argtypes = [vp, ctypes.POINTER(lbpf_facets)]
    lib.lbpf_set_solid.argtypes = [vp, vp]
    keep = ("lbpf_state_bytes", "lbpf_device_bytes", "lbpf_last_error", "lbpf_destroy",
            "lbpf_batch_instance", "lbpf_batch_last_error", "lbpf_batch_destroy",
            "lbpf_unet_param_count", "lbpf_unet_device_bytes", "lbpf_unet_last_error",
            "lbpf_unet_destroy")
    for name in EXPORTED:
        if name not in keep:
            getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load_library()


def _check(h, rc: int):
    if rc != OK:
        msg = _lib.lbpf_last_error(h).decode() if h else ""
        raise LbpfError(rc, msg or "see stderr")


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- C ABI, one function each --------------------------------------------------
def lbpf_params_default(**overrides) -> lbpf_params:
    p = lbpf_params()
    _check(None, _lib.lbpf_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if k == "lambda":
            k = "lambda_"
        if k in ("bc", "body_force"):
            arr = getattr(p, k)
            for i in range(3):
                arr[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def lbpf_create(params: lbpf_params, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    rc = _lib.lbpf_create(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    if rc != OK:
        raise LbpfError(rc, "lbpf_create rejected the parameters (reason on stderr)")
    return h.value


def lbpf_init_seed(h: int, cx, cy, cz, radius, u0, noise_amp, seed) -> None:
    s = lbpf_seed(cx, cy, cz, radius, u0, noise_amp, seed)
    _check(h, _lib.lbpf_init_seed(h, ctypes.byref(s)))


def lbpf_init_polygon(h: int, cx, cy, normals, dist, u0, noise_amp, seed) -> None:
    """normals: [k, 2] outward unit normals; dist: [k] distances from (cx, cy)."""
    n = np.asarray(normals, np.float64).reshape(-1, 2)
    d = np.asarray(dist, np.float64).reshape(-1)
    if n.shape[0] != d.size or not 0 < d.size <= MAX_FACETS:
        raise LbpfError(EINVAL, "normals and dist must have the same length, at most 12")
    s = lbpf_polygon_seed(cx=cx, cy=cy, nfacets=d.size, u0=u0, noise_amp=noise_amp, seed=seed)
    for i in range(d.size):
        s.nx[i], s.ny[i], s.dist[i] = n[i, 0], n[i, 1], d[i]
    _check(h, _lib.lbpf_init_polygon(h, ctypes.byref(s)))


def _normals_xy(normals):
    n = np.ascontiguousarray(np.asarray(normals, np.float64).reshape(-1, 2))
    return np.ascontiguousarray(n[:, 0]), np.ascontiguousarray(n[:, 1])


def lbpf_measure_facets(h: int, normals) -> dict:
    """Crystal shape along the facet normals [k, 2] (k even, counter-clockwise,
    normal i + k/2 opposite to normal i)."""
    nx, ny = _normals_xy(normals)
    f = lbpf_facets()
    _check(h, _lib.lbpf_measure_facets(h, int(nx.size), _dptr(nx), _dptr(ny), ctypes.byref(f)))
    return _facets_dict(f)


def lbpf_facets_enqueue(h: int, normals) -> None:
    nx, ny = _normals_xy(normals)
    _check(h, _lib.lbpf_facets_enqueue(h, int(nx.size), _dptr(nx), _dptr(ny)))


def lbpf_facets_collect(h: int) -> dict:
    f = lbpf_facets()
    _check(h, _lib.lbpf_facets_collect(h, ctypes.byref(f)))
    return _facets_dict(f)


def _facets_dict(f) -> dict:
    k = f.nfacets
    return {"points": int(f.points), "support": np.array(f.support[:k]),
            "side_centre": np.stack([np.array(f.side_cx[:k]), np.array(f.side_cy[:k])], axis=1),
            "centre": np.array([f.cx, f.cy]), "L": np.array(f.L[:k]), "L_avg": f.L_avg,
            "Q": f.Q, "width": f.width, "height": f.height, "aspect": f.aspect}


def lbpf_growth_fit(t, L) -> tuple:
    """(slope, intercept, R^2) of the straight-line fit of L(t) (Eqs. 26-28)."""
    t = np.ascontiguousarray(np.asarray(t, np.float64).reshape(-1))
    L = np.ascontiguousarray(np.asarray(L, np.float64).reshape(-1))
    if t.size != L.size:
        raise LbpfError(EINVAL, "t and L differ in length")
    out = np.zeros(3)
    rc = _lib.lbpf_growth_fit(_dptr(t), _dptr(L), int(t.size), _dptr(out[0:]), _dptr(out[1:]),
                              _dptr(out[2:]))
    if rc != OK:
        raise LbpfError(rc, "lbpf_growth_fit: need >= 2 finite points, t not all equal")
    return float(out[0]), float(out[1]), float(out[2])


def hexagon_normals(theta: float = 0.0) -> np.ndarray:
    """Outward normals of a hexagon's sides, counter-clockwise from theta."""
    a = theta + np.pi / 3.0 * np.arange(6)
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def rhombus_normals(theta: float = 0.0, acute: float = np.pi / 3.0) -> np.ndarray:
    """Outward normals of a rhombus whose long diagonal lies along theta and
    whose acute angle is `acute`, counter-clockwise.  With acute = 60 deg they
    are normals 1, 2, 4, 5 of hexagon_normals(theta)."""
    b = np.pi / 2.0 - acute / 2.0
    a = theta + np.array([b, np.pi - b, np.pi + b, 2.0 * np.pi - b])
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def hexagonal_seed(perimeter: float, theta: float = 0.0):
    """(normals, dist) of a regular hexagon of the given perimeter."""
    side = perimeter / 6.0
    return hexagon_normals(theta), np.full(6, side * np.sqrt(3.0) / 2.0)


def rhombic_seed(perimeter: float, theta: float = 0.0, acute: float = np.pi / 3.0):
    """(normals, dist) of a rhombus of the given perimeter and acute angle."""
    side = perimeter / 4.0
    return rhombus_normals(theta, acute), np.full(4, side * np.sin(acute) / 2.0)


def lbpf_set_solid(h: int, mask) -> None:
    """Solid nodes: mask [ny, nx] or [nz, ny, nx] (nonzero = solid), or None
    to remove."""
    if mask is None:
        _check(h, _lib.lbpf_set_solid(h, None))
        return
    m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
    _check(h, _lib.lbpf_set_solid(h, ctypes.c_void_p(m.ctypes.data)))


def lbpf_init_fields(h: int, phi, U, rho=None, ux=None, uy=None, uz=None) -> None:
    arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1))
            for a in (phi, U, rho, ux, uy, uz)]
    _check(h, _lib.lbpf_init_fields(h, *[_dptr(a) for a in arrs]))


def lbpf_step(h: int, n: int = 1) -> None:
    _check(h, _lib.lbpf_step(h, int(n)))


def lbpf_state_bytes(h: int) -> int:
    return int(_lib.lbpf_state_bytes(h))


def lbpf_read_fields(h: int, mask: int, host_dst_ptr: int, nbytes: int, as_fp64: int) -> None:
    """Raw form: copy into caller-owned host memory at ``host_dst_ptr``."""
    _check(h, _lib.lbpf_read_fields(h, mask, ctypes.c_void_p(host_dst_ptr), nbytes, as_fp64))


def lbpf_write_state(h: int, host_src_ptr: int, nbytes: int) -> None:
    _check(h, _lib.lbpf_write_state(h, ctypes.c_void_p(host_src_ptr), nbytes))


def lbpf_diagnostics(h: int) -> dict:
    d = lbpf_diag()
    _check(h, _lib.lbpf_diagnostics(h, ctypes.byref(d)))
    return {"step": d.step, "solute_total": d.solute_total,
            "solute_drift_rel": d.solute_drift_rel, "mass_total": d.mass_total,
            "solid_volume": d.solid_volume, "r_eq": d.r_eq,
            "iface_pos": np.array(d.iface_pos[:]), "max_u": d.max_u, "nonfinite": d.nonfinite}


def lbpf_set_stream(h: int, stream: int | None) -> None:
    _check(h, _lib.lbpf_set_stream(h, ctypes.c_void_p(stream or 0)))


def lbpf_device_bytes(h: int) -> int:
    return int(_lib.lbpf_device_bytes(h))


def lbpf_last_error(h: int) -> str:
    return _lib.lbpf_last_error(h).decode()


def lbpf_destroy(h: int) -> None:
    _lib.lbpf_destroy(h)


def lbpf_field_sums_noalloc(phi_ptr, phi_prev_ptr, U_ptr, rho_ptr, n: int, fp64: int, out_ptr,
                            stream=None) -> int:
    """FP64 sums of caller-owned device fields without any device allocation
    (for callers that cannot allocate); returns the lbpf status code."""
    return int(_lib.lbpf_field_sums_noalloc(phi_ptr, phi_prev_ptr, U_ptr, rho_ptr, int(n),
                                            int(fp64), out_ptr, stream))


# ---- convenience wrapper -------------------------------------------------------------
def current_stream() -> int:
    """The calling thread's current torch CUDA stream (PyTorch supplies streams)."""
    import torch
    return torch.cuda.current_stream().cuda_stream


class Sim:
    """One simulation handle: owns its device state, runs on a CUDA stream."""

    def __init__(self, stream: int | None = None, **params):
        self.params = lbpf_params_default(**params)
        self.h = lbpf_create(self.params, stream)
        p = self.params
        self.shape = (p.nz, p.ny, p.nx) if p.dim == 3 else (p.ny, p.nx)
        self.nodes = int(np.prod(self.shape))

    def close(self):
        if getattr(self, "h", None):
            lbpf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_seed(self, cx, cy, cz=0.0, radius=8.0, u0=0.3, noise_amp=0.0, seed=1):
        lbpf_init_seed(self.h, cx, cy, cz, radius, u0, noise_amp, seed)

    def init_fields(self, phi, U, rho=None, ux=None, uy=None, uz=None):
        lbpf_init_fields(self.h, phi, U, rho, ux, uy, uz)

    def init_polygon(self, cx, cy, normals, dist, u0=0.3, noise_amp=0.0, seed=1):
        lbpf_init_polygon(self.h, cx, cy, normals, dist, u0, noise_amp, seed)

    def facets(self, normals) -> dict:
        return lbpf_measure_facets(self.h, normals)

    def set_solid(self, mask):
        m = None if mask is None else np.asarray(mask)
        if m is not None and m.size != self.nodes:
            raise LbpfError(EINVAL, f"mask must have {self.nodes} values")
        lbpf_set_solid(self.h, m)

    def step(self, n: int = 1):
        lbpf_step(self.h, n)

    def fields(self, names=("phi", "U", "rho", "ux", "uy"), fp64: bool = True) -> dict:
        mask = 0
        for nm in names:
            mask |= 1 << FIELD_NAMES.index(nm)
        order = [nm for nm in FIELD_NAMES if mask & (1 << FIELD_NAMES.index(nm))]
        out = np.empty((len(order), self.nodes), np.float64 if fp64 else np.float32)
        lbpf_read_fields(self.h, mask, out.ctypes.data, out.nbytes, 1 if fp64 else 0)
        return {nm: out[i].reshape(self.shape) for i, nm in enumerate(order)}

    def state(self) -> np.ndarray:
        buf = np.empty(lbpf_state_bytes(self.h), np.uint8)
        lbpf_read_fields(self.h, FIELD_STATE, buf.ctypes.data, buf.nbytes, 0)
        return buf

    def load_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        lbpf_write_state(self.h, buf.ctypes.data, buf.nbytes)

    def diagnostics(self) -> dict:
        return lbpf_diagnostics(self.h)


class _BorrowedSim(Sim):
    """A batch instance: an ordinary handle owned by its batch."""

    def __init__(self, h, params, batch):
        self.params = params
        self.h = h
        self._batch = batch  # keeps the owner alive
        p = params
        self.shape = (p.nz, p.ny, p.nx) if p.dim == 3 else (p.ny, p.nx)
        self.nodes = int(np.prod(self.shape))

    def close(self):
        self.h = None  # owned by the batch

    def __del__(self):
        pass


def lbpf_batch_create(params: list, seeds: list, stream: int | None = None) -> int:
    n = len(params)
    P_arr = (lbpf_params * n)(*params)
    S_arr = (lbpf_seed * n)(*[lbpf_seed(*s) for s in seeds])
    b = ctypes.c_void_p()
    rc = _lib.lbpf_batch_create(P_arr, S_arr, n, ctypes.c_void_p(stream or 0), ctypes.byref(b))
    if rc != OK:
        raise LbpfError(rc, "lbpf_batch_create failed (reason on stderr)")
    return b.value


def _bcheck(b, rc):
    if rc != OK:
        raise LbpfError(rc, _lib.lbpf_batch_last_error(b).decode())


class Batch:
    """Many 2D instances advanced by one persistent launch per step."""

    def __init__(self, params: list, seeds: list, stream: int | None = None):
        self.params = [lbpf_params_default(**p) for p in params]
        self.b = lbpf_batch_create(self.params, seeds, stream)
        self.count = len(self.params)

    def step(self, n: int = 1):
        _bcheck(self.b, _lib.lbpf_batch_step(self.b, int(n)))

    def instance(self, i: int) -> Sim:
        h = _lib.lbpf_batch_instance(self.b, i)
        if not h:
            raise IndexError(i)
        return _BorrowedSim(h, self.params[i], self)

    def diagnostics(self) -> list:
        arr = (lbpf_diag * self.count)()
        _bcheck(self.b, _lib.lbpf_batch_diagnostics(self.b, arr))
        return [{"step": d.step, "solute_total": d.solute_total, "mass_total": d.mass_total,
                 "solid_volume": d.solid_volume, "r_eq": d.r_eq,
                 "iface_pos": np.array(d.iface_pos[:]), "max_u": d.max_u,
                 "nonfinite": d.nonfinite} for d in arr]

    def tuning(self) -> dict:
        rows, stages, nvar = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * 8)()
        rc = _lib.lbpf_batch_tuning(self.b, ctypes.byref(rows), ctypes.byref(stages), ms,
                                    ctypes.byref(nvar))
        return {"tuned": rc == OK, "tile_rows": rows.value, "stages": stages.value,
                "ms_per_step": list(ms[:nvar.value])}

    def close(self):
        if getattr(self, "b", None):
            _lib.lbpf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UNet:
    """BF16 U-Net surrogate on the library's own kernels.  Inputs and targets
    are device FP32 NHWC arrays (torch tensors or raw pointers) of shape
    [batch, height, width, in_ch / out_ch]."""

    def __init__(self, in_ch=4, out_ch=4, base_ch=32, levels=4, batch=1, height=512, width=512,
                 seed=1, stream: int | None = None):
        self.cfg = lbpf_unet_cfg(in_ch, out_ch, base_ch, levels, batch, height, width, seed)
        self.n = ctypes.c_void_p()
        rc = _lib.lbpf_unet_create(ctypes.byref(self.cfg), ctypes.c_void_p(stream or 0),
                                   ctypes.byref(self.n))
        if rc != OK:
            raise LbpfError(rc, "lbpf_unet_create failed (reason on stderr)")
        self.n = self.n.value

    def _check(self, rc):
        if rc != OK:
            raise LbpfError(rc, _lib.lbpf_unet_last_error(self.n).decode())

    @staticmethod
    def _ptr(a):
        return ctypes.c_void_p(a if isinstance(a, int) else a.data_ptr())

    def forward(self, x, y):
        self._check(_lib.lbpf_unet_forward(self.n, self._ptr(x), self._ptr(y)))

    def grad(self, x, t) -> float:
        loss = ctypes.c_float()
        self._check(_lib.lbpf_unet_grad(self.n, self._ptr(x), self._ptr(t), ctypes.byref(loss)))
        return float(loss.value)

    def train_step(self, x, t, lr: float, loss_dev=None):
        self._check(_lib.lbpf_unet_train_step(self.n, self._ptr(x), self._ptr(t), float(lr),
                                              None if loss_dev is None else self._ptr(loss_dev)))

    def set_tensor_path(self, use_tcgen05: bool):
        """True (default): tcgen05 / TMEM / TMA convolutions; False: mma.sync."""
        self._check(_lib.lbpf_unet_set_tensor_path(self.n, 1 if use_tcgen05 else 0))

    def status(self):
        """Synchronise and raise if a tensor-core kernel gave up waiting."""
        self._check(_lib.lbpf_unet_status(self.n))

    @property
    def param_count(self) -> int:
        return int(_lib.lbpf_unet_param_count(self.n))

    def _params(self, which: int) -> np.ndarray:
        out = np.empty(self.param_count, np.float32)
        self._check(_lib.lbpf_unet_params(self.n, which, out.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), out.size, 0))
        return out

    def weights(self) -> np.ndarray:
        return self._params(0)

    def grads(self) -> np.ndarray:
        return self._params(1)

    def set_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, np.float32)
        if w.size != self.param_count:
            raise ValueError(f"expected {self.param_count} parameters, got {w.size}")
        self._check(_lib.lbpf_unet_params(self.n, 0, w.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), w.size, 1))

    @property
    def device_bytes(self) -> int:
        return int(_lib.lbpf_unet_device_bytes(self.n))

    def close(self):
        if getattr(self, "n", None):
            _lib.lbpf_unet_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def surrogate_cfg(steps_per_block=50, judge_every=8, drift_tol=1e-3, iface_tol=1.0,
                  iface_budget=0.0, iface_rel_tol=0.0, shift=(0.0, 0.3, 0.0, 0.0),
                  scale=(1.0, 0.2, 0.01, 0.01),
                  res_scale=(0.05, 0.005, 0.001, 0.001)) -> lbpf_surrogate_cfg:
    c = lbpf_surrogate_cfg()
    c.steps_per_block, c.judge_every = int(steps_per_block), int(judge_every)
    c.drift_tol, c.iface_tol = float(drift_tol), float(iface_tol)
    c.iface_budget, c.iface_rel_tol = float(iface_budget), float(iface_rel_tol)
    c.shift[:], c.scale[:], c.res_scale[:] = list(shift), list(scale), list(res_scale)
    return c


def lbpf_surrogate_sample(sim: "Sim", cfg: lbpf_surrogate_cfg, x) -> None:
    """Normalised network input of the simulation's state into device x [ny][nx][4]."""
    _check(sim.h, _lib.lbpf_surrogate_sample(sim.h, ctypes.byref(cfg), UNet._ptr(x)))


def lbpf_surrogate_train(net: "UNet", X, T, idx, flip, lr, log_every: int = 50) -> np.ndarray:
    """The library's training loop on device pairs X, T [n, h, w, 4]: idx
    [steps, batch] pair indices, flip [steps] (0, 1 rows, 2 columns) or None,
    lr [steps].  Returns the logged minibatch losses."""
    idx = np.ascontiguousarray(idx, np.int32)
    lr = np.ascontiguousarray(lr, np.float32)
    steps = int(lr.shape[0])
    flip = None if flip is None else np.ascontiguousarray(flip, np.int32)
    nlog = -(-steps // log_every)
    out = np.zeros(nlog, np.float32)
    rc = _lib.lbpf_surrogate_train(net.n, UNet._ptr(X), UNet._ptr(T), int(X.shape[0]), steps,
                                   idx.ctypes.data, None if flip is None else flip.ctypes.data,
                                   lr.ctypes.data, int(log_every), out.ctypes.data)
    if rc != OK:
        raise LbpfError(rc, _lib.lbpf_unet_last_error(net.n).decode())
    return out


def lbpf_surrogate_target(cfg: lbpf_surrogate_cfg, x0, x1, npix: int, t, stream=None) -> None:
    rc = _lib.lbpf_surrogate_target(ctypes.byref(cfg), UNet._ptr(x0), UNet._ptr(x1), int(npix),
                                    UNet._ptr(t), ctypes.c_void_p(stream or 0))
    if rc != OK:
        raise LbpfError(rc, "lbpf_surrogate_target: invalid arguments")


def lbpf_surrogate_advance(sim: "Sim", net: UNet, cfg: lbpf_surrogate_cfg, blocks: int) -> dict:
    rep = lbpf_surrogate_report()
    _check(sim.h, _lib.lbpf_surrogate_advance(sim.h, net.n, ctypes.byref(cfg), int(blocks),
                                              ctypes.byref(rep)))
    return {f: getattr(rep, f) for f, _ in rep._fields_}
