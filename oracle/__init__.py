"""FP64 CPU oracle of the coupled LB phase-field crystal-growth step.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.  The C source (``lbpf_oracle.c``) follows Sec. 2.2 of the paper
(Eqs. 1-23) as plain double-precision loops; this file only builds it with gcc
and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbpf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblbpf_oracle.so")

PERIODIC, INLET_OUTLET, WALL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: the same source builds on
    x86_64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                             os.path.getmtime(_SRC[:-2] + ".h")))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("flow", ctypes.c_int), ("fold", ctypes.c_int),
        ("aniso_literal", ctypes.c_int),
        ("tau_phi0", ctypes.c_double), ("tau_u_liquid", ctypes.c_double),
        ("tau_f", ctypes.c_double), ("w0", ctypes.c_double), ("lambda_", ctypes.c_double),
        ("eps", ctypes.c_double), ("theta0", ctypes.c_double), ("h_drag", ctypes.c_double),
        ("u_inlet", ctypes.c_double), ("u0_inlet", ctypes.c_double),
        ("body", ctypes.c_double * 3),
        ("collision", ctypes.c_int), ("omega_bulk", ctypes.c_double),
        ("omega_high", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        lib.orc_tau0.argtypes = [P]
        lib.orc_tau0.restype = ctypes.c_double
        lib.orc_lambda.argtypes = [P]
        lib.orc_lambda.restype = ctypes.c_double
        lib.orc_create.argtypes = [P]
        lib.orc_create.restype = vp
        lib.orc_destroy.argtypes = [vp]
        lib.orc_init_seed.argtypes = [vp] + [ctypes.c_double] * 6 + [ctypes.c_uint64]
        lib.orc_init_fields.argtypes = [vp] + [dp] * 6
        lib.orc_set_solid.argtypes = [vp, ctypes.c_void_p]
        lib.orc_set_solid.restype = ctypes.c_int
        lib.orc_init_polygon.argtypes = ([vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
                                         + [dp] * 3 + [ctypes.c_double] * 2 + [ctypes.c_uint64])
        lib.orc_step.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        lib.orc_step_count.argtypes = [vp]
        lib.orc_step_count.restype = ctypes.c_longlong
        lib.orc_fields.argtypes = [vp] + [dp] * 6
        lib.orc_phi_prev.argtypes = [vp, dp]
        lib.orc_pops.argtypes = [vp, ctypes.c_int, dp]
        lib.orc_pops.restype = ctypes.c_int
        lib.orc_aux.argtypes = [vp, dp, dp, dp, dp]
        lib.orc_aniso.argtypes = [P, dp, dp, dp]
        lib.orc_diag.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        _lib = lib
    return _lib


@dataclass
class Params:
    """Model parameters (names follow Eqs. 1-23 of the paper)."""
    dim: int = 2
    nx: int = 128
    ny: int = 128
    nz: int = 1
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    flow: int = 0
    fold: int = 4
    aniso_literal: int = 0
    tau_phi0: float = 0.8
    tau_u_liquid: float = 0.8
    tau_f: float = 0.6
    w0: float = 2.0
    lambda_: float = -1.0
    eps: float = 0.05
    theta0: float = 0.0
    h_drag: float = 2.757
    u_inlet: float = 0.0
    u0_inlet: float = 0.0
    body: tuple = (0.0, 0.0, 0.0)
    collision: int = 0
    omega_bulk: float = 0.0
    omega_high: float = 0.0

    def _c(self) -> _Params:
        p = _Params()
        for name, _ in _Params._fields_:
            v = getattr(self, name)
            if name in ("bc", "body"):
                arr = getattr(p, name)
                for i in range(3):
                    arr[i] = v[i]
            else:
                setattr(p, name, v)
        return p

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * (self.nz if self.dim == 3 else 1)

    @property
    def shape(self) -> tuple:
        return (self.nz, self.ny, self.nx) if self.dim == 3 else (self.ny, self.nx)


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def tau0(p: Params) -> float:
    return _load().orc_tau0(ctypes.byref(p._c()))


def coupling(p: Params) -> float:
    return _load().orc_lambda(ctypes.byref(p._c()))


def aniso(p: Params, grad):
    """(a_s, N) for one gradient vector (Eq. 3, Eq. 21)."""
    g = np.ascontiguousarray(np.asarray(grad, dtype=np.float64).reshape(3))
    a = np.zeros(1)
    n = np.zeros(3)
    _load().orc_aniso(ctypes.byref(p._c()), _ptr(g), _ptr(a), _ptr(n))
    return float(a[0]), n


class Oracle:
    """One simulation instance of the FP64 oracle."""

    def __init__(self, params: Params):
        self.p = params
        self._cp = params._c()
        self._lib = _load()
        self._h = self._lib.orc_create(ctypes.byref(self._cp))

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_seed(self, cx, cy, cz, radius, u0, noise_amp, seed):
        self._lib.orc_init_seed(self._h, cx, cy, cz, radius, u0, noise_amp, seed)

    def init_polygon(self, cx, cy, normals, dist, u0, noise_amp, seed):
        """Convex polygon seed: normals [k, 2] outward unit normals, dist [k]."""
        nrm = np.ascontiguousarray(np.asarray(normals, dtype=np.float64).reshape(-1, 2))
        nx, ny = np.ascontiguousarray(nrm[:, 0]), np.ascontiguousarray(nrm[:, 1])
        d = np.ascontiguousarray(np.asarray(dist, dtype=np.float64).reshape(-1))
        assert d.size == nx.size
        self._lib.orc_init_polygon(self._h, cx, cy, int(d.size), _ptr(nx), _ptr(ny), _ptr(d),
                                   u0, noise_amp, seed)

    def set_solid(self, mask):
        """Solid nodes: mask of the grid's shape ([ny, nx] or [nz, ny, nx]),
        nonzero = solid; None removes it."""
        if mask is None:
            rc = self._lib.orc_set_solid(self._h, None)
        else:
            m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.uint8)
            assert m.size == self.p.nodes
            rc = self._lib.orc_set_solid(self._h, m.ctypes.data)
        if rc != 0:
            raise ValueError("solid mask rejected (a solid inlet or outlet column)")

    def init_fields(self, phi, U, rho=None, ux=None, uy=None, uz=None):
        arrs = []
        for a in (phi, U, rho, ux, uy, uz):
            arrs.append(None if a is None else
                        np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)))
        self._lib.orc_init_fields(self._h, *[_ptr(a) for a in arrs])

    def step(self, n: int = 1, threads: int = 1):
        self._lib.orc_step(self._h, int(n), int(threads))

    @property
    def step_count(self) -> int:
        return int(self._lib.orc_step_count(self._h))

    def fields(self) -> dict:
        n = self.p.nodes
        out = {k: np.zeros(n) for k in ("phi", "U", "rho", "ux", "uy", "uz")}
        self._lib.orc_fields(self._h, *[_ptr(out[k]) for k in ("phi", "U", "rho", "ux", "uy", "uz")])
        return {k: v.reshape(self.p.shape) for k, v in out.items()}

    def phi_prev(self):
        out = np.zeros(self.p.nodes)
        self._lib.orc_phi_prev(self._h, _ptr(out))
        return out.reshape(self.p.shape)

    def pops(self, which: str):
        w = {"f": 0, "g": 1, "h": 2}[which]
        q = self._lib.orc_pops(self._h, w, None)
        out = np.zeros((q, self.p.nodes))
        if q:
            self._lib.orc_pops(self._h, w, _ptr(out))
        return out.reshape((q,) + self.p.shape)

    def aux(self) -> dict:
        n = self.p.nodes
        out = {k: np.zeros(n) for k in ("a_s", "gx", "gy", "gz")}
        self._lib.orc_aux(self._h, *[_ptr(out[k]) for k in ("a_s", "gx", "gy", "gz")])
        return {k: v.reshape(self.p.shape) for k, v in out.items()}

    def diag(self, icx: int, icy: int, icz: int = 0) -> dict:
        out = np.zeros(12)
        self._lib.orc_diag(self._h, icx, icy, icz, _ptr(out))
        return {"solute_total": out[0], "mass_total": out[1], "solid_volume": out[2],
                "r_eq": out[3], "max_u": out[4], "nonfinite": int(out[5]),
                "iface_pos": out[6:12].copy()}
