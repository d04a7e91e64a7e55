"""Builds a CUDA-library handle and an oracle instance with the same
parameters and the same initial state.  Holds none of the method's
arithmetic: it only maps parameter names and passes seeds and seeded input
fields to both sides."""
import os

import numpy as np

import oracle
import paper_2206_02145_gb300 as L

THREADS = max(1, min(16, os.cpu_count() or 1))

STORAGE = {"fp32": L.FP32, "fp64": L.FP64, "fp16": L.FP16_SHIFTED, "bf16": L.BF16_SHIFTED}


def params(dim=2, nx=64, ny=64, nz=1, bc=(0, 0, 0), flow=0, fold=4, eps=0.05, theta0=0.0,
           tau_phi0=0.8, tau_u=0.8, tau_f=0.6, w0=2.0, lam=-1.0, u_in=0.0, U_in=0.0,
           body=(0.0, 0.0, 0.0), literal=0):
    return dict(dim=dim, nx=nx, ny=ny, nz=nz, bc=tuple(bc), flow=flow, fold=fold, eps=eps,
                theta0=theta0, tau_phi0=tau_phi0, tau_u=tau_u, tau_f=tau_f, w0=w0, lam=lam,
                u_in=u_in, U_in=U_in, body=tuple(body), literal=literal)


def lib_sim(p, storage="fp32", stream=None):
    return L.Sim(stream=stream, dim=p["dim"], nx=p["nx"], ny=p["ny"], nz=p["nz"], bc=p["bc"],
                 flow=p["flow"], storage=STORAGE[storage], fold=p["fold"],
                 aniso_literal=p["literal"], tau_phi0=p["tau_phi0"],
                 tau_u_liquid=p["tau_u"], tau_f=p["tau_f"], w0=p["w0"], lambda_=p["lam"],
                 eps_aniso=p["eps"], theta0=p["theta0"], u_inlet=p["u_in"],
                 u0_inlet=p["U_in"], body_force=p["body"])


def oracle_sim(p):
    return oracle.Oracle(oracle.Params(
        dim=p["dim"], nx=p["nx"], ny=p["ny"], nz=p["nz"], bc=p["bc"], flow=p["flow"],
        fold=p["fold"], aniso_literal=p["literal"], tau_phi0=p["tau_phi0"],
        tau_u_liquid=p["tau_u"], tau_f=p["tau_f"], w0=p["w0"], lambda_=p["lam"], eps=p["eps"],
        theta0=p["theta0"], u_inlet=p["u_in"], u0_inlet=p["U_in"], body=p["body"]))


def seeded_fields(p, seed, radius, u0, amp_u=0.0, noise=0.01):
    """Seeded synthetic initial fields: a tanh-free blob of phi (smooth bump,
    not the model's profile), uniform U with noise, optional random flow."""
    rng = np.random.default_rng(seed)
    shape = (p["nz"], p["ny"], p["nx"]) if p["dim"] == 3 else (p["ny"], p["nx"])
    grids = np.meshgrid(*[np.arange(s, dtype=float) for s in shape], indexing="ij")
    r2 = sum((g - s / 2.0) ** 2 for g, s in zip(grids, shape))
    phi = 2.0 * np.exp(-r2 / (2.0 * radius ** 2)) - 1.0 + noise * rng.uniform(-1, 1, shape)
    U = u0 + noise * rng.uniform(-1, 1, shape)
    rho = 1.0 + 0.001 * rng.uniform(-1, 1, shape)
    us = [amp_u * rng.uniform(-1, 1, shape) for _ in range(3)]
    return phi, U, rho, us


def pair(p, storage="fp32", seed_args=None, fields=None, stream=None):
    """(lib Sim, Oracle) in the same initial state."""
    a = lib_sim(p, storage, stream)
    b = oracle_sim(p)
    if seed_args is not None:
        a.init_seed(*seed_args)
        b.init_seed(*seed_args)
    else:
        phi, U, rho, us = fields
        uz = us[2] if p["dim"] == 3 else None
        a.init_fields(phi, U, rho, us[0], us[1], uz)
        b.init_fields(phi, U, rho, us[0], us[1], uz)
    return a, b


def max_errors(a, b, fields=("phi", "U", "rho", "ux", "uy")):
    got = a.fields(fields)
    want = b.fields()
    return {k: float(np.abs(got[k] - want[k]).max()) for k in fields}


# lattice weights of the exported state's direction order (for decoding the
# stored deviations d_a = p_a - w_a M_ref back to populations)
_W = {9: [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4,
      19: [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12,
      7: [1 / 4] + [1 / 8] * 6}


HDR = 128  # bytes of the exported state's header


def decode_pops(sim, buf=None):
    """Populations {'f','g','h'} [q, ...] of a library handle's exported state."""
    if buf is None:
        buf = sim.state()
    hdr = np.frombuffer(buf[:48].tobytes(), dtype=np.int32, count=8, offset=16)
    dim, flow, q, elem = int(hdr[0]), int(hdr[5]), int(hdr[6]), int(hdr[7])
    u_ref = float(np.frombuffer(buf[48:56].tobytes(), dtype=np.float64)[0])
    storage = int(hdr[4])
    dt = {8: np.float64, 4: np.float32}.get(elem)
    n = sim.nodes
    raw = np.frombuffer(buf[HDR:HDR + q * n * elem].tobytes(),
                        dtype=dt if dt else np.uint16).reshape((q, n))
    if elem == 2:
        if storage == L.FP16_SHIFTED:
            raw = raw.view(np.float16).astype(np.float64)
        else:  # bfloat16: the upper half of a float32
            raw = (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    raw = raw.astype(np.float64)
    qf = (9 if dim == 2 else 19) if flow else 0
    qs = 9 if dim == 2 else 7
    g_ref = u_ref
    if elem == 2:
        # per-node g reference: the first FP16 plane after the FP32 phi ring
        off = HDR + q * n * elem + n * 4
        g_ref = np.frombuffer(buf[off:off + 2 * n].tobytes(), dtype=np.float16)
        g_ref = g_ref.astype(np.float64)[None, :]
    out = {}
    for name, lo, qq, ref in (("f", 0, qf, 1.0), ("g", qf, qs, g_ref), ("h", qf + qs, qs, -1.0)):
        w = np.array(_W[qq]) if qq else np.zeros(0)
        out[name] = (raw[lo:lo + qq] + w[:, None] * ref).reshape((qq,) + sim.shape)
    return out
