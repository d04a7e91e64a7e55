"""GPU parity of the central Hermite MRT flow collision (LBPF_COLL_CHM)
against the oracle, in 2D (D2Q9) and 3D (D3Q19), with the coupled phase
field (masked velocity u*, drag), other rates, walls, solid nodes and 16-bit
storage; its stability where BGK fails; and the C ABI's rejections."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import _pairs
    return _pairs


@pytest.fixture(scope="module")
def L():
    import paper_2206_02145_gb300 as lib
    return lib


def chm_pair(P, L, p, storage, wb=0.0, wh=0.0):
    a = L.Sim(dim=p["dim"], nx=p["nx"], ny=p["ny"], nz=p["nz"], bc=p["bc"], flow=1,
              storage=P.STORAGE[storage],
              fold=p["fold"], eps_aniso=p["eps"], theta0=p["theta0"], tau_f=p["tau_f"],
              u_inlet=p["u_in"], u0_inlet=p["U_in"], body_force=p["body"],
              collision=L.COLL_CHM, chm_omega_bulk=wb, chm_omega_high=wh)
    b = oracle.Oracle(oracle.Params(
        dim=p["dim"], nx=p["nx"], ny=p["ny"], nz=p["nz"], bc=p["bc"], flow=1, fold=p["fold"],
        eps=p["eps"],
        theta0=p["theta0"], tau_f=p["tau_f"], u_inlet=p["u_in"], u0_inlet=p["U_in"],
        body=p["body"], collision=1, omega_bulk=wb, omega_high=wh))
    return a, b


def inflow_case(P, nx=128, ny=96, tau_f=0.6):
    return P.params(nx=nx, ny=ny, flow=1, fold=5, eps=0.03, bc=(1, 0, 0), u_in=0.01, U_in=0.4,
                    tau_f=tau_f)


SEED = (60.0, 48.0, 0.0, 10.0, 0.4, 0.01, 2)


@pytest.mark.parametrize("storage,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_coupled_inflow_matches_oracle(P, L, storage, tol):
    p = inflow_case(P)
    a, b = chm_pair(P, L, p, storage)
    a.init_seed(*SEED)
    b.init_seed(*SEED)
    a.step(300)
    b.step(300, P.THREADS)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < tol, errs
    pa, pb = P.decode_pops(a), {k: b.pops(k) for k in "fgh"}
    for k in "fgh":
        assert np.abs(pa[k] - pb[k]).max() < tol, k


def test_other_rates_body_force_and_ragged_grid(P, L):
    p = P.params(nx=70, ny=45, flow=1, fold=4, eps=0.04, body=(2e-6, -1e-6, 0.0), tau_f=0.55)
    a, b = chm_pair(P, L, p, "fp64", wb=1.3, wh=1.7)
    a.init_seed(35.0, 22.0, 0.0, 8.0, 0.35, 0.01, 5)
    b.init_seed(35.0, 22.0, 0.0, 8.0, 0.35, 0.01, 5)
    a.step(250)
    b.step(250, P.THREADS)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < TOL64, errs


def test_with_solid_nodes(P, L):
    p = inflow_case(P)
    mask = np.zeros((96, 128), np.uint8)
    mask[30:66, 20:22] = 1
    for storage, tol in (("fp64", TOL64), ("fp32", TOL32)):
        a, b = chm_pair(P, L, p, storage)
        a.init_seed(*SEED)
        b.init_seed(*SEED)
        a.set_solid(mask)
        b.set_solid(mask)
        a.step(300)
        b.step(300, P.THREADS)
        errs = P.max_errors(a, b)
        assert max(errs.values()) < tol, (storage, errs)


def test_16bit_storage(P, L):
    p = inflow_case(P)
    a, b = chm_pair(P, L, p, "fp16")
    a.init_seed(*SEED)
    b.init_seed(*SEED)
    a.step(300)
    b.step(300, P.THREADS)
    errs = P.max_errors(a, b)
    for k, bound in dict(phi=8e-3, U=9e-3, rho=4e-5, ux=4e-5, uy=3e-5).items():
        assert errs[k] < bound, (k, errs)


def test_stable_where_bgk_fails(P, L):
    # a double shear layer at tau_f = 0.5005 (the oracle pin's case)
    n = 64
    y, x = np.mgrid[0:n, 0:n].astype(float)
    ux = 0.1 * np.tanh(80 * (np.minimum(y, n - y) / n - 0.25))
    uy = 0.005 * np.sin(2 * math.pi * x / n)

    def run(collision):
        s = L.Sim(dim=2, nx=n, ny=n, flow=1, eps_aniso=0.0, lambda_=0.0, tau_f=0.5005,
                  collision=collision)
        s.init_fields(-np.ones((n, n)), np.zeros((n, n)), None, ux, uy)
        try:
            s.step(3000)
            f = s.fields(("ux", "uy"))
            return float(np.abs(np.stack([f["ux"], f["uy"]])).max())
        except L.LbpfError as e:
            assert e.code == L.ENONFINITE
            return float("inf")
    assert run(L.COLL_BGK) > 1.0
    assert run(L.COLL_CHM) < 0.2


def test_full_size_sample(P, L):
    p = inflow_case(P, 1024, 1024)
    a, b = chm_pair(P, L, p, "fp32")
    seed = (300.0, 512.0, 0.0, 16.0, 0.4, 0.01, 1)
    a.init_seed(*seed)
    b.init_seed(*seed)
    a.step(10)
    b.step(10, P.THREADS)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < TOL32, errs


def test_rejections(P, L):
    for kw in (dict(dim=3, nx=16, ny=16, nz=16, fold=0, flow=0),  # no flow lattice
               dict(dim=2, nx=16, ny=16, flow=0),
               dict(dim=2, nx=16, ny=16, flow=1, chm_omega_bulk=2.5),
               dict(dim=2, nx=16, ny=16, flow=1, chm_omega_high=-0.5)):
        with pytest.raises(L.LbpfError) as e:
            L.Sim(collision=L.COLL_CHM, **kw)
        assert e.value.code == L.EINVAL
    with pytest.raises(L.LbpfError):
        L.Sim(dim=2, nx=16, ny=16, flow=1, collision=7)
    kw = dict(dim=2, nx=64, ny=64, flow=1)
    with pytest.raises(L.LbpfError) as e:  # one collision per batch
        L.Batch([kw, dict(kw, collision=L.COLL_CHM)], [(32.0, 32.0, 0.0, 6.0, 0.3, 0.0, 1)] * 2,
                None)
    assert e.value.code == L.EINVAL


@pytest.mark.parametrize("storage", ["FP32", "FP16_SHIFTED"])
def test_batch_equals_single_instances_bitwise(L, storage):
    # a CHM sweep of uneven grids and rates, one instance with a baffle: the
    # batched step (every tile shape, through the tuner) evolves each instance
    # bit for bit like the instance stepped alone
    sizes = [(100, 70), (64, 64), (130, 40), (48, 200)]
    params, seeds = [], []
    for i, (nx, ny) in enumerate(sizes):
        params.append(dict(dim=2, nx=nx, ny=ny, flow=1, storage=getattr(L, storage), fold=5,
                           eps_aniso=0.03 + 0.005 * i, bc=(1, 0, 0), u_inlet=0.01,
                           u0_inlet=0.3 + 0.05 * i, tau_f=0.55 + 0.05 * i,
                           collision=L.COLL_CHM, chm_omega_bulk=1.0 + 0.2 * i,
                           chm_omega_high=1.0 + 0.1 * i))
        seeds.append((0.5 * nx, 0.5 * ny, 0.0, min(nx, ny) / 6, 0.3 + 0.05 * i, 0.01, 40 + i))
    mask = np.zeros((40, 130), np.uint8)
    mask[10:30, 20:22] = 1
    b = L.Batch(params, seeds, None)
    b.instance(2).set_solid(mask)
    b.step(131)
    for i, (p, s) in enumerate(zip(params, seeds)):
        sim = L.Sim(**p)
        if i == 2:
            sim.set_solid(mask)
        sim.init_seed(*s)
        sim.step(131)
        assert np.array_equal(b.instance(i).state(), sim.state()), i
    b.close()


# ---- 3D: D3Q19 flow ---------------------------------------------------------------
F3 = ("phi", "U", "rho", "ux", "uy", "uz")
SEED3 = (14.0, 18.0, 10.0, 6.0, 0.5, 0.01, 4)


@pytest.mark.parametrize("storage,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_3d_coupled_inflow_matches_oracle(P, L, storage, tol):
    p = P.params(dim=3, nx=40, ny=36, nz=20, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.5, tau_f=0.55)
    a, b = chm_pair(P, L, p, storage)
    a.init_seed(*SEED3)
    b.init_seed(*SEED3)
    a.step(100)
    b.step(100, P.THREADS)
    errs = P.max_errors(a, b, F3)
    assert max(errs.values()) < tol, errs
    pa, pb = P.decode_pops(a), {k: b.pops(k) for k in "fgh"}
    for k in "fgh":
        assert np.abs(pa[k] - pb[k]).max() < tol, k


@pytest.mark.parametrize("storage,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_3d_ragged_walls_other_rates(P, L, storage, tol):
    # sizes off the 32 x 4 column and the 8-plane z chunk, walls in y and z,
    # an inlet, trace and higher-order rates of their own
    p = P.params(dim=3, nx=37, ny=19, nz=45, flow=1, fold=0, eps=0.04, bc=(1, 2, 2),
                 u_in=0.004, U_in=0.45, tau_f=0.6)
    f = P.seeded_fields(p, seed=11, radius=5.0, u0=0.45, amp_u=0.004)
    a, b = chm_pair(P, L, p, storage, wb=1.3, wh=1.7)
    for s in (a, b):
        s.init_fields(f[0], f[1], f[2], *f[3])
    a.step(60)
    b.step(60, P.THREADS)
    errs = P.max_errors(a, b, F3)
    assert max(errs.values()) < tol, errs


def test_3d_periodic_body_force(P, L):
    p = P.params(dim=3, nx=21, ny=18, nz=14, flow=1, fold=0, eps=0.04, body=(2e-6, -1e-6, 1e-6),
                 tau_f=0.52)
    f = P.seeded_fields(p, seed=7, radius=4.0, u0=0.5, amp_u=0.02)
    a, b = chm_pair(P, L, p, "fp64", wb=0.8, wh=1.2)
    for s in (a, b):
        s.init_fields(f[0], f[1], f[2], *f[3])
    a.step(80)
    b.step(80, P.THREADS)
    errs = P.max_errors(a, b, F3)
    assert max(errs.values()) < TOL64, errs


@pytest.mark.parametrize("storage,bounds", [
    ("fp16", dict(phi=2e-3, U=3e-3, rho=1.3e-5, ux=1e-5, uy=6e-6, uz=6e-6)),
    ("bf16", dict(phi=0.04, U=0.025, rho=1e-4, ux=8e-5, uy=5e-5, uz=5e-5))])
def test_3d_16bit_storage(P, L, storage, bounds):
    p = P.params(dim=3, nx=48, ny=48, nz=48, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.3)
    seed = (24.0, 24.0, 24.0, 10.0, 0.3, 0.01, 1)
    a, b = chm_pair(P, L, p, storage)
    a.init_seed(*seed)
    b.init_seed(*seed)
    a.step(100)
    b.step(100, P.THREADS)
    errs = P.max_errors(a, b, tuple(bounds))
    for k, bound in bounds.items():
        assert errs[k] < bound, (k, errs)


def test_3d_stable_where_bgk_fails(P, L):
    # a 3D double shear layer at tau_f = 0.501 on 64^3: BGK reports
    # non-finite values within 1000 steps; the central Hermite MRT with its
    # default rates stays bounded over 3000
    n = 64
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    ux = 0.1 * np.tanh(80 * (np.minimum(y, n - y) / n - 0.25))
    uy = 0.005 * np.sin(2 * math.pi * x / n)
    uz = 0.005 * np.sin(2 * math.pi * x / n + 1.0)

    def run(collision):
        s = L.Sim(dim=3, nx=n, ny=n, nz=n, fold=0, flow=1, eps_aniso=0.0, lambda_=0.0,
                  tau_f=0.501, collision=collision)
        s.init_fields(-np.ones((n, n, n)), np.zeros((n, n, n)), None, ux, uy, uz)
        try:
            s.step(3000)
            f = s.fields(("ux", "uy", "uz"))
            return float(np.abs(np.stack([f["ux"], f["uy"], f["uz"]])).max())
        except L.LbpfError as e:
            assert e.code == L.ENONFINITE
            return float("inf")
    assert run(L.COLL_BGK) > 1.0
    assert run(L.COLL_CHM) < 0.2


def test_3d_full_size_sample(P, L):
    # the 256^3 problem of the benchmark with CHM, two steps, FP32
    p = P.params(dim=3, nx=256, ny=256, nz=256, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.3)
    seed = (128.0, 128.0, 128.0, 12.0, 0.3, 0.01, 1)
    a, b = chm_pair(P, L, p, "fp32")
    a.init_seed(*seed)
    b.init_seed(*seed)
    a.step(2)
    b.step(2, P.THREADS)
    errs = P.max_errors(a, b, F3)
    assert max(errs.values()) < TOL32, errs
