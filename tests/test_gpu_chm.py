"""GPU parity of the central Hermite MRT flow collision (LBPF_COLL_CHM)
against the oracle, with the coupled phase field (masked velocity u*, drag),
other rates, solid nodes and 16-bit storage; its stability where BGK fails;
and the C ABI's rejections."""
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
    a = L.Sim(dim=2, nx=p["nx"], ny=p["ny"], bc=p["bc"], flow=1, storage=P.STORAGE[storage],
              fold=p["fold"], eps_aniso=p["eps"], theta0=p["theta0"], tau_f=p["tau_f"],
              u_inlet=p["u_in"], u0_inlet=p["U_in"], body_force=p["body"],
              collision=L.COLL_CHM, chm_omega_bulk=wb, chm_omega_high=wh)
    b = oracle.Oracle(oracle.Params(
        dim=2, nx=p["nx"], ny=p["ny"], bc=p["bc"], flow=1, fold=p["fold"], eps=p["eps"],
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
    for kw in (dict(dim=3, nx=16, ny=16, nz=16, fold=0, flow=1),  # 3D
               dict(dim=2, nx=16, ny=16, flow=0),                  # no flow lattice
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
