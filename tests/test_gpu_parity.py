"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

Tolerances: FP32 populations within 1e-5 max-abs per field (phi, U, rho,
u) and interface positions within 0.25 lattice units; the FP64 build within
1e-10.  Sizes span several tiles (32 x 8 in 2D, 32 x 4 x 2 in 3D) and
ragged edges; the 1024^2 case is the benchmark's configuration.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import _pairs
    return _pairs


def check(P, a, b, tol, fields=("phi", "U", "rho", "ux", "uy")):
    errs = P.max_errors(a, b, fields)
    assert max(errs.values()) < tol, errs
    return errs


# --- 2D, no flow: 128^2 periodic, 4-fold eps 0.05, U0 0.3, R 8, noise 0.01 ------
def test_c1_fp32_2000_steps(P):
    p = P.params(nx=128, ny=128, fold=4, eps=0.05)
    seed = (64.0, 64.0, 0.0, 8.0, 0.3, 0.01, 1)
    a, b = P.pair(p, "fp32", seed_args=seed)
    a.step(2000)
    b.step(2000, P.THREADS)
    check(P, a, b, TOL32, ("phi", "U"))
    da, db = a.diagnostics(), b.diag(64, 64)
    assert np.abs(da["iface_pos"][:4] - db["iface_pos"][:4]).max() < 0.25
    assert db["iface_pos"][0] > 10.0  # the seed grew
    assert abs(da["solid_volume"] - db["solid_volume"]) / db["solid_volume"] < 1e-5


def test_c1_fp64_matches_to_1e10(P):
    p = P.params(nx=128, ny=128, fold=4, eps=0.05)
    a, b = P.pair(p, "fp64", seed_args=(64.0, 64.0, 0.0, 8.0, 0.3, 0.01, 1))
    a.step(400)
    b.step(400, P.THREADS)
    check(P, a, b, TOL64, ("phi", "U"))


# --- 2D coupled with inflow (the 1024^2 workload's boundaries), 5-fold -------
def coupled_inlet(P, n=256):
    return P.params(nx=n, ny=n, flow=1, fold=5, eps=0.03, bc=(1, 0, 0), u_in=0.01, U_in=0.4)


def test_coupled_inlet_fp32(P):
    p = coupled_inlet(P)
    a, b = P.pair(p, "fp32", seed_args=(75.0, 128.0, 0.0, 16.0, 0.4, 0.01, 2))
    a.step(300)
    b.step(300, P.THREADS)
    check(P, a, b, TOL32)
    # populations in the documented common order
    pa, pb = P.decode_pops(a), {k: b.pops(k) for k in "fgh"}
    for k in "fgh":
        assert np.abs(pa[k] - pb[k]).max() < TOL32, k


def test_coupled_inlet_fp64(P):
    p = P.params(nx=96, ny=64, flow=1, fold=5, eps=0.03, bc=(1, 0, 0), u_in=0.02, U_in=0.4,
                 theta0=0.2)
    a, b = P.pair(p, "fp64", seed_args=(40.0, 30.0, 0.0, 9.0, 0.45, 0.01, 3))
    a.step(200)
    b.step(200, P.THREADS)
    check(P, a, b, TOL64)


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
@pytest.mark.parametrize("nx,ny", [(100, 70), (33, 9), (4, 4)])
def test_ragged_periodic_coupled(P, nx, ny, storage):
    p = P.params(nx=nx, ny=ny, flow=1, fold=6, eps=0.02, lam=2.0)
    f = P.seeded_fields(p, seed=nx, radius=min(nx, ny) / 5, u0=0.4, amp_u=0.02)
    a, b = P.pair(p, storage, fields=f)
    # The 4 x 4 grid becomes nearly uniform within ~20 steps; a_s then hangs on
    # noise-level gradients at the |grad phi|^2 = 1e-12 cut-off, where FP32 and
    # FP64 take different branches.  FP32 is compared before that point, FP64
    # over the whole run.
    steps = 10 if (nx == 4 and storage == "fp32") else 150
    a.step(steps)
    b.step(steps, P.THREADS)
    check(P, a, b, TOL32 if storage == "fp32" else TOL64)


def test_walls_body_force_and_literal_flux(P):
    p = P.params(nx=64, ny=40, flow=1, fold=4, eps=0.04, bc=(0, 2, 0), body=(2e-6, 0, 0),
                 literal=1)
    f = P.seeded_fields(p, seed=9, radius=6.0, u0=0.35, amp_u=0.005)
    a, b = P.pair(p, "fp32", fields=f)
    a.step(200)
    b.step(200, P.THREADS)
    check(P, a, b, TOL32)


def test_wall_x_and_inflow_corner_cases(P):
    # x walls + y walls (all four corners bounce) with flow, and inflow with y walls
    for bc in ((2, 2, 0), (1, 2, 0)):
        p = P.params(nx=40, ny=24, flow=1, fold=4, eps=0.03, bc=bc, u_in=0.01, U_in=0.3)
        f = P.seeded_fields(p, seed=4, radius=5.0, u0=0.3, amp_u=0.01)
        a, b = P.pair(p, "fp32", fields=f)
        a.step(120)
        b.step(120, P.THREADS)
        check(P, a, b, TOL32)


# --- 3D: D3Q19 flow, D3Q7 solute and phase field, cubic anisotropy -----------
def test_3d_coupled_inlet_fp32(P):
    p = P.params(dim=3, nx=40, ny=36, nz=20, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.5)
    a, b = P.pair(p, "fp32", seed_args=(14.0, 18.0, 10.0, 6.0, 0.5, 0.01, 4))
    a.step(100)
    b.step(100, P.THREADS)
    check(P, a, b, TOL32, ("phi", "U", "rho", "ux", "uy", "uz"))


def test_3d_fp64_walls(P):
    p = P.params(dim=3, nx=21, ny=18, nz=14, flow=1, fold=0, eps=0.04, bc=(0, 2, 2),
                 body=(1e-6, 0, 0))
    f = P.seeded_fields(p, seed=7, radius=4.0, u0=0.5, amp_u=0.01)
    a, b = P.pair(p, "fp64", fields=f)
    a.step(60)
    b.step(60, P.THREADS)
    check(P, a, b, TOL64, ("phi", "U", "rho", "ux", "uy", "uz"))


def test_3d_fp32_ragged_walls_inlet(P):
    # sizes that are not multiples of the 32 x 8 column or of the z chunk of
    # the z-marching kernel (two chunks, a partial one), walls in y and z
    p = P.params(dim=3, nx=37, ny=19, nz=45, flow=1, fold=0, eps=0.04, bc=(1, 2, 2),
                 u_in=0.004, U_in=0.45)
    f = P.seeded_fields(p, seed=11, radius=5.0, u0=0.45, amp_u=0.004)
    a, b = P.pair(p, "fp32", fields=f)
    a.step(80)
    b.step(80, P.THREADS)
    check(P, a, b, TOL32, ("phi", "U", "rho", "ux", "uy", "uz"))


def test_3d_fp32_walls_periodic_body(P):
    p = P.params(dim=3, nx=21, ny=18, nz=14, flow=1, fold=0, eps=0.04, bc=(0, 2, 2),
                 body=(1e-6, 0, 0))
    f = P.seeded_fields(p, seed=7, radius=4.0, u0=0.5, amp_u=0.01)
    a, b = P.pair(p, "fp32", fields=f)
    a.step(60)
    b.step(60, P.THREADS)
    check(P, a, b, TOL32, ("phi", "U", "rho", "ux", "uy", "uz"))


def test_3d_no_flow_periodic(P):
    p = P.params(dim=3, nx=32, ny=32, nz=32, flow=0, fold=0, eps=0.04)
    a, b = P.pair(p, "fp32", seed_args=(16.0, 16.0, 16.0, 7.0, 0.5, 0.01, 8))
    a.step(150)
    b.step(150, P.THREADS)
    check(P, a, b, TOL32, ("phi", "U"))


# --- the benchmark's workload at full size: 1024^2 coupled with inflow --------
def test_full_size_1024_coupled(P):
    p = coupled_inlet(P, 1024)
    p["U_in"] = 0.4
    a, b = P.pair(p, "fp32", seed_args=(300.0, 512.0, 0.0, 16.0, 0.4, 0.01, 1))
    a.step(64)  # one replay of the step graph
    b.step(64, P.THREADS)
    check(P, a, b, TOL32)


# --- the 3D workload at full size: 256^3 coupled with inflow, FP32 and 16-bit ------
def test_full_size_256_cubed_3d(P):
    # the 256^3 problem in the benchmark's launch configuration (one replay of
    # the step graph), FP32 to 1e-5; the 16-bit storages within the bounds of
    # their 3D storage error (the 48^3 case over 200 steps)
    p = P.params(dim=3, nx=256, ny=256, nz=256, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.3)
    seed = (128.0, 128.0, 128.0, 12.0, 0.3, 0.01, 1)
    b = P.oracle_sim(p)
    b.init_seed(*seed)
    b.step(64, P.THREADS)
    fields = ("phi", "U", "rho", "ux", "uy", "uz")
    bounds = {"fp32": dict.fromkeys(fields, TOL32),
              "fp16": dict(phi=2e-3, U=3e-3, rho=1.3e-5, ux=1e-5, uy=6e-6, uz=6e-6),
              "bf16": dict(phi=0.04, U=0.025, rho=1e-4, ux=8e-5, uy=5e-5, uz=5e-5)}
    for storage, bound in bounds.items():
        a = P.lib_sim(p, storage)
        a.init_seed(*seed)
        a.step(64)
        errs = P.max_errors(a, b, fields)
        for k in fields:
            assert errs[k] < bound[k], (storage, k, errs)
        a.close()


# --- properties of the library path -------------------------------------------------
def test_graph_replay_equals_single_launches(P):
    p = coupled_inlet(P, 128)
    a = P.lib_sim(p)
    b = P.lib_sim(p)
    for s in (a, b):
        s.init_seed(40.0, 64.0, 0.0, 10.0, 0.4, 0.01, 6)
    a.step(131)  # odd start + graph replays + remainder
    for _ in range(131):
        b.step(1)
    assert np.array_equal(a.state(), b.state())


def test_checkpoint_restart_is_bitwise(P):
    p = coupled_inlet(P, 96)
    a = P.lib_sim(p)
    a.init_seed(30.0, 48.0, 0.0, 8.0, 0.4, 0.01, 7)
    a.step(70)
    st = a.state()
    a.step(70)
    final = a.state()
    da = a.diagnostics()
    b = P.lib_sim(p)
    b.load_state(st)
    b.step(70)
    assert np.array_equal(b.state(), final)
    # the restored run measures from the seed centre (not the grid centre) and
    # its solute drift from the total at initialisation, as the uninterrupted
    # run does
    db = b.diagnostics()
    assert db["step"] == da["step"] == 140
    np.testing.assert_array_equal(db["iface_pos"], da["iface_pos"])
    assert db["solute_drift_rel"] == da["solute_drift_rel"]
    assert da["solute_drift_rel"] != 0.0


def test_conservation_on_the_gpu(P):
    p = P.params(nx=128, ny=128, flow=1, fold=4, eps=0.05)
    a = P.lib_sim(p)
    f = P.seeded_fields(p, seed=3, radius=10.0, u0=0.3, amp_u=0.01)
    a.init_fields(*f[:3], f[3][0], f[3][1])
    d0 = a.diagnostics()
    a.step(2000)
    d1 = a.diagnostics()
    assert abs(d1["solute_drift_rel"]) < 1e-6, d1
    assert abs(d1["mass_total"] / d0["mass_total"] - 1) < 1e-6
    assert d1["step"] == 2000 and d1["nonfinite"] == 0


def test_diagnostics_match_the_oracle(P):
    p = coupled_inlet(P, 128)
    a, b = P.pair(p, "fp32", seed_args=(50.0, 64.0, 0.0, 10.0, 0.4, 0.01, 2))
    a.step(100)
    b.step(100, P.THREADS)
    da, db = a.diagnostics(), b.diag(50, 64)
    for k in ("solute_total", "mass_total", "solid_volume", "r_eq", "max_u"):
        assert abs(da[k] - db[k]) <= 1e-5 * max(1.0, abs(db[k])), (k, da[k], db[k])
    assert np.abs(da["iface_pos"] - db["iface_pos"]).max() < 0.25


def test_empty_step_and_state_errors(P):
    import paper_2206_02145_gb300 as L
    p = P.params(nx=16, ny=16)
    a = P.lib_sim(p)
    with pytest.raises(L.LbpfError) as e:
        a.step(1)  # before init
    assert e.value.code == L.ESTATE
    a.init_seed(8.0, 8.0, 0.0, 3.0, 0.3, 0.0, 1)
    before = a.state()
    a.step(0)
    assert np.array_equal(a.state(), before)
    with pytest.raises(L.LbpfError):
        a.step(-1)
    b = P.lib_sim(P.params(nx=16, ny=17))
    with pytest.raises(L.LbpfError) as e:
        b.load_state(before)
    assert e.value.code == L.EINVAL


def test_nonfinite_is_reported(P):
    import paper_2206_02145_gb300 as L
    p = P.params(nx=16, ny=16)
    a = P.lib_sim(p)
    phi = np.full((16, 16), -1.0)
    phi[3, 4] = np.nan
    a.init_fields(phi, np.full((16, 16), 0.3))
    a.step(2)
    with pytest.raises(L.LbpfError) as e:
        a.diagnostics()
    assert e.value.code == L.ENONFINITE
    with pytest.raises(L.LbpfError):  # sticky
        a.step(1)
