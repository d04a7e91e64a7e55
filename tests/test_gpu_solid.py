"""GPU parity of solid nodes (walls and obstacles) against the oracle, and
their invariants on the device: rows of solid nodes reproduce the domain
walls, solid nodes keep their state, batching and restart are unchanged by a
mask, and the rejections of the C ABI."""
import math

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


@pytest.fixture(scope="module")
def L():
    import paper_2206_02145_gb300 as lib
    return lib


def baffle(nx, ny, x0, y0, y1, w=2):
    m = np.zeros((ny, nx), np.uint8)
    m[y0:y1, x0:x0 + w] = 1
    return m


def inflow_case(P, nx=128, ny=96):
    return P.params(nx=nx, ny=ny, flow=1, fold=5, eps=0.03, bc=(1, 0, 0), u_in=0.01, U_in=0.4)


def masked_pair(P, p, storage, mask, seed):
    a, b = P.pair(p, storage, seed_args=seed)
    a.set_solid(mask)
    b.set_solid(mask)
    return a, b


@pytest.mark.parametrize("storage,tol", [("fp64", TOL64), ("fp32", TOL32)])
def test_baffle_in_the_inflow_matches_oracle(P, L, storage, tol):
    p = inflow_case(P)
    mask = baffle(128, 96, 20, 30, 66) | baffle(128, 96, 90, 5, 12, 3)
    a, b = masked_pair(P, p, storage, mask, (60.0, 48.0, 0.0, 10.0, 0.4, 0.01, 2))
    a.step(300)
    b.step(300, P.THREADS)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < tol, errs
    pa, pb = P.decode_pops(a), {k: b.pops(k) for k in "fgh"}
    for k in "fgh":
        assert np.abs(pa[k] - pb[k]).max() < tol, k
    assert np.abs(a.fields(("uy",))["uy"]).max() > 1e-4  # deflected by the baffle


def test_ragged_grid_obstacle_near_every_edge(P, L):
    # obstacles in edge tiles and across the periodic wrap of a ragged grid
    p = P.params(nx=70, ny=45, flow=1, fold=4, eps=0.04, body=(2e-6, 1e-6, 0.0))
    m = np.zeros((45, 70), np.uint8)
    m[0:3, 10:14] = 1      # at the lower edge (wraps to the top)
    m[40:45, 66:70] = 1    # corner
    m[20:24, 0:2] = 1      # left edge
    m[30, 33] = 1          # a single node
    a, b = masked_pair(P, p, "fp64", m, (35.0, 22.0, 0.0, 8.0, 0.35, 0.01, 5))
    a.step(200)
    b.step(200, P.THREADS)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < TOL64, errs


def test_solid_rows_reproduce_the_domain_walls(P, L):
    nx, ny = 96, 62
    pw = P.params(nx=nx, ny=ny, flow=1, fold=4, eps=0.04, bc=(0, 2, 0), body=(2e-6, 0.0, 0.0))
    pm = P.params(nx=nx, ny=ny + 2, flow=1, fold=4, eps=0.04, bc=(0, 0, 0),
                  body=(2e-6, 0.0, 0.0))
    rng = np.random.default_rng(9)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    phi = np.tanh((9.0 - np.hypot(x - 40.3, y - 4.2)) / (math.sqrt(2) * 2.0))
    phi += 0.01 * rng.uniform(-1, 1, phi.shape)
    U = 0.35 + 0.01 * rng.uniform(-1, 1, phi.shape)
    pad = lambda f, v: np.concatenate([np.full((1, nx), v), f, np.full((1, nx), v)])
    for storage, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        a = P.lib_sim(pw, storage)
        a.init_fields(phi, U)
        b = P.lib_sim(pm, storage)
        m = np.zeros((ny + 2, nx), np.uint8)
        m[0] = m[-1] = 1
        b.set_solid(m)
        b.init_fields(pad(phi, -1.0), pad(U, 0.35))
        a.step(300)
        b.step(300)
        fa, fb = a.fields(), b.fields()
        for k in ("phi", "U", "rho", "ux", "uy"):
            assert np.abs(fa[k] - fb[k][1:-1]).max() < tol, (storage, k)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_storage_with_obstacles(P, L, storage):
    p = inflow_case(P)
    mask = baffle(128, 96, 20, 30, 66)
    a, b = masked_pair(P, p, storage, mask, (60.0, 48.0, 0.0, 10.0, 0.4, 0.01, 2))
    s0 = a.fields()
    a.step(300)
    b.step(300, P.THREADS)
    errs = P.max_errors(a, b)
    bounds = dict(phi=8e-3, U=9e-3, rho=4e-5, ux=4e-5, uy=3e-5) if storage == "fp16" else \
        dict(phi=0.08, U=0.08, rho=4e-4, ux=3e-4, uy=2e-4)
    for k, bound in bounds.items():
        assert errs[k] < bound, (k, errs)
    s1 = a.fields()
    sel = mask.astype(bool)
    for k in ("phi", "U", "rho"):  # the solid nodes kept their state
        assert np.array_equal(s1[k][sel], s0[k][sel]), k


def test_graph_batch_and_restart_with_a_mask(P, L):
    p = inflow_case(P, 100, 72)
    seed = (60.0, 36.0, 0.0, 9.0, 0.4, 0.01, 3)
    mask = baffle(100, 72, 15, 20, 50)
    one = P.lib_sim(p, "fp32")
    one.set_solid(mask)
    one.init_seed(*seed)
    for _ in range(70):
        one.step(1)  # launch by launch
    g = P.lib_sim(p, "fp32")
    g.set_solid(mask)
    g.init_seed(*seed)
    g.step(70)  # through the step graph
    assert np.array_equal(one.state(), g.state())
    # restart: the state of step 70, 30 more steps, against 30 more steps
    r = P.lib_sim(p, "fp32")
    r.set_solid(mask)
    r.load_state(g.state())
    g.step(30)
    r.step(30)
    assert np.array_equal(g.state(), r.state())
    # the batched step: a masked and a free instance side by side evolve bit
    # for bit like each stepped alone; removing the mask is picked up too
    kw = dict(dim=2, nx=100, ny=72, bc=(1, 0, 0), flow=1, fold=5, eps_aniso=0.03,
              u_inlet=0.01, u0_inlet=0.4, storage=L.FP32)
    bt = L.Batch([kw, kw], [seed, seed], None)
    bt.instance(0).set_solid(mask)
    bt.step(100)
    free = P.lib_sim(p, "fp32")
    free.init_seed(*seed)
    free.step(100)
    masked = P.lib_sim(p, "fp32")
    masked.set_solid(mask)
    masked.init_seed(*seed)
    masked.step(100)
    assert np.array_equal(bt.instance(0).state(), masked.state())
    assert np.array_equal(bt.instance(1).state(), free.state())
    bt.instance(0).set_solid(None)
    masked.set_solid(None)
    bt.step(30)
    free.step(30)
    masked.step(30)
    assert np.array_equal(bt.instance(0).state(), masked.state())
    assert np.array_equal(bt.instance(1).state(), free.state())
    bt.close()


def test_full_size_baffle_sample(P, L):
    # the 1024^2 inflow problem with a baffle in front of the inlet, in the
    # launch configuration of the benchmark, against the oracle over 10 steps
    p = inflow_case(P, 1024, 1024)
    mask = baffle(1024, 1024, 150, 352, 672, 4)
    a, b = masked_pair(P, p, "fp32", mask, (300.0, 512.0, 0.0, 16.0, 0.4, 0.01, 1))
    a.step(10)
    b.step(10, P.THREADS)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < TOL32, errs


def test_rejections(P, L):
    p = inflow_case(P, 40, 30)
    a = P.lib_sim(p, "fp32")
    m = np.zeros((30, 40), np.uint8)
    m[5, 0] = 1
    with pytest.raises(L.LbpfError) as e:
        a.set_solid(m)
    assert e.value.code == L.EINVAL
    m[5, 0] = 0
    m[5, 39] = 1
    with pytest.raises(L.LbpfError) as e:
        a.set_solid(m)
    assert e.value.code == L.EINVAL
    # 3D: the inlet and outlet columns (x = 0 and nx - 1 of every row) too
    q = P.lib_sim(P.params(dim=3, nx=16, ny=16, nz=16, fold=0, eps=0.04, flow=1,
                           bc=(1, 0, 0), u_in=0.005, U_in=0.3), "fp32")
    m3 = np.zeros((16, 16, 16), np.uint8)
    m3[9, 3, 15] = 1
    with pytest.raises(L.LbpfError) as e:
        q.set_solid(m3)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.LbpfError) as e:  # a mask of the wrong size
        q.set_solid(np.zeros(16 ** 2, np.uint8))
    assert e.value.code == L.EINVAL
    a.set_solid(None)  # removing a mask that is not there is fine


# ---- 3D: D3Q19 flow, D3Q7 solute and phase field, the z-marching kernel ------
F3 = ("phi", "U", "rho", "ux", "uy", "uz")


def obstacles3(nx, ny, nz):
    """A baffle plate across the inflow, a block, and a bar across the
    periodic wrap in y and z (the solid nodes of Sec. 3.1.2 / 3.2 in 3D)."""
    m = np.zeros((nz, ny, nx), np.uint8)
    m[4:nz - 6, 6:ny - 10, 9:11] = 1       # plate normal to x
    m[nz // 2:nz // 2 + 3, 2:5, 30:33] = 1  # block
    m[0:2, ny - 2:ny, 20:24] = 1            # bar in the corner of the wrap
    m[nz - 1, 0, 25] = 1                    # ... and its other side
    return m


@pytest.mark.parametrize("storage,tol", [("fp64", TOL64), ("fp32", TOL32)])
@pytest.mark.parametrize("collision", ["bgk", "chm"])
def test_3d_obstacles_in_the_inflow_match_oracle(P, L, storage, tol, collision):
    # sizes off the 32 x 4 column and the 8-plane chunk, obstacles in edge
    # columns and chunks and across the wrap
    nx, ny, nz = 44, 26, 21
    p = P.params(dim=3, nx=nx, ny=ny, nz=nz, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.45)
    mask = obstacles3(nx, ny, nz)
    seed = (24.0, 13.0, 10.0, 5.0, 0.45, 0.01, 3)
    if collision == "chm":
        import oracle
        a = L.Sim(dim=3, nx=nx, ny=ny, nz=nz, bc=(1, 0, 0), flow=1, storage=P.STORAGE[storage],
                  fold=0, eps_aniso=0.04, u_inlet=0.005, u0_inlet=0.45, collision=L.COLL_CHM)
        b = oracle.Oracle(oracle.Params(dim=3, nx=nx, ny=ny, nz=nz, bc=(1, 0, 0), flow=1,
                                        fold=0, eps=0.04, u_inlet=0.005, u0_inlet=0.45,
                                        collision=1))
    else:
        a, b = P.lib_sim(p, storage), P.oracle_sim(p)
    a.set_solid(mask)
    b.set_solid(mask)
    a.init_seed(*seed)
    b.init_seed(*seed)
    a.step(80)
    b.step(80, P.THREADS)
    errs = P.max_errors(a, b, F3)
    assert max(errs.values()) < tol, errs
    pa, pb = P.decode_pops(a), {k: b.pops(k) for k in "fgh"}
    for k in "fgh":
        assert np.abs(pa[k] - pb[k]).max() < tol, k
    f = a.fields(("uy", "uz"))
    assert np.abs(f["uy"]).max() > 1e-5  # deflected by the obstacles


def test_3d_walls_with_flow_and_a_crystal_on_a_ragged_grid(P, L):
    # walls in y and z, a periodic x, a body force, a crystal touching an
    # obstacle; FP64 to the oracle
    nx, ny, nz = 37, 19, 27
    p = P.params(dim=3, nx=nx, ny=ny, nz=nz, flow=1, fold=0, eps=0.04, bc=(0, 2, 2),
                 body=(3e-6, 0.0, 1e-6))
    m = np.zeros((nz, ny, nx), np.uint8)
    m[10:14, 0:4, 15:19] = 1
    m[20:27, 12:15, 2:4] = 1
    m[5, 9, 0] = m[5, 9, nx - 1] = 1  # across the periodic wrap in x
    f = P.seeded_fields(p, seed=21, radius=5.0, u0=0.4, amp_u=0.003)
    a, b = P.lib_sim(p, "fp64"), P.oracle_sim(p)
    a.set_solid(m)
    b.set_solid(m)
    a.init_fields(f[0], f[1], f[2], *f[3])
    b.init_fields(f[0], f[1], f[2], *f[3])
    a.step(60)
    b.step(60, P.THREADS)
    errs = P.max_errors(a, b, F3)
    assert max(errs.values()) < TOL64, errs


def test_3d_solid_planes_reproduce_the_domain_walls(P, L):
    # planes of solid nodes at y = 0 and y = ny + 1 of a periodic domain act
    # as the walls of LBPF_BC_WALL in y (bounce-back of f, g, h and the
    # gradient's nearest-node copy), with a crystal touching the wall
    nx, ny, nz = 36, 22, 18
    kw = dict(dim=3, nx=nx, nz=nz, flow=1, fold=0, eps=0.04, body=(2e-6, 0.0, 0.0))
    pw = P.params(ny=ny, bc=(0, 2, 0), **kw)
    pm = P.params(ny=ny + 2, bc=(0, 0, 0), **kw)
    rng = np.random.default_rng(4)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    phi = np.tanh((6.0 - np.sqrt((x - 17.2) ** 2 + (y - 2.4) ** 2 + (z - 9.1) ** 2))
                  / (math.sqrt(2) * 2.0))
    phi += 0.01 * rng.uniform(-1, 1, phi.shape)
    U = 0.35 + 0.01 * rng.uniform(-1, 1, phi.shape)
    pad = lambda f, v: np.concatenate([np.full((nz, 1, nx), v), f, np.full((nz, 1, nx), v)],
                                      axis=1)
    for storage, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        a = P.lib_sim(pw, storage)
        a.init_fields(phi, U)
        b = P.lib_sim(pm, storage)
        m = np.zeros((nz, ny + 2, nx), np.uint8)
        m[:, 0] = m[:, -1] = 1
        b.set_solid(m)
        b.init_fields(pad(phi, -1.0), pad(U, 0.35))
        a.step(120)
        b.step(120)
        fa, fb = a.fields(F3), b.fields(F3)
        for k in F3:
            assert np.abs(fa[k] - fb[k][:, 1:-1]).max() < tol, (storage, k)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_3d_16bit_storage_with_obstacles(P, L, storage):
    nx, ny, nz = 48, 40, 32
    p = P.params(dim=3, nx=nx, ny=ny, nz=nz, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.3)
    mask = obstacles3(nx, ny, nz)
    a, b = P.lib_sim(p, storage), P.oracle_sim(p)
    a.set_solid(mask)
    b.set_solid(mask)
    seed = (26.0, 20.0, 16.0, 7.0, 0.3, 0.01, 1)
    a.init_seed(*seed)
    b.init_seed(*seed)
    s0 = a.fields(F3)
    a.step(100)
    b.step(100, P.THREADS)
    errs = P.max_errors(a, b, F3)
    # the 3D storage bounds of the plain problem (test_gpu_chm, test_gpu_precision)
    bounds = dict(phi=2e-3, U=3e-3, rho=1.3e-5, ux=1e-5, uy=6e-6, uz=6e-6) if storage == "fp16" \
        else dict(phi=0.04, U=0.025, rho=1e-4, ux=8e-5, uy=5e-5, uz=5e-5)
    for k, bound in bounds.items():
        assert errs[k] < bound, (k, errs)
    s1 = a.fields(F3)
    sel = mask.astype(bool)
    for k in ("phi", "U", "rho"):  # the solid nodes kept their state
        assert np.array_equal(s1[k][sel], s0[k][sel]), k


def test_3d_graph_restart_and_mask_removal(P, L):
    nx, ny, nz = 40, 24, 20
    p = P.params(dim=3, nx=nx, ny=ny, nz=nz, flow=1, fold=0, eps=0.04, bc=(1, 0, 0),
                 u_in=0.005, U_in=0.4)
    mask = obstacles3(nx, ny, nz)
    seed = (22.0, 12.0, 10.0, 5.0, 0.4, 0.01, 6)
    one = P.lib_sim(p, "fp32")
    one.set_solid(mask)
    one.init_seed(*seed)
    for _ in range(70):
        one.step(1)  # launch by launch
    g = P.lib_sim(p, "fp32")
    g.set_solid(mask)
    g.init_seed(*seed)
    g.step(70)  # graphs
    assert np.array_equal(one.state(), g.state())
    r = P.lib_sim(p, "fp32")
    r.set_solid(mask)
    r.load_state(g.state())
    g.step(30)
    r.step(30)
    assert np.array_equal(g.state(), r.state())
    # removing the mask: the plain kernel continues from the same state
    free = P.lib_sim(p, "fp32")
    free.load_state(g.state())
    g.set_solid(None)
    g.step(20)
    free.step(20)
    assert np.array_equal(g.state(), free.state())

