"""Batched sweep: many 2D instances of different sizes and parameters
advanced by one persistent launch per step.  A batched instance must evolve
bit for bit like the same instance stepped alone (the per-tile work is the
same code), whichever tile shape the tuner picks, and match the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import paper_2206_02145_gb300
    return paper_2206_02145_gb300


def sweep(storage, n=5, seed=4):
    """Seeded uneven sweep: sizes, supersaturation, seed radius, inflow, fold, eps."""
    rng = np.random.default_rng(seed)
    params, seeds = [], []
    sizes = [(100, 70), (64, 64), (130, 40), (256, 96), (33, 9), (48, 200)][:n]
    for i, (nx, ny) in enumerate(sizes):
        u0 = float(rng.uniform(0.1, 0.6))
        r = float(rng.uniform(2.0, max(2.5, min(nx, ny) / 4)))
        params.append(dict(dim=2, nx=nx, ny=ny, flow=1, storage=storage,
                           fold=int(rng.choice([4, 5])), eps_aniso=float(rng.uniform(0.02, 0.06)),
                           bc=(1, 0, 0), u_inlet=float(rng.uniform(0, 0.02)), u0_inlet=u0))
        seeds.append((0.3 * nx, 0.5 * ny, 0.0, r, u0, 0.01, 100 + i))
    return params, seeds


@pytest.mark.parametrize("storage_name", ["FP32", "FP16_SHIFTED"])
def test_batch_equals_single_instances_bitwise(L, storage_name):
    storage = getattr(L, storage_name)
    params, seeds = sweep(storage)
    b = L.Batch(params, seeds)
    b.step(131)  # tuning (48) + graph replays + remainder, odd total
    singles = []
    for p, s in zip(params, seeds):
        sim = L.Sim(**p)
        sim.init_seed(*s)
        sim.step(131)
        singles.append(sim)
    for i, sim in enumerate(singles):
        assert np.array_equal(b.instance(i).state(), sim.state()), i
    t = b.tuning()
    # four tile shapes, each in the two tile orders
    assert t["tuned"] and t["tile_rows"] in (2, 4, 8) and len(t["ms_per_step"]) == 8
    d = b.diagnostics()
    assert all(x["step"] == 131 and x["nonfinite"] == 0 for x in d)


def test_batched_instance_matches_oracle(L):
    import _pairs as P
    params, seeds = sweep(L.FP32, n=4)
    b = L.Batch(params, seeds)
    b.step(100)
    k = 3  # the 256 x 96 instance
    p = params[k]
    o = P.oracle_sim(P.params(nx=p["nx"], ny=p["ny"], flow=1, fold=p["fold"], eps=p["eps_aniso"],
                              bc=(1, 0, 0), u_in=p["u_inlet"], U_in=p["u0_inlet"]))
    o.init_seed(*seeds[k])
    o.step(100, P.THREADS)
    errs = P.max_errors(b.instance(k), o)
    assert max(errs.values()) < 1e-5, errs


def test_batch_picks_up_reinitialised_instance(L):
    params, seeds = sweep(L.FP32, n=3)
    b = L.Batch(params, seeds)
    b.step(30)
    inst = b.instance(1)
    new_seed = (20.0, 30.0, 0.0, 9.0, 0.5, 0.01, 77)
    inst.init_seed(*new_seed)  # changes U_ref: the batch must rebuild its tables
    b.instance(0).init_seed(*seeds[0])
    b.instance(2).init_seed(*seeds[2])
    b.step(40)
    sim = L.Sim(**params[1])
    sim.init_seed(*new_seed)
    sim.step(40)
    assert np.array_equal(b.instance(1).state(), sim.state())


@pytest.mark.parametrize("storage_name", ["FP32", "BF16_SHIFTED"])
def test_batch_with_obstacles_equals_single_instances_bitwise(L, storage_name):
    # obstacles in some instances (edge tiles, across the periodic wrap, a
    # single node): each variant's per-tile solid flags are its own
    storage = getattr(L, storage_name)
    params, seeds = sweep(storage)
    masks = {}
    for i in (0, 3, 4):
        nx, ny = params[i]["nx"], params[i]["ny"]
        m = np.zeros((ny, nx), np.uint8)
        m[ny // 4:3 * ny // 4, nx // 5:nx // 5 + 2] = 1
        m[0, nx // 2] = 1          # wraps to the top row
        m[ny - 1, 3 * nx // 4] = 1
        masks[i] = m
    b = L.Batch(params, seeds)
    for i, m in masks.items():
        b.instance(i).set_solid(m)
    b.step(131)
    for i, (p, s) in enumerate(zip(params, seeds)):
        sim = L.Sim(**p)
        if i in masks:
            sim.set_solid(masks[i])
        sim.init_seed(*s)
        sim.step(131)
        assert np.array_equal(b.instance(i).state(), sim.state()), i


def test_full_size_sweep_sampled_instances_match_oracle(L):
    # the benchmark's sweep (64 instances of 256^2..768^2, FP16 storage) over
    # the tuner's 24 steps and one graph replay; its smallest and largest
    # instance against the oracle within the 2D FP16 storage bounds
    import bench
    import _pairs as P
    params, seeds = bench.sweep_members(64, 4)
    params = [dict(p, storage=L.FP16_SHIFTED) for p in params]
    b = L.Batch(params, seeds)
    b.step(88)
    sizes = [p["nx"] for p in params]
    for k in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        p = params[k]
        o = P.oracle_sim(P.params(nx=p["nx"], ny=p["ny"], flow=1, fold=p["fold"],
                                  eps=p["eps_aniso"], bc=(1, 0, 0), u_in=p["u_inlet"],
                                  U_in=p["u0_inlet"]))
        o.init_seed(*seeds[k])
        o.step(88, P.THREADS)
        errs = P.max_errors(b.instance(k), o)
        for f, bound in dict(phi=8e-3, U=9e-3, rho=4e-5, ux=4e-5, uy=3e-5).items():
            assert errs[f] < bound, (k, f, errs)
    assert b.tuning()["tuned"]
    b.close()


def test_batch_rejects_mixed_instances(L):
    params, seeds = sweep(L.FP32, n=2)
    params[1]["storage"] = L.FP16_SHIFTED
    with pytest.raises(L.LbpfError):
        L.Batch(params, seeds)
