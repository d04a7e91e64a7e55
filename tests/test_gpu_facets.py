"""GPU parity of the polygon seed and of the crystal-shape measurement
(Sec. 3.1.2, Sec. 3.2) against the oracle.

The support values are FP64 maxima over the phi = 0 contour; measured by the
device on a field and by the oracle on the same field read back in FP64, they
agree to rounding of the last bit, and so do the side centres, the centre
and the side lengths built from them.  Where the two sides evolve the field
themselves (FP64 storage), the fields differ by the step's rounding only."""
import math

import numpy as np
import pytest

from oracle import facets as F

pytestmark = pytest.mark.gpu


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


def hex_case(P, n=128, flow=0, u_in=0.0):
    # 6-fold anisotropy with its fast directions at theta0: the sides' normals
    # sit halfway between them
    return P.params(nx=n, ny=n, flow=flow, fold=6, eps=0.03, theta0=0.1,
                    bc=(1, 0, 0) if flow else (0, 0, 0), u_in=u_in, U_in=0.3 if flow else 0.0)


def same_field(L, sim, normals):
    got = sim.facets(normals)
    want = F.facets(sim.fields(("phi",))["phi"], normals)
    return got, want


def assert_same_shape(got, want, tol):
    assert got["points"] == want["points"]
    for k in ("support", "side_centre", "centre", "L"):
        assert np.abs(np.asarray(got[k]) - np.asarray(want[k])).max() < tol, k
    for k in ("L_avg", "Q", "width", "height", "aspect"):
        assert abs(got[k] - want[k]) < tol, k


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_polygon_seed_matches_oracle(P, L, storage, tol):
    p = hex_case(P, 96, flow=1, u_in=0.01)
    nrm, d = L.hexagonal_seed(70.0, 0.1 + math.pi / 6)
    a = P.lib_sim(p, storage)
    b = P.oracle_sim(p)
    a.init_polygon(47.3, 44.8, nrm, d, 0.3, 0.01, 5)
    b.init_polygon(47.3, 44.8, nrm, d, 0.3, 0.01, 5)
    errs = P.max_errors(a, b)
    assert max(errs.values()) < tol, errs
    pa, pb = P.decode_pops(a), {k: b.pops(k) for k in "fgh"}
    for k in "fgh":
        assert np.abs(pa[k] - pb[k]).max() < tol, k


def test_polygon_seed_shape_at_start(P, L):
    # the measured sides of the seed are the polygon's own (plane geometry)
    p = hex_case(P, 128)
    nrm, d = L.hexagonal_seed(90.0, 0.1 + math.pi / 6)
    a = P.lib_sim(p, "fp32")
    a.init_polygon(63.4, 61.7, nrm, d, 0.2, 0.0, 1)
    r = a.facets(nrm)
    assert np.abs(r["L"] - d).max() < 0.02, r["L"]
    assert np.abs(r["centre"] - [63.4, 61.7]).max() < 0.02
    assert abs(r["Q"] - 1.0) < 2e-3


@pytest.mark.parametrize("storage", ["fp64", "fp32", "fp16", "bf16"])
def test_facets_of_the_same_field_match_oracle(P, L, storage):
    p = hex_case(P, 128, flow=1, u_in=0.01)
    nrm, d = L.rhombic_seed(100.0, 0.1)
    a = P.lib_sim(p, storage)
    a.init_polygon(60.2, 64.9, nrm, d, 0.3, 0.01, 2)
    a.step(300)
    meas = L.hexagon_normals(0.1 + math.pi / 6)
    got, want = same_field(L, a, meas)
    assert got["points"] > 50
    assert_same_shape(got, want, 1e-9)


def test_facets_follow_the_oracle_run(P, L):
    # both sides evolve the rhombic seed for 400 steps in FP64
    p = hex_case(P, 112)
    nrm, d = L.rhombic_seed(90.0, 0.1 + math.pi / 2)
    a, b = P.lib_sim(p, "fp64"), P.oracle_sim(p)
    for s in (a, b):
        s.init_polygon(55.5, 57.25, nrm, d, 0.35, 0.01, 3)
    a.step(400)
    b.step(400, P.THREADS)
    meas = L.hexagon_normals(0.1 + math.pi / 6)
    got = a.facets(meas)
    want = F.facets(b.fields()["phi"], meas)
    assert_same_shape(got, want, 1e-8)


@pytest.mark.parametrize("nx,ny", [(33, 9), (100, 70), (45, 128)])
def test_facets_ragged_grids_and_edge_contact(P, L, nx, ny):
    # a crystal that runs off the grid: the contour ends at the edges
    p = P.params(nx=nx, ny=ny, fold=6, eps=0.03)
    nrm, d = L.hexagonal_seed(0.9 * 6 * min(nx, ny) / 2, 0.0)
    a = P.lib_sim(p, "fp64")
    a.init_polygon(nx / 2 + 0.3, ny / 2 - 0.2, nrm, d, 0.2, 0.0, 1)
    a.step(20)
    got, want = same_field(L, a, nrm)
    assert got["points"] > 0
    assert_same_shape(got, want, 1e-9)


def test_full_size_hexagon_with_inflow(P, L):
    # the 1024^2 inflow problem with a hexagonal seed, in the launch
    # configuration of the benchmark; the device's measurement of its own
    # field against the oracle's measurement of that field
    p = hex_case(P, 1024, flow=1, u_in=0.01)
    nrm, d = L.hexagonal_seed(120.0, 0.1 + math.pi / 6)
    a = P.lib_sim(p, "fp32")
    a.init_polygon(300.0, 512.0, nrm, d, 0.4, 0.01, 1)
    a.step(2000)
    got, want = same_field(L, a, nrm)
    assert_same_shape(got, want, 1e-9)
    assert got["L_avg"] > d[0]  # it grew


def test_no_crystal_and_invalid_arguments(P, L):
    p = P.params(nx=40, ny=30)
    a = P.lib_sim(p, "fp32")
    with pytest.raises(L.LbpfError) as e:
        a.facets(L.hexagon_normals())
    assert e.value.code == L.ESTATE
    a.init_fields(np.full((30, 40), -1.0), np.full((30, 40), 0.2))
    r = a.facets(L.hexagon_normals())
    assert r["points"] == 0 and np.isnan(r["L_avg"]) and np.all(np.isnan(r["L"]))
    want = F.facets(np.full((30, 40), -1.0), L.hexagon_normals())
    assert want["points"] == 0
    bad = [L.hexagon_normals()[:5],                       # odd count
           L.hexagon_normals()[::-1],                     # clockwise
           L.hexagon_normals() * 1.01,                    # not unit
           np.concatenate([L.hexagon_normals()[:3], L.hexagon_normals(0.2)[3:]])]  # not opposite
    for nrm in bad:
        with pytest.raises(L.LbpfError) as e:
            a.facets(nrm)
        assert e.value.code == L.EINVAL
    q = P.lib_sim(P.params(dim=3, nx=16, ny=16, nz=16, fold=0, eps=0.04), "fp32")
    with pytest.raises(L.LbpfError) as e:
        q.init_polygon(8.0, 8.0, L.hexagon_normals(), np.full(6, 4.0))
    assert e.value.code == L.EINVAL


def test_enqueue_measures_the_state_at_its_point_of_the_stream(P, L):
    p = hex_case(P, 128)
    nrm, d = L.hexagonal_seed(80.0, 0.1 + math.pi / 6)
    a = P.lib_sim(p, "fp32")
    a.init_polygon(64.0, 64.0, nrm, d, 0.35, 0.01, 4)
    a.step(100)
    want = a.facets(nrm)
    L.lbpf_facets_enqueue(a.h, nrm)
    a.step(300)  # queued behind the measurement
    got = L.lbpf_facets_collect(a.h)
    assert got["points"] == want["points"]
    for k in ("support", "centre", "L"):  # the same state: bit for bit
        assert np.array_equal(got[k], want[k]), k
    later = a.facets(nrm)
    assert later["L_avg"] > got["L_avg"]
    with pytest.raises(L.LbpfError) as e:
        L.lbpf_facets_collect(a.h)
    assert e.value.code == L.ESTATE
