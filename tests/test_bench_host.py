"""Host logic of bench.py (no GPU): workload resolution, the algorithmic bytes
per node update that the HBM roofline divides by, the seeded sweep of the
batched workload, and the rule that a profile's DRAM traffic is reported
only while the kernel's sources still match the digest it was taken with."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_workload_resolves(bench):
    for name in bench.WORKLOADS:
        w = bench.workload(name)
        assert w["nodes"] > 0 and w["bytes_per_lup"] > 0 and w["desc"], name


@pytest.mark.parametrize("name,bytes_per_lup", [
    # 2D coupled: 27 populations read and written + the phi ring read and written
    ("c2", 27 * 4 * 2 + 8), ("f3", 27 * 4 * 2 + 8),
    # + the solid mask byte
    ("f2", 27 * 4 * 2 + 8 + 1),
    # 16-bit storage + the per-node g reference (own read, neighbours' read, write)
    ("c2_fp16", 27 * 2 * 2 + 8 + 6), ("c4", 27 * 2 * 2 + 8 + 6),
    # 2D no flow
    ("c1", 18 * 4 * 2 + 8),
    # 3D: 19 + 7 + 7 populations
    ("c3", 33 * 4 * 2 + 8), ("f3_3d", 33 * 4 * 2 + 8), ("c3_fp16", 33 * 2 * 2 + 8 + 6),
    ("c3s_fp16", 33 * 2 * 2 + 8 + 6),
])
def test_algorithmic_bytes_per_node_update(bench, name, bytes_per_lup):
    assert bench.workload(name)["bytes_per_lup"] == bytes_per_lup


def test_fp16_arm_counts_the_fp16_node_update(bench):
    # the default line's FP16-storage arm takes the C2 grid's bytes in FP16
    # storage for its own roofline, the bytes of the c2_fp16 workload
    c2 = bench.workload("c2")
    assert bench.lup_bytes(c2, "fp16") == bench.workload("c2_fp16")["bytes_per_lup"] == 122
    assert bench.lup_bytes(c2, "fp32") == c2["bytes_per_lup"] == 224


def test_sweep_is_seeded_and_within_its_ranges(bench):
    a = bench.sweep_members(64, 4)
    b = bench.sweep_members(64, 4)
    assert a == b
    params, seeds = a
    assert len(params) == len(seeds) == 64
    for p, s in zip(params, seeds):
        n = p["nx"]
        assert p["ny"] == n and 256 <= n <= 768
        assert 0.1 <= p["u0_inlet"] <= 0.6 and 0.0 <= p["u_inlet"] <= 0.02
        assert p["fold"] in (4, 5) and 0.02 <= p["eps_aniso"] <= 0.06
        assert 4.0 <= s[3] <= min(24.0, n / 5) and s[4] == p["u0_inlet"]
    assert bench.sweep_members(64, 5) != a
    w = bench.workload("c4")
    assert w["nodes"] == sum(p["nx"] * p["ny"] for p in params)


def test_sweep_shards_over_ranks(bench):
    # N ranks advance disjoint shards of one sweep of N x 64 instances; the
    # whole-job node count is the same on every rank; N = 1 is the plain sweep
    one = bench.workload("c4")
    assert one["nodes_all"] == one["nodes"]
    assert one["members"] == bench.sweep_members(64, 4)
    world = 3
    full = bench.sweep_members(64 * world, 4)
    shards = [bench.workload("c4", r, world) for r in range(world)]
    seen = sorted(s for w in shards for s in w["members"][1])
    assert seen == sorted(full[1])  # every instance exactly once
    for w in shards:
        assert len(w["members"][0]) == 64
        assert w["nodes_all"] == sum(p["nx"] * p["ny"] for p in full[0])
    assert sum(w["nodes"] for w in shards) == shards[0]["nodes_all"]
    # a single grid runs as replicas
    c2 = bench.workload("c2", 1, world)
    assert c2["nodes_all"] == world * c2["nodes"]


def test_profiled_traffic_follows_the_source_digest(bench, tmp_path, monkeypatch):
    w = dict(bench.workload("f3_3d"))
    got = bench.profiled_traffic(w)
    if got is not None:  # the committed summary matches the current sources
        text = open(os.path.join(ROOT, "profiles", "step3d_march_kernel_chm_256_fp32.md")).read()
        assert f"dram_bytes_per_launch: {int(got)}" in text
    # a summary whose digest differs from the sources gives no traffic
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_8_fp32.md").write_text("source_sha256: 00ff\ndram_bytes_per_launch: 123\n")
    digest = bench.source_digest(w["src"])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda files: digest)
    assert bench.profiled_traffic(dict(kernel="k", nx=8, storage="fp32", src=w["src"])) is None
    (prof / "k_8_fp32.md").write_text(f"source_sha256: {digest}\ndram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic(dict(kernel="k", nx=8, storage="fp32", src=w["src"])) == 123.0
