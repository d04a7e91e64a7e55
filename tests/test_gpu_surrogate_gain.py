"""What the trained network gains over the method without it.

A three-level U-Net is trained on the GPU (the library's forward, backward
and Adam kernels) on LB trajectories of the seeded channel problems, then
used as the block propagator on a held-out problem, with the LB as judge and
fallback.  Checked: its held-out prediction error against predicting no
change; that the network advances most blocks under the checks; that the
solute invariant is kept; and the growth of the crystal against the plain LB
run from the same start.  The wall-time comparison is printed (the timed
speed-up at full size is the bench's surrogate workload)."""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NX = NY = 256
NB = 100  # LB steps per block


@pytest.fixture(scope="module")
def trained():
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import paper_2206_02145_gb300 as L
    from paper_2206_02145_gb300 import surrogate as S
    cfg = S.default_cfg(NB)
    X, T = S.generate_pairs(12, 4000, 200, NX, NY, cfg, seed=100, crop=128)
    Xv, Tv = S.generate_pairs(2, 4000, 400, NX, NY, cfg, seed=999, crop=128)
    net = L.UNet(in_ch=4, out_ch=4, levels=3, batch=8, height=128, width=NX, seed=1,
                 stream=L.current_stream())
    # measured across seeds: 2000 Adam steps at 3e-4 with mirror augmentation
    # learn reliably (shorter schedules at 1e-3 did not for some seeds)
    hist = S.train(net, X, T, 2000, lr=3e-4, log_every=500, augment=True)
    net.status()
    return L, S, cfg, net, (Xv, Tv), hist


def test_trained_network_beats_no_network(trained):
    L, S, cfg, net, (Xv, Tv), hist = trained
    ev = S.inference_net(net, NX, 128)
    err, base = S.prediction_error(ev, Xv, Tv)
    print("loss history", hist, "held-out mse", err, "no network", base)
    assert np.isfinite(err) and err < 0.5 * base
    ev.close()


def test_propagator_gains_at_the_stated_error(trained):
    L, S, cfg, net, _, _ = trained
    inf = S.inference_net(net, NX, NY)
    rng = np.random.default_rng(4242)
    params, fields, _ = S.channel_problem(rng, NX, NY)
    a = S.make_sim(params, fields)
    b = S.make_sim(params, fields)
    a.step(400)
    b.step(400)
    d0 = b.diagnostics()
    K = 20
    pcfg = S.default_cfg(NB, judge_every=4, drift_tol=1e-3, iface_tol=1.0)
    L.lbpf_surrogate_advance(a, inf, pcfg, 1)  # capture the prediction graph
    b.step(NB)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = L.lbpf_surrogate_advance(a, inf, pcfg, K)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    t0 = time.perf_counter()
    b.step(K * NB)
    torch.cuda.synchronize()
    tl = time.perf_counter() - t0
    da, db = a.diagnostics(), b.diagnostics()
    grow_lb = db["iface_pos"][:4] - d0["iface_pos"][:4]
    grow_s = da["iface_pos"][:4] - d0["iface_pos"][:4]
    print("report", rep, f"time {ts * 1e3:.1f} ms vs LB {tl * 1e3:.1f} ms",
          "growth LB", grow_lb, "network", grow_s)
    assert da["step"] == db["step"]
    assert rep["blocks"] == K and rep["surrogate_blocks"] >= K // 2
    # the checks held for every block the network advanced (a prediction that
    # failed one went to the LB instead and counts as a fallback)
    assert rep["max_drift_committed"] <= 1e-3 and rep["max_iface_est"] <= 1.0
    # committed states keep the solute invariant as the LB does
    assert abs(da["solute_drift_rel"]) < 1e-6
    # interface positions within 1 lattice unit, growth within 25 %
    assert np.all(np.abs(da["iface_pos"][:4] - db["iface_pos"][:4]) <= 1.0)
    assert np.all(np.abs(grow_s - grow_lb) <= 0.25 * np.abs(grow_lb) + 0.1)
    for x in (a, b, inf):
        x.close()
