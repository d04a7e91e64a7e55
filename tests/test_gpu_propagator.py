"""The learned block propagator's controller: read-out, targets, and the
checks that decide between the network and the LB step.  The network here is
untrained or has hand-set weights, so that each path is forced; the trained
network is covered by test_gpu_surrogate_gain.py."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

NX = NY = 256


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import paper_2206_02145_gb300
    return paper_2206_02145_gb300


@pytest.fixture(scope="module")
def S(L):
    from paper_2206_02145_gb300 import surrogate
    return surrogate


def _problem(S, seed):
    return S.channel_problem(np.random.default_rng(seed), NX, NY)


def _net(L, seed=5):
    return L.UNet(in_ch=4, out_ch=4, levels=3, batch=1, height=NY, width=NX, seed=seed,
                  stream=L.current_stream())


def test_sample_is_the_normalised_fields(L, S):
    params, fields, _ = _problem(S, 1)
    sim = S.make_sim(params, fields)
    sim.step(30)
    cfg = L.surrogate_cfg()
    x = torch.empty(NY, NX, 4, device="cuda")
    L.lbpf_surrogate_sample(sim, cfg, x)
    f = sim.fields(("phi", "U", "ux", "uy"), fp64=False)
    xs = x.cpu().numpy()
    for c, name in enumerate(("phi", "U", "ux", "uy")):
        want = (f[name] - np.float32(cfg.shift[c])) / np.float32(cfg.scale[c])
        np.testing.assert_allclose(xs[..., c], want, rtol=1e-6, atol=1e-6)
    sim.close()


def test_target_is_the_scaled_change(L):
    cfg = L.surrogate_cfg()
    g = torch.Generator(device="cpu").manual_seed(2)
    x0 = torch.randn(1000, 4, generator=g).cuda()
    x1 = torch.randn(1000, 4, generator=g).cuda()
    t = torch.empty_like(x0)
    L.lbpf_surrogate_target(cfg, x0, x1, 1000, t, L.current_stream())
    gain = torch.tensor([cfg.scale[c] / cfg.res_scale[c] for c in range(4)], device="cuda")
    torch.testing.assert_close(t, (x1 - x0) * gain, rtol=1e-6, atol=0)


def test_judging_every_block_is_the_plain_lb(L, S):
    params, fields, _ = _problem(S, 3)
    a = S.make_sim(params, fields)
    b = S.make_sim(params, fields)
    net = _net(L)
    rep = L.lbpf_surrogate_advance(a, net, L.surrogate_cfg(judge_every=1), 6)
    b.step(300)
    assert rep["blocks"] == rep["judged_blocks"] == 6 and rep["surrogate_blocks"] == 0
    assert a.diagnostics()["step"] == 300
    np.testing.assert_array_equal(a.state(), b.state())
    for s in (a, b, net):
        s.close()


def test_biased_network_fails_the_drift_check(L, S):
    # zero weights and a bias on the U output: a uniform gain of solute
    params, fields, _ = _problem(S, 4)
    a = S.make_sim(params, fields)
    b = S.make_sim(params, fields)
    net = _net(L)
    w = np.zeros(net.param_count, np.float32)
    w[-3] = 10.0  # head bias of output channel 1 (U)
    net.set_weights(w)
    rep = L.lbpf_surrogate_advance(a, net, L.surrogate_cfg(judge_every=0), 5)
    b.step(250)
    assert rep["surrogate_blocks"] == 0, rep
    assert rep["max_drift"] > 1e-3
    np.testing.assert_array_equal(a.state(), b.state())
    for s in (a, b, net):
        s.close()


def test_frozen_network_is_caught_by_the_interface_estimate(L, S):
    # all-zero network: predicts no change.  Its per-block interface error is
    # the LB displacement, below a 1-lattice-unit bound; the accumulated
    # estimate must stay within its budget and send blocks back to the LB.
    rng = np.random.default_rng(6)
    params, fields, _ = S.channel_problem(rng, NX, NY)
    fields["U"][:] = 0.45
    a = S.make_sim(params, fields)
    a.step(200)
    net = _net(L)
    net.set_weights(np.zeros(net.param_count, np.float32))
    tol = 0.5
    cfg = L.surrogate_cfg(judge_every=0, iface_tol=1.0, iface_budget=tol)
    rep = L.lbpf_surrogate_advance(a, net, cfg, 16)
    assert rep["blocks"] == 16
    assert rep["judged_blocks"] + rep["fallback_blocks"] >= 2, rep
    # once trusted after a judged block, the frozen network is accepted until
    # its accumulated estimate passes the budget: that block falls back
    assert rep["fallback_blocks"] >= 1, rep
    assert rep["iface_acc"] <= tol
    assert a.diagnostics()["step"] == 200 + 16 * 50
    for s in (a, net):
        s.close()


def test_frozen_network_fails_the_relative_interface_check(L, S):
    # the same frozen network: its estimate equals the LB's displacement, so a
    # bound relative to that displacement rejects every prediction and the
    # LB advances every block (judged or fallback), the result the plain LB's
    rng = np.random.default_rng(6)
    params, fields, _ = S.channel_problem(rng, NX, NY)
    fields["U"][:] = 0.45
    a = S.make_sim(params, fields)
    b = S.make_sim(params, fields)
    a.step(200)
    b.step(200)
    net = _net(L)
    net.set_weights(np.zeros(net.param_count, np.float32))
    cfg = L.surrogate_cfg(judge_every=0, iface_tol=1.0, iface_rel_tol=0.75)
    rep = L.lbpf_surrogate_advance(a, net, cfg, 12)
    assert rep["blocks"] == 12 and rep["surrogate_blocks"] == 0, rep
    assert rep["judged_blocks"] + rep["fallback_blocks"] == 12, rep
    b.step(12 * 50)
    np.testing.assert_array_equal(a.state(), b.state())
    # without the relative bound the same network is committed (absolute bound 1 lu)
    rep0 = L.lbpf_surrogate_advance(b, net, L.surrogate_cfg(judge_every=0, iface_tol=1.0), 12)
    assert rep0["surrogate_blocks"] > 0, rep0
    for s_ in (a, b, net):
        s_.close()


def test_rejects_mismatched_network(L, S):
    params, fields, _ = _problem(S, 7)
    a = S.make_sim(params, fields)
    net = L.UNet(in_ch=4, out_ch=4, levels=3, batch=1, height=NY, width=2 * NX, seed=1,
                 stream=L.current_stream())
    with pytest.raises(L.LbpfError):
        L.lbpf_surrogate_advance(a, net, L.surrogate_cfg(), 1)
    with pytest.raises(L.LbpfError):
        L.lbpf_surrogate_advance(a, _net(L), L.surrogate_cfg(steps_per_block=0), 1)
    with pytest.raises(L.LbpfError):
        L.lbpf_surrogate_advance(a, _net(L), L.surrogate_cfg(iface_rel_tol=-1.0), 1)
    a.close()
    net.close()


def test_two_propagators_on_unordered_streams(L, S):
    # each network holds its own propagator scratch (the FP64 reduction of the
    # prediction included): two propagators advanced at the same time from two
    # host threads on two unordered streams give what each gives alone
    import threading
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    probs = [_problem(S, 11), _problem(S, 12)]

    def run(i, stream, out):
        params, fields, _ = probs[i]
        sim = S.make_sim(params, fields, stream.cuda_stream)
        sim.step(100)
        net = L.UNet(in_ch=4, out_ch=4, levels=3, batch=1, height=NY, width=NX, seed=5,
                     stream=stream.cuda_stream)
        net.set_weights(np.zeros(net.param_count, np.float32))  # predicts no change
        cfg = L.surrogate_cfg(judge_every=3, iface_tol=1.0)
        out[i] = (L.lbpf_surrogate_advance(sim, net, cfg, 9), sim.state())
        sim.close()
        net.close()

    alone = [None, None]
    for i in range(2):
        run(i, streams[i], alone)
    both = [None, None]
    threads = [threading.Thread(target=run, args=(i, streams[i], both)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i in range(2):
        assert both[i][0] == alone[i][0], (both[i][0], alone[i][0])
        assert alone[i][0]["surrogate_blocks"] > 0, alone[i][0]
        np.testing.assert_array_equal(both[i][1], alone[i][1])
