"""The allocation-free reduction entry point against lbpf_diagnostics.

lbpf_field_sums_noalloc serves callers that cannot allocate device memory
where they need the conservation sums (allocator callbacks, hosts whose arena
owns the whole GPU, real-time loops).  This test gives it device copies of a
simulation's fields and checks its three FP64 sums against the handle's own
diagnostics, on two calls in a row with different data.  It lives in a file of
its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-9  # both sides sum the same per-node FP64 values in a different order


def _sums(L, torch, fields, fp64):
    dt = torch.float64 if fp64 else torch.float32
    dev = {k: torch.from_numpy(np.ascontiguousarray(fields[k])).to("cuda", dt)
           for k in ("phi", "phi_prev", "U", "rho")}
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.lbpf_field_sums_noalloc(dev["phi"].data_ptr(), dev["phi_prev"].data_ptr(),
                                   dev["U"].data_ptr(), dev["rho"].data_ptr(),
                                   fields["phi"].size, 1 if fp64 else 0, out.data_ptr(), stream)
    assert rc == L.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("fp64", [1, 0])
def test_noalloc_sums_match_diagnostics_twice(fp64):
    import torch
    assert torch.cuda.is_available()
    import paper_2206_02145_gb300 as L
    sim = L.Sim(stream=L.current_stream(), nx=200, ny=150, flow=1, fold=5, eps_aniso=0.03)
    sim.init_seed(80.0, 75.0, 0.0, 12.0, 0.4, 0.01, 11)
    for call in range(2):  # two calls in a row, on different states
        sim.step(150 + 100 * call)
        f = sim.fields(("phi", "U", "rho", "phi_prev"), fp64=True)
        d = sim.diagnostics()
        got = _sums(L, torch, f, fp64)
        want = np.array([d["solute_total"], d["mass_total"], d["solid_volume"]])
        tol = REL if fp64 else 1e-6  # FP32 inputs round each field value once
        assert np.all(np.abs(got - want) <= tol * np.abs(want)), (call, got, want)
    sim.close()


def test_noalloc_rejects_bad_arguments():
    import torch
    import paper_2206_02145_gb300 as L
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    big = L.NOALLOC_MAX_NODES + 1
    assert L.lbpf_field_sums_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), None, big, 1,
                                     out.data_ptr(), None) == L.EINVAL
    assert L.lbpf_field_sums_noalloc(None, x.data_ptr(), x.data_ptr(), None, 4, 1,
                                     out.data_ptr(), None) == L.EINVAL
