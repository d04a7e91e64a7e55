"""CPU checks of the C ABI boundary: the library builds, loads, exports every
symbol include/lbpf.h declares, and rejects invalid parameters before it
touches the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    import paper_2206_02145_gb300 as L
    assert os.path.samefile(L.LIB_PATH, path)
    return L


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbpf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbpf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbpf_create", "lbpf_init_seed", "lbpf_step", "lbpf_read_fields",
                     "lbpf_diagnostics"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert set(lib.EXPORTED) <= set(declared_functions())


def test_struct_layouts_match_header(lib, tmp_path):
    # the C compiler's sizeof/offsetof of the header structs against ctypes
    prog = tmp_path / "layout.c"
    fields = {"lbpf_params": [f for f, _ in lib.lbpf_params._fields_],
              "lbpf_seed": [f for f, _ in lib.lbpf_seed._fields_],
              "lbpf_diag": [f for f, _ in lib.lbpf_diag._fields_],
              "lbpf_unet_cfg": [f for f, _ in lib.lbpf_unet_cfg._fields_],
              "lbpf_surrogate_cfg": [f for f, _ in lib.lbpf_surrogate_cfg._fields_],
              "lbpf_surrogate_report": [f for f, _ in lib.lbpf_surrogate_report._fields_],
              "lbpf_polygon_seed": [f for f, _ in lib.lbpf_polygon_seed._fields_],
              "lbpf_facets": [f for f, _ in lib.lbpf_facets._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbpf.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {cf}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, fs in fields.items():
        cls = getattr(lib, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


@pytest.mark.parametrize("bad", [
    dict(tau_phi0=0.5), dict(tau_u_liquid=0.4), dict(flow=1, tau_f=0.5), dict(w0=0.0),
    dict(eps_aniso=1.0), dict(eps_aniso=-0.1), dict(fold=13), dict(dim=3, nz=8, fold=4),
    dict(nx=3), dict(dim=4), dict(bc=(0, 1, 0)), dict(u_inlet=0.2), dict(storage=7),
    dict(lambda_=float("nan")),
    # the central Hermite MRT: with flow, rates in (0, 2) or 0 for the default
    dict(collision=1), dict(collision=1, flow=0, dim=3, nz=8, fold=0), dict(collision=2, flow=1),
    dict(collision=1, flow=1, chm_omega_bulk=2.0), dict(collision=1, flow=1, chm_omega_high=-1.0),
])
def test_invalid_parameters_are_rejected_without_a_gpu(lib, bad):
    p = lib.lbpf_params_default(**bad)
    with pytest.raises(lib.LbpfError) as e:
        lib.lbpf_create(p)
    assert e.value.code == lib.EINVAL


def test_null_handle_calls_return_einval(lib):
    so = lib._lib
    assert so.lbpf_step(None, 1) == lib.EINVAL
    assert so.lbpf_diagnostics(None, None) == lib.EINVAL
    assert so.lbpf_state_bytes(None) == 0
    assert so.lbpf_surrogate_train(None, None, None, 1, 1, None, None, None, 1, None) == lib.EINVAL
    so.lbpf_destroy(None)


def test_batch_validation_before_any_gpu_work(lib):
    # a 3D instance and mixed storages are rejected before anything is allocated
    p3 = [lib.lbpf_params_default(dim=3, nz=8, fold=0), lib.lbpf_params_default()]
    with pytest.raises(lib.LbpfError) as e:
        lib.lbpf_batch_create(p3, [(4, 4, 4, 2, 0.3, 0, 1)] * 2)
    assert e.value.code == lib.EINVAL
    pm = [lib.lbpf_params_default(), lib.lbpf_params_default(storage=lib.FP16_SHIFTED)]
    with pytest.raises(lib.LbpfError) as e:
        lib.lbpf_batch_create(pm, [(4, 4, 0, 2, 0.3, 0, 1)] * 2)
    assert e.value.code == lib.EINVAL
    # one flow collision per batch
    pc = [lib.lbpf_params_default(flow=1),
          lib.lbpf_params_default(flow=1, collision=lib.COLL_CHM)]
    with pytest.raises(lib.LbpfError) as e:
        lib.lbpf_batch_create(pc, [(4, 4, 0, 2, 0.3, 0, 1)] * 2)
    assert e.value.code == lib.EINVAL
    assert lib._lib.lbpf_batch_step(None, 1) == lib.EINVAL
    assert lib._lib.lbpf_batch_count(None) == 0


def test_growth_fit_host_logic_matches_the_oracle(lib):
    # lbpf_growth_fit is host code: checked here without a GPU
    from oracle import facets as F
    import numpy as np
    rng = np.random.default_rng(11)
    for n in (2, 5, 40):
        t = np.sort(rng.uniform(0, 20, n)) + np.arange(n)
        L = 3.0 + 0.06 * t + rng.normal(0, 0.1, n)
        got = lib.lbpf_growth_fit(t, L)
        want = F.growth_fit(t, L)
        assert np.allclose(got[:2], want[:2], rtol=0, atol=1e-12)
        if n > 2:
            assert abs(got[2] - want[2]) < 1e-12
    assert np.isnan(lib.lbpf_growth_fit([0.0, 1.0, 2.0], [1.0, 1.0, 1.0])[2])
    for t, L in (([1.0], [2.0]), ([1.0, 1.0], [2.0, 3.0]), ([0.0, np.nan], [1.0, 2.0])):
        with pytest.raises(lib.LbpfError):
            lib.lbpf_growth_fit(t, L)
