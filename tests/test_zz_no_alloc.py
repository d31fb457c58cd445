"""tomo_oc_step_noalloc: the allocation-free OC update agrees with tomo_oc_step.

Collected last on purpose (file name), so that a run stopping at the first failure has
already run every other test.  It must pass alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_12282_gb300 import problems as P  # noqa: E402
from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _inputs(d, seed):
    z = torch.tensor(P.random_field(d, seed, 0.0, 1.0), dtype=torch.float32, device=DEV)
    dc = torch.tensor(P.random_sensitivity(d, seed + 1), dtype=torch.float32, device=DEV)
    dv = torch.tensor(np.random.default_rng(seed + 2).uniform(0.5, 1.5, d.n_el),
                      dtype=torch.float32, device=DEV)
    return z, dc, dv


@pytest.mark.parametrize("dims,volfrac,move", [((33, 17, 9), 0.3, 0.2), ((40, 20, 20), 0.12, 0.2)])
def test_noalloc_matches_handle_entry_point_twice(dims, volfrac, move):
    p = P.cantilever(*dims, volfrac=volfrac)
    d = p.dims
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        for call in range(2):  # two calls in a row: the shared scratch is reused
            z, dc, dv = _inputs(d, 100 + 10 * call)
            ref = torch.empty_like(z)
            ch_ref = g.oc_step(z, dc, dv, volfrac, move, ref)
            out = torch.full_like(z, -1.0)
            ch = torch.full((1,), -1.0, dtype=torch.float64, device=DEV)
            tomo.oc_step_noalloc(d.n_el, p.h, z, dc, dv, volfrac, move, out, ch)
            torch.cuda.synchronize()
            assert torch.max(torch.abs(out - ref)).item() <= 1e-6
            assert abs(ch.item() - ch_ref) <= 1e-6


def test_noalloc_rejects_oversize_and_host_arrays():
    z = torch.zeros(8, device=DEV)
    with pytest.raises(tomo.TomoError) as e:
        tomo.oc_step_noalloc((1 << 22) + 1, 1.0, torch.zeros((1 << 22) + 1, device=DEV),
                             torch.zeros((1 << 22) + 1, device=DEV),
                             torch.zeros((1 << 22) + 1, device=DEV), 0.3, 0.2,
                             torch.zeros((1 << 22) + 1, device=DEV))
    assert e.value.status == 1 and "4194304" in str(e.value)
    with pytest.raises(tomo.TomoError) as e:
        tomo.oc_step_noalloc(8, 1.0, z.cpu(), z, z.clone(), 0.3, 0.2, torch.zeros(8, device=DEV))
    assert e.value.status == 1 and "device" in str(e.value)


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs two visible devices")
def test_noalloc_rejects_memory_of_another_device():
    import ctypes
    a1 = torch.zeros(8, device="cuda:1")
    a0 = torch.zeros(8, device="cuda:0")
    ch = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    lib = tomo.lib()
    with torch.cuda.device(0):  # current device 0, z on device 1: rejected before any launch
        st = lib.tomo_oc_step_noalloc(ctypes.c_int64(8), ctypes.c_double(1.0),
                                      ctypes.c_void_p(a1.data_ptr()),
                                      ctypes.c_void_p(a0.data_ptr()),
                                      ctypes.c_void_p(a0.data_ptr()), ctypes.c_double(0.3),
                                      ctypes.c_double(0.2), ctypes.c_void_p(a0.data_ptr()),
                                      ctypes.c_void_p(ch.data_ptr()), ctypes.c_void_p(0))
    assert st == 1 and "current device" in lib.tomo_last_error(None).decode()
