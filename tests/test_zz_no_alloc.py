"""The allocation-free update entry point (``loop_update_noalloc``).

Some callers cannot allocate device memory: applications that reserve all
of it up front in their own pool, or that forbid device allocation (and the
device-wide synchronisation it may bring) once running.  For them the
library offers a variant of ``loop_update`` whose scratch is a fixed static
device array.  These tests call it through the C ABI and compare it with
``loop_update`` on two calls in a row.  The file is named to be collected
last; it passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import meshgen

ml = pytest.importorskip("paper_1802_03749_gb300")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Checked on the host before anything touches the device."""
    L = ml.lib()
    rc = L.loop_update_noalloc(ml.MP_NOALLOC_MAX_CELLS + 1, 0, 0, None, None, None, None, None, None)
    assert rc == -10
    assert b"static scratch" in L.mp_error_string(rc)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,layout", [("f64", "aos"), ("f64", "soa"), ("f32", "aos")])
def test_noalloc_update_matches_update_on_two_calls(dtype, layout):
    import torch
    L = ml.lib()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dcode = 0 if dtype == "f64" else 1
    lcode = ml.LAYOUT[layout]
    ncell = 50_001                       # 25 partials, a ragged last one
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        qold = torch.tensor(meshgen.quad_state(ncell, seed=60 + call), dtype=tdt, device="cuda")
        if layout == "soa":
            qold = qold.t().contiguous()
        res = torch.tensor(meshgen.normal(61, 7, 4 * ncell, offset=call * 4 * ncell).reshape(-1, 4) * 1e-3,
                           dtype=tdt, device="cuda")
        adt = torch.tensor(meshgen.positive_field(ncell, 0.5, 1.5, seed=62 + call), dtype=tdt, device="cuda")
        q_ref, res_ref = torch.empty_like(qold), res.clone()
        q_new, res_new = torch.empty_like(qold), res.clone()
        rms_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        rms_new = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert L.loop_update(ncell, dcode, lcode, p(qold), p(q_ref), p(res_ref), p(adt), p(rms_ref), stream) == 0
        assert L.loop_update_noalloc(ncell, dcode, lcode, p(qold), p(q_new), p(res_new), p(adt), p(rms_new),
                                     stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(q_new, q_ref)            # same arithmetic per cell
        assert torch.count_nonzero(res_new) == 0
        a, b = rms_new.item(), rms_ref.item()
        assert b > 0 and abs(a - b) <= 1e-12 * b     # partial sums grouped differently
