"""bpx_schedule_noalloc: the schedule for callers that cannot allocate.

Callers embedded in a runtime that owns the device memory pool, or on a
latency-critical path that cannot take the synchronisation of cudaMalloc /
cudaFree, cannot hand the library a workspace.  This entry point keeps its
scratch in a fixed array inside the library.  The test calls it through the
C ABI twice in a row -- with two different codes, so the second call starts
from the first call's leftovers -- and checks each result against the
workspace-based bpx_schedule, bit for bit (the schedule is integer work).
It also checks that a code too large for the fixed array is refused.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _noalloc(bpx, code, mask):
    S = code.num_sources
    order = torch.full((S, 3), 7, dtype=torch.int32, device="cuda")
    rec = torch.full((S,), 7, dtype=torch.uint8, device="cuda")
    info = torch.full((bpx.INFO_LEN,), 7, dtype=torch.int32, device="cuda")
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = bpx.lib().bpx_schedule_noalloc(code.handle, ct.c_void_p(mask.data_ptr()),
                                        ct.c_void_p(order.data_ptr()), ct.c_void_p(rec.data_ptr()),
                                        ct.c_void_p(info.data_ptr()), stream)
    assert rc == bpx.OK, bpx.lib().bpx_last_error()
    torch.cuda.synchronize()
    return order.cpu().numpy(), rec.cpu().numpy(), info.cpu().numpy()


def _with_workspace(bpx, code, mask):
    ws = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32)
    order, rec, info = bpx.schedule(code, mask, ws)
    torch.cuda.synchronize()
    return order.cpu().numpy(), rec.cpu().numpy(), info.cpu().numpy()


def test_noalloc_matches_workspace_schedule_twice(libbpx):
    bpx = libbpx
    calls = [
        (bpx.Code.mojette_a(11, 8, 12), W.erasure_mask(11, 3, 5)),
        (bpx.Code.table3(), W.mask_from_columns(5, [0, 4])),
    ]
    for code, m in calls:
        dm = torch.from_numpy(m).cuda()
        got = _noalloc(bpx, code, dm)
        exp = _with_workspace(bpx, code, dm)
        for g, e in zip(got, exp):
            assert np.array_equal(g, e)
        assert got[2][bpx.INFO_STATUS] == bpx.OK


def test_noalloc_rejects_codes_beyond_the_fixed_array(libbpx):
    bpx = libbpx
    big = bpx.Code.mojette_a(32, 24, 6000)   # ~30 MB of graph + plan
    m = torch.zeros(32, dtype=torch.uint8, device="cuda")
    S = big.num_sources
    out = torch.empty((S, 3), dtype=torch.int32, device="cuda")
    rc = bpx.lib().bpx_schedule_noalloc(big.handle, ct.c_void_p(m.data_ptr()),
                                        ct.c_void_p(out.data_ptr()), None, None,
                                        ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bpx.ERR_INVAL
    assert b"fixed" in bpx.lib().bpx_last_error()
