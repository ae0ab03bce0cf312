"""Failure detection on the GPU without a GPU fault: a bounded wait runs out
and the kernel reports BPX_ERR_TIMEOUT; the context stays usable.  Stragglers
beyond what the code tolerates are reported as BPX_ERR_UNDECODABLE (see
test_gpu_parity.test_undecodable_partial)."""
import ctypes as ct

import numpy as np
import pytest

from oracle import bpx_oracle as o
from paper_1904_11563_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_wait_timeout_reports_and_context_survives(libbpx):
    bpx = libbpx
    info = torch.zeros(16, dtype=torch.int32, device="cuda")
    budget = 2_000_000  # ~1 ms of SM clock
    rc = bpx.lib().bpx_selftest_wait_timeout(budget, ct.c_void_p(info.data_ptr()),
                                             ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bpx.OK
    torch.cuda.synchronize()
    inf = info.cpu().numpy()
    assert inf[bpx.INFO_STATUS] == bpx.ERR_TIMEOUT
    assert inf[bpx.INFO_DEVICE_ERR] == bpx.ERR_TIMEOUT
    assert inf[6] >= budget
    # the context is still usable: a normal coded multiplication is exact
    code = bpx.Code.table1()
    A = W.matrix((64, 32), "int", 1)
    B = W.matrix((32, 16), "int", 2)
    ws = bpx.Workspace(code, 64, 16, 32, 16, bpx.BF16X3)
    C, inf2 = bpx.coded_matmul(code, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 16, bpx.BF16X3,
                               torch.from_numpy(W.mask_from_columns(5, [0, 2])).cuda(), ws)
    torch.cuda.synchronize()
    assert inf2.cpu().numpy()[bpx.INFO_STATUS] == bpx.OK
    assert np.array_equal(C[:64].cpu().numpy(), o.reference_product(A, B))


def test_selftest_rejects_bad_budget(libbpx):
    bpx = libbpx
    info = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = bpx.lib().bpx_selftest_wait_timeout(0, ct.c_void_p(info.data_ptr()), None)
    assert rc == bpx.ERR_INVAL
