"""lbem_diagnostics_static, the entry point for callers that cannot allocate device memory.

It must give the same FP64 diagnostics as lbem_diagnostics (within the 1e-5
relative tolerance of the other diagnostics tests) from a state and medium the
caller holds, with its scratch in the library's static device array, and keep
doing so on back-to-back calls (the static array is reused).  This file is
collected last, so a failure here does not hide any other test.
"""
import numpy as np
import pytest

from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,shape", [(2, (61, 90)), (3, (9, 10, 13))])
def test_static_scratch_diagnostics_match_handle_diagnostics(lbem, D, shape):
    import torch

    p = W.Problem("static", D, shape, W.random_medium(shape, 5)[0], None, 40)
    p.E0, p.B0 = W.random_fields(shape, 6, 0.5)
    n = int(np.prod(shape))
    p.src_site = np.array([n // 2], np.int64)
    p.src_comp = np.array([2], np.int32)
    p.src_amp = W.ricker(40, 0.1)[None, :]
    s = lbem.Solver(shape)
    s.set_problem(p)
    nbytes = lbem.lbem_info(s.h)[1]
    state = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    eps = torch.as_tensor(np.ascontiguousarray(p.eps_r, np.float32).ravel(), device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    nz, ny, nx = (1,) + shape if D == 2 else shape
    for call in range(2):
        s.step(20)
        ref = s.diagnostics()
        lbem.lbem_save_state(s.h, state)
        torch.cuda.synchronize()
        lbem.lbem_diagnostics_static(D, nx, ny, nz, state, eps, None, 0.0, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for a, b in zip(got, ref):
            assert abs(a - b) <= 1e-5 * abs(b) + 1e-9, (call, got, ref)
    s.close()


def test_static_scratch_rejects_oversized_grids_and_host_pointers(lbem):
    import torch

    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    eps = torch.ones(4, device="cuda")
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_diagnostics_static(2, 8192, 8192, 1, dummy, eps, None, 0.0, out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_diagnostics_static(2, 2, 2, 1, np.zeros(64, np.uint8), eps, None, 0.0, out)
    assert e.value.status == 1
