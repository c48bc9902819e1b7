"""The bounded device-side wait gives up cleanly (failure detection without a GPU fault).

The multi-step kernels wait on an mbarrier for each tile's TMA window (the strip
kernel for each chunk of rows).  With the
wait limit set to 0 every such wait gives up at once on ordinary, in-bounds
loads: each CTA lets its copies in flight land (a separate bounded wait), flags
the failure and exits, and the next lbem_sync reports LBEM_ERR_TIMEOUT.  After
the limit is restored the same handle, reloaded from a snapshot, steps
correctly against the oracle and its guard bands are intact.
"""
import numpy as np
import pytest

from gpu_helpers import oracle_run, rel
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,spp,tile_shape", [("f32", 2, -1), ("f32", 3, -1), ("i16b", 2, -1), ("f32", 2, 9)])
def test_zero_wait_limit_reports_timeout_then_handle_recovers(lbem, storage, spp, tile_shape):
    import torch

    shape = (64, 512)  # wide enough for interior tiles, whose windows are TMA loads
    eps, _ = W.random_medium(shape, 11)
    p = W.Problem("wait", 2, shape, eps, None, 10)
    p.E0, p.B0 = W.random_fields(shape, 12, 0.5)
    n = int(np.prod(shape))
    p.src_site = np.array([n // 3], np.int64)
    p.src_comp = np.array([2], np.int32)
    p.src_amp = W.ricker(10, 0.1)[None, :]
    p.rec_site = np.array([n // 2, n - 7], np.int64)
    p.rec_comp = np.array([2, 3], np.int32)
    s = lbem.Solver(shape, storage=storage)
    try:
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, spp, tile_shape)
        assert lbem.lbem_get_temporal_blocking(s.h)[0] == spp
        snap = torch.empty(lbem.lbem_info(s.h)[1], dtype=torch.uint8, device="cuda")
        lbem.lbem_save_state(s.h, snap)
        lbem.lbem_sync(s.h)
        try:
            lbem.lbem_set_wait_limit(0.0)
            s.step(spp)  # one launch
            with pytest.raises(lbem.LbemError) as e:
                lbem.lbem_sync(s.h)
            assert e.value.status == 5, str(e.value)  # LBEM_ERR_TIMEOUT
        finally:
            lbem.lbem_set_wait_limit(2.0)
        lbem.lbem_sync(s.h)  # the flag was read and cleared; the context is healthy
        lbem.lbem_load_state(s.h, snap, 0)
        s.step(p.nsteps)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_sync(s.h)
        lbem.lbem_check_guards(s.h)
        oE, oB, otr, _, _ = oracle_run(p)
        E = np.moveaxis(E.cpu().double().numpy(), 0, -1)
        B = np.moveaxis(B.cpu().double().numpy(), 0, -1)
        tol = 1e-5 if storage == "f32" else 1e-3
        assert rel(E[..., 2], oE[..., 2]) < tol and rel(B[..., :2], oB[..., :2]) < tol
        assert rel(tr.cpu().double().numpy(), otr) < tol
    finally:
        s.close()

