"""lbem_diagnostics_static, the entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc once they are running: a program that
hands all device memory to its own pool at start-up, or a loop whose memory
budget is fixed after initialisation.  For them the library offers the FP64
diagnostics of lbem_diagnostics from a state and medium the caller holds, with
its only scratch in a static device array of the library.

These tests check that it gives the same diagnostics as lbem_diagnostics
(within the 1e-5 relative tolerance of the other diagnostics tests), with and
without a permeability array, on back-to-back calls (the static array is
reused), that free device memory does not change across calls, and that bad
sizes are rejected on the host before anything is launched.  This file is
collected last, so a failure here does not hide any other test.
"""
import numpy as np
import pytest

from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,shape,with_mu", [(2, (61, 90), False), (2, (61, 90), True), (3, (9, 10, 13), False),
                                             (3, (9, 10, 13), True)])
def test_static_scratch_diagnostics_match_handle_diagnostics(lbem, D, shape, with_mu):
    import torch

    eps_r, mu_r = W.random_medium(shape, 5, mu=with_mu)
    p = W.Problem("static", D, shape, eps_r, mu_r, 40)
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
    mu = torch.as_tensor(np.ascontiguousarray(mu_r, np.float32).ravel(), device="cuda") if with_mu else None
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    nz, ny, nx = (1,) + shape if D == 2 else shape
    free = []
    for call in range(3):
        s.step(20)
        ref = s.diagnostics()
        lbem.lbem_save_state(s.h, state)
        torch.cuda.synchronize()
        if call:
            free.append(torch.cuda.mem_get_info()[0])
        lbem.lbem_diagnostics_static(D, nx, ny, nz, state, eps, mu, 0.0, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for a, b in zip(got, ref):
            assert abs(a - b) <= 1e-5 * abs(b) + 1e-9, (call, got, ref)
    # the first call loads the library's module for this entry point; later calls allocate nothing
    lbem.lbem_diagnostics_static(D, nx, ny, nz, state, eps, mu, 0.0, out)
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
    assert len(set(free)) == 1, free
    s.close()


def test_static_scratch_rejects_bad_sizes_and_host_pointers(lbem):
    import torch

    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    eps = torch.ones(4, device="cuda")
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_diagnostics_static(2, 8192, 8192, 1, dummy, eps, None, 0.0, out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    # each dimension within int range, their product far beyond it: rejected, not wrapped
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_diagnostics_static(3, 1 << 21, 1 << 21, 1 << 21, dummy, eps, None, 0.0, out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_diagnostics_static(2, 2, 2, 1, np.zeros(64, np.uint8), eps, None, 0.0, out)
    assert e.value.status == 1


def _cudart():
    """The CUDA runtime of the toolkit, for exactly sized allocations (torch's caching allocator carves small
    tensors out of larger segments, so a short torch tensor does not end where its allocation ends)."""
    import ctypes
    import os

    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for name in (os.path.join(home, "lib64", "libcudart.so"), "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    else:
        pytest.skip("no libcudart.so for an exactly sized allocation")
    rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
    rt.cudaFree.argtypes = [ctypes.c_void_p]
    rt.cudaMemset.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t]
    return rt


def test_static_scratch_rejects_undersized_buffers(lbem):
    """Each caller buffer is checked against the end of the device allocation that holds it, before anything is
    launched: pointers placed so that the buffer ends exactly at the end of a 4 MiB allocation pass, and the same
    pointers moved closer to its end (a dense, unpadded state; a medium or output one element short) are refused
    with LBEM_ERR_ARG, so nothing is read out of bounds."""
    import ctypes

    import torch

    torch.cuda.synchronize()
    rt = _cudart()
    size = 4 << 20  # a multiple of the allocation granularity, so its reported extent is exactly this
    base = ctypes.c_void_p()
    assert rt.cudaMalloc(ctypes.byref(base), size) == 0
    lib = lbem.load()
    try:
        assert rt.cudaMemset(base, 0, size) == 0
        end = base.value + size
        nx, ny = 20, 16  # rows padded to 32 floats in the saved layout
        need = {"state": 4 * 5 * 32 * ny, "eps_r": 4 * nx * ny, "mu_r": 4 * nx * ny, "out": 24}
        dense = 4 * 5 * nx * ny
        ok = {"state": end - need["state"], "eps_r": end - need["eps_r"], "mu_r": end - need["mu_r"],
              "out": end - need["out"]}

        def call(ptrs):
            return lib.lbem_diagnostics_static(2, nx, ny, 1, ptrs["state"], ptrs["eps_r"], ptrs["mu_r"], 0.0,
                                               ptrs["out"], None)

        # each buffer alone at the very end of the allocation fits (the others point at its start)
        for k in need:
            ptrs = {j: base.value for j in need}
            ptrs[k] = ok[k]
            assert call(ptrs) == 0, (k, lbem.lbem_last_error())
        torch.cuda.synchronize()
        short = {"state": end - dense, "eps_r": end - need["eps_r"] + 4, "mu_r": end - need["mu_r"] + 4,
                 "out": end - 16}
        for k in need:
            ptrs = {j: base.value for j in need}
            ptrs[k] = short[k]
            assert call(ptrs) == 1, k
            assert k in lbem.lbem_last_error(), lbem.lbem_last_error()
    finally:
        torch.cuda.synchronize()
        rt.cudaFree(base)
