"""Every kernel stays inside its arrays: after runs over ragged grids in every storage form, every launch
shape, 3D, fields, diagnostics, save/load, the adjoint and a batch, the guard bands the library keeps around
each handle-owned array are intact."""
import numpy as np
import pytest

from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 45), (9, 130), (33, 257)])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "i16b"])
def test_guards_intact_2d(lbem, shape, storage):
    import torch

    eps, mu = W.random_medium(shape, 3, mu=True)
    p = W.Problem("g", 2, shape, eps, mu, 12)
    p.E0, p.B0 = W.random_fields(shape, 4, 0.2)
    n = int(np.prod(shape))
    p.src_site = np.array([0, n - 1], np.int64)
    p.src_comp = np.array([2, 2], np.int32)
    p.src_amp = np.ones((2, 12))
    p.rec_site = np.array([0, n // 2, n - 1], np.int64)
    p.rec_comp = np.array([2, 3, 4], np.int32)
    s = lbem.Solver(shape, storage=storage)
    s.set_problem(p)
    lbem.lbem_set_temporal_blocking(s.h, 1, -1)
    for v in range(lbem.lbem_get_variant(s.h)[1]):
        lbem.lbem_set_variant(s.h, v)
        s.step(3)
    s.fields()
    s.diagnostics()
    nb = lbem.lbem_info(s.h)[1]
    snap = torch.empty(nb, dtype=torch.uint8, device="cuda")
    lbem.lbem_save_state(s.h, snap)
    lbem.lbem_load_state(s.h, snap, 3)
    torch.cuda.synchronize()
    lbem.lbem_check_guards(s.h)
    s.close()


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 45), (9, 130), (33, 257), (40, 300), (130, 644)])
def test_guards_intact_two_step(lbem, shape):
    """The two- and three-step kernels in every tile shape, on ragged grids, with sources and receivers at the
    corners."""
    import torch

    eps, _ = W.random_medium(shape, 6)
    p = W.Problem("g2", 2, shape, eps, None, 13)
    p.E0, p.B0 = W.random_fields(shape, 7, 0.2)
    n = int(np.prod(shape))
    p.src_site = np.array([0, n - 1], np.int64)
    p.src_comp = np.array([2, 2], np.int32)
    p.src_amp = np.ones((2, 13))
    p.rec_site = np.array([0, n // 2, n - 1], np.int64)
    p.rec_comp = np.array([2, 3, 4], np.int32)
    s = lbem.Solver(shape)
    s.set_problem(p)
    for spp in (2, 3):
        lbem.lbem_set_temporal_blocking(s.h, spp, 0)
        for k in range(lbem.lbem_get_temporal_blocking(s.h)[2]):
            lbem.lbem_set_temporal_blocking(s.h, spp, k)
            s.step(4)
    torch.cuda.synchronize()
    lbem.lbem_sync(s.h)
    lbem.lbem_check_guards(s.h)
    s.close()


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (5, 6, 130)])
def test_guards_intact_3d_and_adjoint(lbem, shape):
    import torch

    eps, _ = W.random_medium(shape, 5)
    p = W.Problem("g3", 3, shape, eps, None, 10)
    n = int(np.prod(shape))
    p.src_site = np.array([n // 2], np.int64)
    p.src_comp = np.array([1], np.int32)
    p.src_amp = np.ones((1, 10))
    p.rec_site = np.array([0, n - 1], np.int64)
    p.rec_comp = np.array([2, 5], np.int32)
    s = lbem.Solver(shape)
    s.set_problem(p)
    for v in range(lbem.lbem_get_variant(s.h)[1]):
        lbem.lbem_set_variant(s.h, v)
        s.step(2)
    s.fields()
    s.diagnostics()
    lbem.lbem_set_fields(s.h)
    lbem.lbem_forward_record(s.h, 10, 3)
    cot = torch.ones(2 * 10, device="cuda")
    g = torch.empty(n, device="cuda")
    lbem.lbem_adjoint(s.h, cot, g)
    torch.cuda.synchronize()
    lbem.lbem_check_guards(s.h)
    s.close()


def test_guards_intact_after_batch(lbem):
    import torch

    st = torch.cuda.Stream()
    probs = [W.heterogeneous_2d(N, seed=50 + N, nsteps=20, sigma=3.0, nrec=4, rec_radius=N // 4) for N in (64, 65, 99, 130)]
    ss = []
    for q in probs:
        s = lbem.Solver(q.shape, stream=st.cuda_stream)
        s.set_problem(q)
        ss.append(s)
    b = lbem.lbem_batch_create([s.h for s in ss], st.cuda_stream)
    for v in range(lbem.lbem_batch_get_variant(b)[1]):
        lbem.lbem_batch_set_variant(b, v)
        lbem.lbem_batch_step(b, 2)
    lbem.lbem_batch_destroy(b)
    torch.cuda.synchronize()
    for s in ss:
        lbem.lbem_check_guards(s.h)
        s.close()
