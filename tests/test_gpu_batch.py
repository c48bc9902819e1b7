"""Batched stepping: 256 independent media of log-uniform sizes 64..512, 2000 steps, one launch per step over
a flattened warp table, captured in a CUDA graph.  Each member must equal, bit for bit, the same member
stepped alone (which the other parity tests tie to the oracle), and sampled members must match the oracle."""
import numpy as np
import pytest

from gpu_helpers import oracle_run, rel
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


def _solvers(probs, stream):
    out = []
    for p in probs:
        s = lbem.Solver(p.shape, stream=stream)
        s.set_problem(p)
        out.append(s)
    return out


def _read(s, p):
    import torch

    E, B = s.fields()
    tr = s.traces(p.rec_site.size)
    torch.cuda.synchronize()
    return E.cpu().numpy(), B.cpu().numpy(), tr.cpu().numpy()


def test_batch_of_256_equals_members_stepped_alone(lbem):
    import torch

    probs = W.batch_2d(256, nsteps=2000)
    st = torch.cuda.Stream()
    batch_s = _solvers(probs, st.cuda_stream)
    b = lbem.lbem_batch_create([s.h for s in batch_s], st.cuda_stream)
    v = lbem.lbem_batch_autotune(b, 20)
    assert 0 <= v < lbem.lbem_batch_get_variant(b)[1]
    lbem.lbem_batch_step(b, 1500)
    lbem.lbem_batch_step(b, 500)  # a second call reuses nothing but the members' state
    for s, p in zip(batch_s, probs):
        assert lbem.lbem_time(s.h) == 2000
    got = [_read(s, p) for s, p in zip(batch_s, probs)]
    lbem.lbem_batch_destroy(b)
    for s in batch_s:
        s.close()
    for k, p in enumerate(probs):
        alone = lbem.Solver(p.shape, stream=st.cuda_stream)
        alone.set_problem(p)
        alone.step(2000)
        ref = _read(alone, p)
        alone.close()
        for a, r in zip(got[k], ref):
            np.testing.assert_array_equal(a, r, err_msg=f"member {k} ({p.shape}), variant {v}")


def test_batch_members_match_oracle(lbem):
    import torch

    sizes = sorted(W.batch_sizes(256))
    pick = sizes[:4] + [sizes[128]]
    probs = [W.heterogeneous_2d(N, seed=1000 + k, nsteps=2000, sigma=min(20.0, N / 8.0), nrec=8,
                                rec_radius=max(1, N // 4)) for k, N in enumerate(pick)]
    st = torch.cuda.Stream()
    ss = _solvers(probs, st.cuda_stream)
    b = lbem.lbem_batch_create([s.h for s in ss], st.cuda_stream)
    lbem.lbem_batch_step(b, 2000)
    for s, p in zip(ss, probs):
        E, B, tr = _read(s, p)
        oE, oB, otr, _, _ = oracle_run(p)
        assert rel(np.moveaxis(E, 0, -1), oE) < 1e-4
        assert rel(np.moveaxis(B, 0, -1), oB) < 1e-4
        assert rel(tr, otr) < 1e-4
    lbem.lbem_batch_destroy(b)
    for s in ss:
        s.close()


def test_batch_rejects_mismatched_members(lbem):
    import torch

    a = lbem.Solver((16, 16))
    c = lbem.Solver((16, 16, 16))
    with pytest.raises(lbem.LbemError):
        lbem.lbem_batch_create([a.h, c.h])
    with pytest.raises(lbem.LbemError):
        lbem.lbem_batch_create([a.h, a.h])
    d = lbem.Solver((20, 24))
    lbem.lbem_set_medium(a.h, torch.ones(256, device="cuda"))
    lbem.lbem_set_medium(d.h, torch.ones(480, device="cuda"))
    lbem.lbem_set_fields(a.h)
    lbem.lbem_set_fields(d.h)
    lbem.lbem_step(a.h, 1)
    b = lbem.lbem_batch_create([a.h, d.h])
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_batch_step(b, 1)
    assert e.value.status == 6  # members at different times
    lbem.lbem_batch_destroy(b)
    for s in (a, c, d):
        s.close()


def test_every_batch_variant_is_bitwise_identical(lbem):
    import torch

    sizes = [64, 70, 97, 130, 200, 257, 333, 512]
    probs = [W.heterogeneous_2d(N, seed=2000 + k, nsteps=120, sigma=min(20.0, N / 8.0), nrec=8,
                                rec_radius=max(1, N // 4)) for k, N in enumerate(sizes)]
    st = torch.cuda.Stream()
    ref = []
    for p in probs:
        s = lbem.Solver(p.shape, stream=st.cuda_stream)
        s.set_problem(p)
        s.step(120)
        ref.append(_read(s, p))
        s.close()
    ss = _solvers(probs, st.cuda_stream)
    b = lbem.lbem_batch_create([s.h for s in ss], st.cuda_stream)
    nv = lbem.lbem_batch_get_variant(b)[1]
    for v in range(nv):
        for s, p in zip(ss, probs):
            s.set_problem(p)
        lbem.lbem_batch_set_variant(b, v)
        lbem.lbem_batch_step(b, 120)
        for s, p, r in zip(ss, probs, ref):
            for a, q in zip(_read(s, p), r):
                np.testing.assert_array_equal(a, q, err_msg=f"variant {v}, {p.shape}")
    lbem.lbem_batch_destroy(b)
    for s in ss:
        s.close()


def test_two_step_batch_ragged_members_odd_steps(lbem):
    """The two-steps-per-launch batch kernels (every tile shape) on tiny and odd-width members (1x1, 3x5, widths
    not a multiple of 4, one tile wide, a width just past one tile), sources and receivers at the corners, odd
    step counts split over two calls (a single step first, then pairs): bit-identical to each member stepped
    alone, and no write outside a member's arrays."""
    import torch

    shapes = [(1, 1), (3, 5), (17, 45), (9, 130), (64, 64), (70, 97), (41, 129), (33, 257)]
    probs = []
    for k, shp in enumerate(shapes):
        eps, _ = W.random_medium(shp, 300 + k)
        p = W.Problem("rb", 2, shp, eps, None, 40)
        p.E0, p.B0 = W.random_fields(shp, 400 + k, 0.2)
        n = int(np.prod(shp))
        p.src_site = np.array([0, n - 1], np.int64)
        p.src_comp = np.array([2, 2], np.int32)
        p.src_amp = np.ones((2, 40))
        p.rec_site = np.array([0, n // 2, n - 1], np.int64)
        p.rec_comp = np.array([2, 3, 4], np.int32)
        probs.append(p)
    st = torch.cuda.Stream()
    ref = []
    for p in probs:
        s = lbem.Solver(p.shape, stream=st.cuda_stream)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, 1, -1)
        s.step(37)
        ref.append(_read(s, p))
        s.close()
    ss = _solvers(probs, st.cuda_stream)
    b = lbem.lbem_batch_create([s.h for s in ss], st.cuda_stream)
    nv = lbem.lbem_batch_get_variant(b)[1]
    for v in range(9, nv):  # the two-step tile shapes (variants 9 ..)
        for s, p in zip(ss, probs):
            s.set_problem(p)
        lbem.lbem_batch_set_variant(b, v)
        lbem.lbem_batch_step(b, 13)
        lbem.lbem_batch_step(b, 24)
        for s, p, r in zip(ss, probs, ref):
            assert lbem.lbem_time(s.h) == 37
            lbem.lbem_check_guards(s.h)
            for a, q in zip(_read(s, p), r):
                np.testing.assert_array_equal(a, q, err_msg=f"variant {v}, {p.shape}")
    lbem.lbem_batch_destroy(b)
    for s in ss:
        s.close()
