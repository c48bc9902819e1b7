"""Anisotropic media (a uniform in-plane permeability tensor, per-axis lattice weights) on the GPU.

Tolerance as for the periodic parity tests: relative L2 of E, B and receiver traces <= 1e-5 against the FP64
oracle.  Also: the per-axis dispersion of plane waves, the isotropic tensor against the plain scheme with a
uniform mu, combinations with walls, layers and a dispersive pole, two steps per launch against single steps
bit for bit, and the errors.
"""
import numpy as np
import pytest

from gpu_helpers import gpu_run, oracle_run, rel
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu

PEC, PMC = lbem.BC_PEC, lbem.BC_PMC


def _problem(shape, seed, nsteps, aniso, bc=(0, 0), layer=0, pole=False):
    eps, _ = W.random_medium(shape, seed, lo=1.2, hi=3.0)
    p = W.Problem("aniso", 2, shape, eps, None, nsteps)
    p.aniso = aniso
    p.E0, p.B0 = W.random_fields(shape, seed + 1, 0.3)
    p.E0[..., :2] = 0
    p.B0[..., 2] = 0
    rng = np.random.default_rng(seed + 2)
    n = int(np.prod(shape))
    ny, nx = shape
    p.src_site = np.unique(np.concatenate([[0, n - 1, nx - 1], rng.integers(0, n, 4)])).astype(np.int64)
    p.src_comp = np.full(p.src_site.size, 2, np.int32)
    p.src_amp = rng.standard_normal((p.src_site.size, nsteps))
    p.rec_site = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 9)])).astype(np.int64)
    p.rec_comp = np.array([2, 3, 4] * ((p.rec_site.size + 2) // 3), np.int32)[: p.rec_site.size]
    p.bc = tuple(bc) + (0,)
    p.layer = layer
    p.gamma_max = 0.3 if layer else 0.0
    if pole:
        r = np.sqrt(aniso[0] / aniso[1])
        cbar2 = 0.5 / (np.asarray(eps, np.float32).astype(np.float64) * np.sqrt(aniso[0] * aniso[1]))
        w0 = 1 - (r + 1 / r) * cbar2
        p.wp2 = 0.9 * 4 * w0 * rng.random(shape)
        p.gamma = 0.1 * rng.random(shape)
    return p


CASES = [((1, 1), (1.0, 2.0), (0, 0), 0, False), ((3, 5), (2.5, 1.2), (0, 0), 0, True),
         ((17, 45), (0.7, 1.6), (PEC, 0), 0, False), ((33, 257), (2.0, 1.0), (PMC, PEC), 6, True),
         ((130, 131), (1.3, 1.3), (0, 0), 0, False), ((64, 300), (3.0, 1.5), (PEC, PEC), 12, False)]


@pytest.mark.parametrize("shape,aniso,bc,layer,pole", CASES)
def test_anisotropic_media_match_oracle(lbem, shape, aniso, bc, layer, pole):
    p = _problem(shape, 800 + shape[1], 43, aniso, bc, layer, pole)
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    eE, eB, eT = rel(E, oE), rel(B, oB), rel(tr, otr)
    print(f"{shape} mu {aniso} bc {bc} layer {layer} pole {pole}: rel-L2 E {eE:.1e} B {eB:.1e} traces {eT:.1e}")
    assert eE < 1e-5 and eB < 1e-5 and eT < 1e-5


def test_isotropic_tensor_is_the_plain_scheme_with_uniform_mu(lbem):
    p = _problem((40, 70), 21, 30, (1.7, 1.7))
    q = _problem((40, 70), 21, 30, (1.7, 1.7))
    q.aniso = None
    q.mu_r = np.full(q.shape, 1.7)
    a, b = gpu_run(p), gpu_run(q)
    for x, y in zip(a, b):
        assert rel(x, y) < 1e-6


def test_plane_waves_on_gpu_follow_the_per_axis_dispersion(lbem):
    import torch

    N, w_eps, aniso, mode = 64, 1.6, (2.5, 1.2), (3, 5)
    p = W.Problem("plane", 2, (N, N), np.full((N, N), w_eps), None, 80)
    p.aniso = aniso
    y, x = np.mgrid[0:N, 0:N]
    kx, ky = 2 * np.pi * mode[0] / N, 2 * np.pi * mode[1] / N
    p.E0 = np.zeros((N, N, 3))
    p.E0[..., 2] = np.cos(kx * x + ky * y)
    p.B0 = np.zeros_like(p.E0)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    basis = np.exp(-1j * (kx * x + ky * y))
    amp = []
    for _ in range(80):
        E, _ = s.fields()
        torch.cuda.synchronize()
        amp.append(np.real((E[2].cpu().double().numpy() * basis).sum()) / (N * N / 2))
        s.step(1)
    s.close()
    amp = np.array(amp)
    e = np.float32(w_eps).astype(np.float64)
    cx2, cy2 = 0.5 / (e * aniso[1]), 0.5 / (e * aniso[0])
    om = 2 * np.arcsin(np.sqrt(cx2 * np.sin(kx / 2) ** 2 + cy2 * np.sin(ky / 2) ** 2))
    t = np.arange(80)
    b = (amp[1] - amp[0] * np.cos(om)) / np.sin(om)
    np.testing.assert_allclose(amp, amp[0] * np.cos(om * t) + b * np.sin(om * t), rtol=0, atol=2e-5)


@pytest.mark.parametrize("shape,aniso", [((3, 5), (2.5, 1.2)), ((37, 130), (0.7, 1.6)), ((130, 259), (1.7, 1.7))])
def test_two_step_launches_equal_single_steps_bit_for_bit(lbem, shape, aniso):
    """Without walls or a pole an anisotropic medium steps in pairs (the tile kernel, shape 0, or the strip
    kernel, shape 1, with per-axis weights): the same bits as one step per launch (the general kernel), with
    and without graph replay, odd step counts included."""
    import torch

    p = _problem(shape, 900 + shape[1], 37, aniso)
    ref = gpu_run(p, steps_per_pass=1)
    for tile_shape, graphs in ((0, False), (0, True), (1, False), (1, True)):
        stream = torch.cuda.Stream()  # graph capture needs a non-default stream
        s = lbem.Solver(p.shape, stream=stream.cuda_stream)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, 2, tile_shape)
        assert lbem.lbem_get_temporal_blocking(s.h)[:2] == (2, tile_shape)
        lbem.lbem_set_graphs(s.h, graphs)
        s.step(10)
        s.step(27)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_check_guards(s.h)
        s.close()
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
        np.testing.assert_array_equal(tr.cpu().double().numpy()[:, :37], ref[2])


@pytest.mark.parametrize("shape,aniso,bc,layer", [((17, 45), (0.7, 1.6), (PEC, 0), 0),
                                                ((40, 131), (2.0, 1.0), (PMC, PEC), 6),
                                                ((64, 300), (3.0, 1.5), (PEC, PEC), 12),
                                                ((9, 7), (1.3, 2.2), (PEC, PMC), 3)])
def test_walls_two_step_launches_equal_single_steps_bit_for_bit(lbem, shape, aniso, bc, layer):
    """With walls and absorbing layers an anisotropic medium also steps in pairs: the tile or the strip kernel
    (periodic), then the edge pass recomputing the two steps on the bands next to the walls with the per-axis
    collision. The same bits as single steps of the general kernel, which applies the walls and layers itself,
    with graphs and odd step counts; with a pole as well the medium steps singly."""
    import torch

    p = _problem(shape, 950 + shape[1], 37, aniso, bc, layer)
    ref = gpu_run(p, steps_per_pass=1)
    for tile_shape, graphs in ((0, False), (0, True), (1, False), (1, True)):
        stream = torch.cuda.Stream()
        s = lbem.Solver(p.shape, stream=stream.cuda_stream)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, 2, tile_shape)
        assert lbem.lbem_get_temporal_blocking(s.h)[:2] == (2, tile_shape)
        lbem.lbem_set_graphs(s.h, graphs)
        s.step(10)
        s.step(27)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_sync(s.h)
        lbem.lbem_check_guards(s.h)
        s.close()
        msg = f"tile shape {tile_shape}, graphs {graphs}"
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0], err_msg=msg)
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1], err_msg=msg)
        np.testing.assert_array_equal(tr.cpu().double().numpy()[:, :37], ref[2], err_msg=msg)
    q = _problem(shape, 950 + shape[1], 5, aniso, bc, layer, pole=True)
    s = lbem.Solver(q.shape)
    s.set_problem(q)
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 1
    s.close()


def test_anisotropic_full_size_matches_oracle(lbem):
    """4096^2 heterogeneous medium with mu = diag(2, 1) (the benchmark's anisotropic workload), 20 steps."""
    p = W.heterogeneous_2d_aniso(4096, seed=2, nsteps=20)
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    assert rel(E, oE) < 1e-5 and rel(B, oB) < 1e-5 and rel(tr, otr) < 1e-5


def test_anisotropy_errors_and_switching_back(lbem):
    import torch

    p = _problem((16, 20), 13, 5, (2.0, 1.0))
    s = lbem.Solver(p.shape)
    eps = np.ascontiguousarray(np.asarray(p.eps_r, np.float32).ravel())
    for mxx, myy in ((0.0, 1.0), (1.0, -2.0), (np.inf, 1.0)):
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_medium_aniso(s.h, eps, mxx, myy)
        assert e.value.status == 1
    with pytest.raises(lbem.LbemError) as e:  # c_x^2 + c_y^2 > 1 somewhere: rest weight < 0
        lbem.lbem_set_medium_aniso(s.h, eps, 0.3, 0.3)
    assert e.value.status == 3
    s.set_problem(p)
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 2  # no walls, no pole: two steps per launch
    assert lbem.lbem_get_temporal_blocking(s.h)[2] == 2  # the tile kernel and the strip kernel
    lbem.lbem_set_boundaries(s.h, (PEC, 0, 0), 0, 0.0)
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 2  # walls: still pairs, then the anisotropic edge pass
    lbem.lbem_set_boundaries(s.h, (0, 0, 0), 0, 0.0)
    with pytest.raises(lbem.LbemError):
        lbem.lbem_forward_record(s.h, 4, 2)
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_batch_create([s.h], torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 1
    lbem.lbem_set_medium(s.h, eps)  # isotropic again: the fast two-step kernel
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 2
    s.close()
    for shape, kw in (((8, 32), dict(storage="bf16")), ((4, 4, 8), {})):
        h = lbem.Solver(shape, **kw)
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_medium_aniso(h.h, np.full(int(np.prod(shape)), 2.0, np.float32), 2.0, 1.0)
        assert e.value.status == 1
        h.close()
