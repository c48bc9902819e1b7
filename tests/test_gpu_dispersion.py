"""Frequency-dispersive permittivity (one Drude-Lorentz pole per site) on the GPU, against the oracle.

Tolerance as for the periodic parity tests: relative L2 of E, B and receiver traces <= 1e-5 against the FP64
oracle (FP32 arithmetic).  Also: the lattice plasma dispersion of a Drude plane wave, graphs and split step counts
bit for bit, two steps per launch against single steps bit for bit, save / load of the pole's state, and the
argument, state and stability errors.
"""
import numpy as np
import pytest

from gpu_helpers import gpu_run, oracle_run, rel
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu

PEC, PMC = lbem.BC_PEC, lbem.BC_PMC


def _problem(shape, seed, nsteps, mu=False, bc=(0, 0), layer=0):
    eps, mu_r = W.random_medium(shape, seed, lo=1.2, hi=3.0, mu=mu)
    p = W.Problem("disp", 2, shape, eps, mu_r, nsteps)
    p.E0, p.B0 = W.random_fields(shape, seed + 1, 0.3)
    p.E0[..., :2] = 0
    p.B0[..., 2] = 0
    rng = np.random.default_rng(seed + 2)
    w0 = 1 - 1.0 / (np.asarray(eps, np.float32).astype(np.float64) * (1.0 if mu_r is None else mu_r))
    room = 4 * w0 * 0.95  # below the stability bound wp^2 + wr^2 <= 4 w0
    share = rng.random(shape)
    on = rng.random(shape) < 0.7
    p.wp2 = np.where(on, room * share * rng.random(shape), 0.0)
    p.wr2 = np.where(on, room * (1 - share) * rng.random(shape), 0.0)
    p.gamma = np.where(on, 0.2 * rng.random(shape), 0.0)
    n = int(np.prod(shape))
    ny, nx = shape
    p.src_site = np.unique(np.concatenate([[0, n - 1, nx - 1], rng.integers(0, n, 4)])).astype(np.int64)
    p.src_comp = np.full(p.src_site.size, 2, np.int32)
    p.src_amp = rng.standard_normal((p.src_site.size, nsteps))
    p.rec_site = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 8)])).astype(np.int64)
    p.rec_comp = np.array([2, 3, 4] * ((p.rec_site.size + 2) // 3), np.int32)[: p.rec_site.size]
    p.bc = tuple(bc) + (0,)
    p.layer = layer
    p.gamma_max = 0.3 if layer else 0.0
    return p


CASES = [((1, 1), False, (0, 0), 0), ((3, 5), True, (0, 0), 0), ((17, 45), False, (PEC, 0), 0),
         ((33, 257), True, (PMC, PEC), 6), ((130, 131), False, (0, 0), 0), ((64, 300), True, (PEC, PEC), 12)]


@pytest.mark.parametrize("shape,mu,bc,layer", CASES)
def test_dispersive_media_match_oracle(lbem, shape, mu, bc, layer):
    p = _problem(shape, 700 + shape[1], 47, mu, bc, layer)
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    eE, eB, eT = rel(E, oE), rel(B, oB), rel(tr, otr)
    print(f"{shape} mu {mu} bc {bc} layer {layer}: rel-L2 E {eE:.1e} B {eB:.1e} traces {eT:.1e}")
    assert eE < 1e-5 and eB < 1e-5 and eT < 1e-5


def test_drude_plane_wave_on_gpu_follows_the_lattice_plasma_dispersion(lbem):
    """E_z = cos(k.x) in a homogeneous lossless Drude medium: the GPU's E_z amplitude follows cos, sin of
    omega t with 4 sin^2(omega/2) = 4 c^2 (sin^2(kx/2) + sin^2(ky/2)) + wp^2 (to FP32 rounding)."""
    import torch

    N, w_eps, wp2, mode = 64, 1.6, 0.2, (3, 5)
    p = W.Problem("plasma", 2, (N, N), np.full((N, N), w_eps), None, 80)
    y, x = np.mgrid[0:N, 0:N]
    kx, ky = 2 * np.pi * mode[0] / N, 2 * np.pi * mode[1] / N
    p.E0 = np.zeros((N, N, 3))
    p.E0[..., 2] = np.cos(kx * x + ky * y)
    p.B0 = np.zeros_like(p.E0)
    p.wp2 = np.full((N, N), wp2)
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
    c2 = 0.5 / np.float32(w_eps).astype(np.float64)
    om = 2 * np.arcsin(np.sqrt(c2 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2) + np.float32(wp2) / 4))
    t = np.arange(80)
    b = (amp[1] - amp[0] * np.cos(om)) / np.sin(om)
    np.testing.assert_allclose(amp, amp[0] * np.cos(om * t) + b * np.sin(om * t), rtol=0, atol=2e-5)


def test_dispersive_graphs_splits_and_state_round_trip(lbem):
    import torch

    p = _problem((40, 130), 11, 31, True, (PEC, 0), 4)
    ref = gpu_run(p)
    stream = torch.cuda.Stream()
    s = lbem.Solver(p.shape, stream=stream.cuda_stream)
    s.set_problem(p)
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 1  # one step per launch with a pole
    lbem.lbem_set_graphs(s.h, True)
    s.step(10)
    nb = lbem.lbem_info(s.h)[1]
    assert nb == 5 * 40 * 160 * 4 + 2 * 40 * 160 * 4  # populations (pitch 160) + the pole's J and P planes
    saved = torch.empty(nb, dtype=torch.uint8, device="cuda")
    lbem.lbem_save_state(s.h, saved)
    s.step(11)
    lbem.lbem_load_state(s.h, saved, 10)  # back to t = 10, pole included
    s.step(11)
    s.step(10)
    E, B = s.fields()
    tr = s.traces(p.rec_site.size)
    torch.cuda.synchronize()
    lbem.lbem_check_guards(s.h)
    s.close()
    np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
    np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
    np.testing.assert_array_equal(tr.cpu().double().numpy()[:, :31], ref[2])


@pytest.mark.parametrize("shape,aniso", [((1, 1), None), ((3, 5), None), ((37, 130), None), ((130, 259), None),
                                         ((40, 70), (2.0, 1.3))])
def test_two_step_launches_equal_single_steps_bit_for_bit(lbem, shape, aniso):
    """Without walls or a heterogeneous mu a dispersive medium steps in pairs (the tile kernel carrying the pole's
    J and P; P alternates between two planes with the population buffers): the same bits as one step per launch,
    with and without graph replay, odd step counts, and a save / load across launches of both parities."""
    import torch

    p = _problem(shape, 600 + shape[1], 40)
    if aniso is not None:  # a uniform tensor with the pole: the pole's bound uses the per-axis rest weight
        p.aniso = aniso
        p.wp2 = p.wp2 * 0.5
        p.wr2 = p.wr2 * 0.5
    ref = gpu_run(p, steps_per_pass=1)
    for graphs in (False, True):
        stream = torch.cuda.Stream()  # graph capture needs a non-default stream
        s = lbem.Solver(p.shape, stream=stream.cuda_stream)
        s.set_problem(p)
        assert lbem.lbem_get_temporal_blocking(s.h)[0] == 2
        lbem.lbem_set_graphs(s.h, graphs)
        s.step(7)  # three pairs and a single step
        saved = torch.empty(lbem.lbem_info(s.h)[1], dtype=torch.uint8, device="cuda")
        lbem.lbem_save_state(s.h, saved)
        s.step(9)
        lbem.lbem_load_state(s.h, saved, 7)  # back to t = 7 with the buffers' parity flipped
        s.step(20)
        s.step(13)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_check_guards(s.h)
        s.close()
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
        np.testing.assert_array_equal(tr.cpu().double().numpy()[:, :40], ref[2])


def test_dispersion_full_size_matches_oracle(lbem):
    """4096^2 heterogeneous medium with a lossy Drude cylinder (the benchmark's dispersive workload), 20 steps."""
    p = W.heterogeneous_2d_drude(4096, seed=2, nsteps=20)
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    assert rel(E, oE) < 1e-5 and rel(B, oB) < 1e-5 and rel(tr, otr) < 1e-5


def test_dispersion_errors(lbem):
    import torch

    p = _problem((16, 20), 13, 5)
    s = lbem.Solver(p.shape)
    with pytest.raises(lbem.LbemError) as e:  # no medium yet
        lbem.lbem_set_dispersion(s.h, np.zeros(320, np.float32))
    assert e.value.status == 6
    s.set_problem(p)
    w0 = 1 - 1.0 / np.asarray(p.eps_r, np.float32).astype(np.float64)
    over = np.ascontiguousarray((4 * w0 + 0.01).ravel(), np.float32)
    for wp2, wr2, g in ((over, None, None), (np.full(320, -0.1, np.float32), None, None),
                        (np.zeros(320, np.float32), None, np.full(320, np.nan, np.float32))):
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_dispersion(s.h, wp2, wr2, g)
        assert e.value.status == 3
    # a medium that would break the pole's bound is refused and the old one kept
    lbem.lbem_set_dispersion(s.h, np.ascontiguousarray((3.9 * w0).ravel(), np.float32))
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_set_medium(s.h, np.ascontiguousarray(np.asarray(p.eps_r, np.float32).ravel() * 0.9))
    assert e.value.status == 3
    with pytest.raises(lbem.LbemError):  # the adjoint is non-dispersive only
        lbem.lbem_forward_record(s.h, 4, 2)
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_batch_create([s.h], torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 1
    lbem.lbem_set_dispersion(s.h, None)  # removed: the plain scheme again
    assert lbem.lbem_info(s.h)[1] == 5 * 16 * 32 * 4
    s.close()
    for shape, kw in (((8, 32), dict(storage="bf16")), ((4, 4, 8), {})):
        h = lbem.Solver(shape, **kw)
        n = int(np.prod(shape))
        lbem.lbem_set_medium(h.h, np.full(n, 2.0, np.float32))
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_dispersion(h.h, np.zeros(n, np.float32))
        assert e.value.status == 1
        h.close()
