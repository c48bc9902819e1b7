"""Walls and absorbing layers on the GPU, against the oracle and across stepping modes.

Tolerances as for the periodic parity tests: relative L2 of E, B and the
receiver traces <= 1e-5 against the FP64 oracle on small grids.  Every
stepping mode (single steps, two and three steps per launch with every tile
shape, graphs) must give the same bits, since the sites next to walls are
recomputed after each launch with the same per-site arithmetic.
"""
import numpy as np
import pytest

from gpu_helpers import gpu_run, oracle_run, rel
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu

PEC, PMC = lbem.BC_PEC, lbem.BC_PMC


def _problem(shape, seed, nsteps, bc, layer, gamma_max, mu):
    eps, mu_r = W.random_medium(shape, seed, mu=mu)
    p = W.Problem("walls", 2, shape, eps, mu_r, nsteps)
    p.E0, p.B0 = W.random_fields(shape, seed + 1, 0.3)
    p.E0[..., :2] = 0
    p.B0[..., 2] = 0
    ny, nx = shape
    n = ny * nx
    rng = np.random.default_rng(seed + 2)
    corners = [0, nx - 1, (ny - 1) * nx, n - 1, (ny // 2) * nx, (ny // 2) * nx + nx - 1]
    p.src_site = np.unique(np.concatenate([corners, rng.integers(0, n, 3)])).astype(np.int64)
    p.src_comp = np.full(p.src_site.size, 2, np.int32)
    p.src_amp = rng.standard_normal((p.src_site.size, nsteps))
    p.rec_site = np.unique(np.concatenate([corners, rng.integers(0, n, 6)])).astype(np.int64)
    p.rec_comp = np.array([2, 3, 4] * ((p.rec_site.size + 2) // 3), np.int32)[: p.rec_site.size]
    p.bc = tuple(bc) + (0,)
    p.layer = layer
    p.gamma_max = gamma_max
    return p


CASES = [((1, 1), (PEC, PEC), 0, False), ((3, 5), (PMC, PEC), 1, True), ((17, 45), (PEC, 0), 4, True),
         ((33, 257), (0, PMC), 8, False), ((130, 131), (PEC, PMC), 8, True), ((64, 300), (PMC, PMC), 16, False),
         ((200, 7), (PEC, PEC), 3, True), ((40, 264), (PEC, PEC), 0, True)]


@pytest.mark.parametrize("shape,bc,layer,mu", CASES)
def test_walls_and_layers_match_oracle(lbem, shape, bc, layer, mu):
    p = _problem(shape, 500 + shape[1], 37, bc, layer, 0.3 if layer else 0.0, mu)
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    eE, eB, eT = rel(E, oE), rel(B, oB), rel(tr, otr)
    print(f"{shape} bc {bc} layer {layer} mu {mu}: rel-L2 E {eE:.1e} B {eB:.1e} traces {eT:.1e}")
    assert eE < 1e-5 and eB < 1e-5 and eT < 1e-5


@pytest.mark.parametrize("shape,bc,layer,mu", CASES)
def test_walls_are_bitwise_identical_across_stepping_modes(lbem, shape, bc, layer, mu):
    import torch

    p = _problem(shape, 600 + shape[0], 41, bc, layer, 0.25 if layer else 0.0, mu)
    ref = gpu_run(p, steps_per_pass=1)
    modes = [(1, 0, True), (2, 0, False), (2, 1, True), (3, 0, False), (3, 2, True)]
    if not mu:  # the other tile shapes, the register-streaming kernel and the strip-streaming kernel
        modes += [(2, k, False) for k in range(2, 15)]
    for spp, tile, graphs in modes:
        stream = torch.cuda.Stream() if graphs else None
        s = lbem.Solver(p.shape, stream=stream.cuda_stream if stream else None)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, spp, tile if tile < lbem.lbem_get_temporal_blocking(s.h)[2] or spp == 3
                                        else 0)
        if graphs:
            lbem.lbem_set_graphs(s.h, True)
        s.step(20)
        s.step(21)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_sync(s.h)
        lbem.lbem_check_guards(s.h)
        s.close()
        msg = f"steps per launch {spp}, tile {tile}, graphs {graphs}"
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0], err_msg=msg)
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1], err_msg=msg)
        np.testing.assert_array_equal(tr.cpu().double().numpy(), ref[2], err_msg=msg)


def test_walls_full_size_match_oracle(lbem):
    """4096^2 heterogeneous medium in a PEC box with a 32-site absorbing layer (the benchmark's wall
    workload), 20 steps in the default launch configuration."""
    p = W.heterogeneous_2d_walls(4096, seed=2, nsteps=20)
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    assert rel(E, oE) < 1e-5 and rel(B, oB) < 1e-5 and rel(tr, otr) < 1e-5


def test_layer_absorbs_on_gpu(lbem):
    """The oracle's absorption pin, on the GPU: a Gaussian E_z slab between two PEC walls comes back from a
    32-site layer (gamma_max = 0.2) with less than 1e-5 of its energy; without the layer all of it returns."""
    import torch

    ny, nx = 4, 600
    x = np.arange(nx)
    E0 = np.zeros((ny, nx, 3))
    E0[..., 2] = np.exp(-((x - nx / 2) / 6.0) ** 2)[None, :]
    T = int(nx / 2 / np.sqrt(0.5)) + 50
    left = []
    for layer, gmax in ((0, 0.0), (32, 0.2)):
        p = W.Problem("slab", 2, (ny, nx), np.ones((ny, nx)), None, T, E0=E0, B0=np.zeros_like(E0))
        p.bc, p.layer, p.gamma_max = (PEC, 0, 0), layer, gmax
        s = lbem.Solver(p.shape)
        s.set_problem(p)
        e0 = lbem.lbem_diagnostics(s.h)[0]
        s.step(T)
        torch.cuda.synchronize()
        left.append(lbem.lbem_diagnostics(s.h)[0] / e0)
        s.close()
    assert abs(left[0] - 1) < 1e-2 and left[1] < 1e-5, left


def test_boundaries_round_trip_and_errors(lbem):
    import torch

    p = _problem((30, 70), 7, 25, (PEC, PMC), 5, 0.3, False)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    assert lbem.lbem_get_boundaries(s.h) == ((PEC, PMC, 0), 5, 0.3)
    for kind, layer, g in (((3, 0, 0), 0, 0.0), ((PEC, 0, PEC), 0, 0.0), ((PEC, 0, 0), -1, 0.0),
                           ((PEC, 0, 0), 2, 1.0), ((0, 0, 0), 2, 0.1), ((PEC, 0, 0), 36, 0.1)):
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_boundaries(s.h, kind, layer, g)
        assert e.value.status == 1
    # walls off again: the periodic result, bit for bit
    q = _problem((30, 70), 7, 25, (0, 0), 0, 0.0, False)
    lbem.lbem_set_boundaries(s.h, (0, 0, 0))
    lbem.lbem_set_fields(s.h, torch.as_tensor(np.moveaxis(q.E0, -1, 0).astype(np.float32).ravel()).cuda(),
                         torch.as_tensor(np.moveaxis(q.B0, -1, 0).astype(np.float32).ravel()).cuda())
    s.step(25)
    E, B = s.fields()
    ref = gpu_run(q)
    np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
    with pytest.raises(lbem.LbemError):  # the adjoint is periodic only
        lbem.lbem_set_boundaries(s.h, (PEC, 0, 0))
        lbem.lbem_forward_record(s.h, 4, 2)
    s.close()
    for kw in (dict(storage="bf16"),):
        h = lbem.Solver((8, 32), **kw)
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_boundaries(h.h, (PEC, 0, 0))
        assert e.value.status == 1
        h.close()
    h2 = lbem.Solver((8, 8))
    with pytest.raises(lbem.LbemError) as e:  # a 2D grid has no z walls
        lbem.lbem_set_boundaries(h2.h, (0, 0, PEC))
    assert e.value.status == 1
    h2.close()
    m = lbem.Solver((16, 16))
    m.set_problem(_problem((16, 16), 9, 5, (PEC, 0), 0, 0.0, False))
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_batch_create([m.h], torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 1
    m.close()


def _problem3(shape, seed, nsteps, bc, layer, mu):
    eps, mu_r = W.random_medium(shape, seed, mu=mu)
    p = W.Problem("walls3", 3, shape, eps, mu_r, nsteps)
    p.E0, p.B0 = W.random_fields(shape, seed + 1, 0.3)
    rng = np.random.default_rng(seed + 2)
    nz, ny, nx = shape
    n = nz * ny * nx
    corners = [0, nx - 1, (ny - 1) * nx, n - 1, n - nx * ny]
    p.src_site = np.unique(np.concatenate([corners, rng.integers(0, n, 3)])).astype(np.int64)
    p.src_comp = (np.arange(p.src_site.size) % 3).astype(np.int32)
    p.src_amp = rng.standard_normal((p.src_site.size, nsteps))
    p.rec_site = np.unique(np.concatenate([corners, rng.integers(0, n, 7)])).astype(np.int64)
    p.rec_comp = (np.arange(p.rec_site.size) % 6).astype(np.int32)
    p.bc = tuple(bc)
    p.layer = layer
    p.gamma_max = 0.3 if layer else 0.0
    return p


CASES3 = [((4, 5, 6), (PEC, 0, 0), 0, False), ((6, 7, 33), (0, PMC, PEC), 2, True),
          ((9, 3, 40), (PEC, PEC, PMC), 1, False), ((5, 8, 64), (PMC, 0, PMC), 2, True)]


@pytest.mark.parametrize("shape,bc,layer,mu", CASES3)
def test_3d_walls_and_layers_match_oracle(lbem, shape, bc, layer, mu):
    p = _problem3(shape, 900 + shape[2], 21, bc, layer, mu)
    outs = [gpu_run(p, variant=v) for v in (0, 1)]
    for a, b in zip(*outs):  # every launch shape takes the kernel that applies walls: the same bits
        np.testing.assert_array_equal(a, b)
    E, B, tr = outs[0]
    oE, oB, otr, _, _ = oracle_run(p)
    eE, eB, eT = rel(E, oE), rel(B, oB), rel(tr, otr)
    print(f"3D {shape} bc {bc} layer {layer} mu {mu}: rel-L2 E {eE:.1e} B {eB:.1e} traces {eT:.1e}")
    assert eE < 1e-5 and eB < 1e-5 and eT < 1e-5


def test_3d_walls_full_size_match_oracle(lbem):
    """192^3 heterogeneous medium in a PEC box with an 8-site absorbing layer, 3 steps."""
    p = W.heterogeneous_3d(192, nsteps=3)
    p.bc, p.layer, p.gamma_max = (PEC, PEC, PEC), 8, 0.2
    E, B, tr = gpu_run(p)
    oE, oB, otr, _, _ = oracle_run(p)
    assert rel(E, oE) < 1e-5 and rel(B, oB) < 1e-5 and rel(tr, otr) < 1e-5
