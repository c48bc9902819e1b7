"""GPU library vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 of E and B, and of receiver traces): FP32 storage
<= 1e-5 at the 128^2 / 500-step homogeneous case and on small grids, <= 1e-4
after 5000 steps.  Full-size grids are compared element by element over a
bounded number of steps and, after the full number of steps, through the
exact finite-difference identities that every FP32 state must satisfy.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import gpu_run, oracle_run, rel, f32
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


def _problem_small(D, shape, seed, nsteps, mu=True, nsrc=5, nrec=12):
    eps, mu_r = W.random_medium(shape, seed, mu=mu)
    p = W.Problem(f"small{D}", D, shape, eps, mu_r, nsteps)
    E, B = W.random_fields(shape, seed + 1, 0.3)
    p.E0, p.B0 = E, B
    rng = np.random.default_rng(seed + 2)
    n = int(np.prod(shape))
    p.src_site = rng.choice(n, nsrc, replace=n < nsrc).astype(np.int64)
    p.src_site[0] = 0
    p.src_site[-1] = n - 1
    p.src_comp = (rng.integers(0, 3, nsrc) if D == 3 else np.full(nsrc, 2)).astype(np.int32)
    p.src_amp = rng.standard_normal((nsrc, nsteps))
    p.rec_site = rng.choice(n, nrec, replace=True).astype(np.int64)
    p.rec_comp = rng.integers(0, 6, nrec).astype(np.int32)
    return p


def _check(p, storage="f32", tol=1e-5, nsteps=None, **kw):
    E, B, tr = gpu_run(p, storage, nsteps=nsteps, **kw)
    oE, oB, otr, _, _ = oracle_run(p, nsteps=nsteps)
    assert rel(E, oE) < tol, rel(E, oE)
    assert rel(B, oB) < tol, rel(B, oB)
    if otr.size:
        assert rel(tr, otr) < tol, rel(tr, otr)
    return rel(E, oE), rel(B, oB)


def test_homogeneous_pulse_128_500_steps(lbem):
    p = W.homogeneous_pulse(128, 6.0, 500)
    eE, eB = _check(p, tol=1e-5)
    print(f"128^2 x 500 FP32: rel-L2 E {eE:.2e} B {eB:.2e}")


@pytest.mark.parametrize("shape", [(23, 37), (7, 130), (3, 5), (1, 1), (4, 1), (1, 9), (33, 129)])
def test_small_ragged_2d(lbem, shape):
    _check(_problem_small(2, shape, 11, 40), tol=1e-5)


@pytest.mark.parametrize("shape", [(7, 9, 13), (3, 5, 130), (1, 1, 1), (2, 3, 1), (5, 1, 6)])
def test_small_ragged_3d(lbem, shape):
    _check(_problem_small(3, shape, 21, 25), tol=1e-5)


@pytest.mark.parametrize("D,shape", [(2, (17, 45)), (3, (6, 7, 9))])
def test_fields_round_trip(lbem, D, shape):
    p = _problem_small(D, shape, 31, 1)
    if D == 2:
        p.E0[..., :2] = 0
        p.B0[..., 2] = 0
    E, B, _ = gpu_run(p, nsteps=0)
    np.testing.assert_allclose(E, f32(p.E0), rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(B, f32(p.B0), rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("D,shape", [(2, (40, 52)), (3, (10, 11, 12))])
def test_diagnostics_match_oracle(lbem, D, shape):
    p = _problem_small(D, shape, 41, 30, mu=False)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    s.step(30)
    d = s.diagnostics()
    s.close()
    _, _, _, m, g = oracle_run(p)
    od = O.diagnostics(m, g)
    for a, b in zip(d, od):
        assert abs(a - b) <= 1e-5 * abs(b) + 1e-9, (d, od)


def test_5000_steps_fp32_heterogeneous_256(lbem):
    """1024^2 recipe (n = 1 + 2 s, smoothing 20 cells, Ricker at ~20 cells per wavelength) at 256^2."""
    p = W.heterogeneous_2d(256, seed=1, nsteps=5000)
    eE, eB = _check(p, tol=1e-4)
    print(f"256^2 x 5000 FP32: rel-L2 E {eE:.2e} B {eB:.2e}")


def test_1024_full_size_elementwise_200_steps(lbem):
    p = W.heterogeneous_2d(1024, seed=1, nsteps=200)
    _check(p, tol=1e-5)


def _leapfrog_residual(E3, cL2, S3):
    """max |E^{t+1} - 2E^t + E^{t-1} - (c2 Lap5 E^t + S^t + c2/2 Lap5 S^t - S^{t-1})| over the grid."""
    import crosscheck as X

    Em, E0, Ep = E3
    Sm, S0 = S3
    r = Ep - 2 * E0 + Em - (cL2 * X.lap5(E0) + S0 + 0.5 * cL2 * X.lap5(S0) - Sm)
    return np.abs(r).max()


@pytest.mark.parametrize("n,seed", [(1024, 1), (4096, 2)])
def test_full_size_5000_steps_satisfy_exact_fd_form(lbem, n, seed):
    """After the full 5000 steps, the FP32 state obeys the scheme's exact FD form (a property the FP64
    oracle is pinned to) at every site, to FP32 rounding of one step."""
    import torch

    p = W.heterogeneous_2d(n, seed=seed, nsteps=5000)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    s.step(4998)
    Es = []
    for _ in range(3):
        E, _ = s.fields()
        Es.append(E[2].double().cpu().numpy())
        s.step(1)
    torch.cuda.synchronize()
    m = O.medium(2, f32(p.eps_r))
    amp = f32(p.src_amp[0])
    S = []
    for t in (4998, 4999):
        st = np.zeros(p.shape)
        st.flat[p.src_site[0]] = -m.ceff2.flat[p.src_site[0]] * amp[t]
        S.append(st)
    r = _leapfrog_residual(Es, m.cL2, S)
    scale = max(np.abs(e).max() for e in Es)
    s.close()
    assert r < 2e-6 * scale, (r, scale)


def test_4096_full_size_elementwise_20_steps(lbem):
    p = W.heterogeneous_2d(4096, seed=2, nsteps=20)
    _check(p, tol=1e-5)


def test_192_cubed_full_size_elementwise_3_steps(lbem):
    p = W.heterogeneous_3d(192, nsteps=3)
    B = np.zeros(p.shape + (3,))
    p.E0, B0 = W.random_fields(p.shape, 5, 0.1)
    p.B0 = B0
    _check(p, tol=1e-5)


@pytest.mark.parametrize("steps_per_pass", [1, 2])
@pytest.mark.parametrize("storage", ["f16", "bf16", "i16b"])
def test_reduced_storage_short_run_tracks_oracle(lbem, storage, steps_per_pass):
    """Half-precision storage on the homogeneous 128^2 pulse: error within the format's rounding bound
    2 u sqrt(N/3) (u = unit roundoff; 2^-11 FP16, 2^-8 BF16, 2 * 2^-16 block int16), with single steps and
    with two steps per launch (one rounding per two steps).  A regression check of each codec against the
    rounding-walk model; the benchmark spec's 1e-3 bar is asserted on config 2's 5000-step crop below."""
    p = W.homogeneous_pulse(128, 6.0, 500)
    E, B, _ = gpu_run(p, storage, steps_per_pass=steps_per_pass)
    oE, oB, _, _, _ = oracle_run(p)
    u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "i16b": 2.0 ** -15}[storage]
    bound = 2 * u * np.sqrt(500 / 3)
    eE, eB = rel(E, oE), rel(B, oB)
    print(f"{storage} 128^2 x 500, {steps_per_pass} step(s)/launch: rel-L2 E {eE:.2e} B {eB:.2e} "
          f"(bound {bound:.1e})")
    assert eE < bound and eB < bound


def test_variants_and_graphs_are_bitwise_identical(lbem):
    p = _problem_small(2, (64, 300), 51, 30)
    ref = gpu_run(p, variant=0)
    n = lbem.lbem_get_variant(lbem.Solver((4, 4)).h)[1]
    for v in range(n):
        for graphs in (False, True):
            out = gpu_run(p, variant=v, graphs=graphs)
            for a, b in zip(out, ref):
                np.testing.assert_array_equal(a, b)


def test_3d_launch_shapes_agree(lbem):
    p = _problem_small(3, (6, 7, 70), 52, 20)
    ref = gpu_run(p, variant=0)
    out = gpu_run(p, variant=1)
    for a, b in zip(out, ref):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-6 * max(1.0, np.abs(b).max()))


def test_host_and_device_pointers_agree(lbem):
    import torch

    p = _problem_small(2, (20, 30), 61, 15, mu=True)
    ref = gpu_run(p)
    s = lbem.Solver(p.shape)
    lbem.lbem_set_medium(s.h, np.ascontiguousarray(p.eps_r, np.float32).ravel(),
                         np.ascontiguousarray(p.mu_r, np.float32).ravel())
    lbem.lbem_set_sources(s.h, p.src_site, p.src_comp, p.src_amp)
    lbem.lbem_set_receivers(s.h, p.rec_site, p.rec_comp, p.nsteps)
    lbem.lbem_set_fields(s.h, np.ascontiguousarray(np.moveaxis(p.E0, -1, 0), np.float32).ravel(),
                         np.ascontiguousarray(np.moveaxis(p.B0, -1, 0), np.float32).ravel())
    s.step(15)
    E = np.zeros(3 * s.nsite, np.float32)
    B = np.zeros(3 * s.nsite, np.float32)
    lbem.lbem_fields(s.h, E, B)
    tr = np.zeros(p.rec_site.size * 15, np.float32)
    lbem.lbem_traces(s.h, tr)
    s.close()
    np.testing.assert_array_equal(np.moveaxis(E.reshape((3,) + p.shape), 0, -1), ref[0])
    np.testing.assert_array_equal(np.moveaxis(B.reshape((3,) + p.shape), 0, -1), ref[1])
    np.testing.assert_array_equal(tr.reshape(-1, 15), ref[2])


def test_save_and_load_state_resume_bitwise(lbem):
    import torch

    p = _problem_small(2, (31, 70), 71, 60)
    ref = gpu_run(p, nsteps=60)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    s.step(25)
    n, nbytes = lbem.lbem_info(s.h)
    snap = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lbem.lbem_save_state(s.h, snap)
    s.step(10)  # diverge, then resume from the snapshot
    lbem.lbem_load_state(s.h, snap, 25)
    s.step(35)
    E, B = s.fields()
    torch.cuda.synchronize()
    s.close()
    np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])


def test_errors_are_reported_and_handle_survives(lbem):
    import torch

    s = lbem.Solver((8, 8))
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_step(s.h, 1)
    assert e.value.status == 6  # no medium yet
    bad = torch.ones(64, device="cuda")
    bad[5] = 0.25  # faster than the reference speed: w0 < 0
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_set_medium(s.h, bad)
    assert e.value.status == 3
    bad[5] = float("nan")
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_set_medium(s.h, bad)
    assert e.value.status == 3
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_set_receivers(s.h, [64], [2], 10)
    assert e.value.status == 1
    with pytest.raises(lbem.LbemError) as e:
        lbem.lbem_set_sources(s.h, [3], [7], np.zeros((1, 4), np.float32))
    assert e.value.status == 1
    lbem.lbem_set_medium(s.h, torch.ones(64, device="cuda"))
    lbem.lbem_set_fields(s.h)
    lbem.lbem_step(s.h, 3)
    assert lbem.lbem_time(s.h) == 3
    s.close()


def test_homogeneous_invariant_conserved_full_size(lbem):
    """sum g^2/w is exactly conserved by the scheme (homogeneous, source-free); FP32 drift stays small."""
    p = W.homogeneous_pulse(4096, 40.0, 1000)
    p.eps_r = np.full(p.shape, 2.0)  # w0 = 1/2
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    d0 = s.diagnostics()
    s.step(1000)
    d1 = s.diagnostics()
    s.close()
    assert abs(d1[1] - d0[1]) < 1e-5 * d0[1], (d0, d1)


def _crop512_problem():
    big = W.heterogeneous_2d(4096, seed=2, nsteps=5000)
    c0 = 2048 - 256
    eps = big.eps_r[c0:c0 + 512, c0:c0 + 512].copy()
    n_idx = np.sqrt(eps)
    recs = W.circle_receivers((256, 256), 128, 64)
    return W.point_source_problem(2, (512, 512), n_idx, 5000, (256, 256), 64, recs, name="crop512")


_CROP_REPORT = {}


def _crop512_report():
    """rel-L2 (E, B, traces) against the FP64 oracle of the 512^2 crop x 5000 steps, per (storage, steps per
    launch); computed once per session."""
    if not _CROP_REPORT:
        p = _crop512_problem()
        oE, oB, otr, _, _ = oracle_run(p)
        for st in ("f32", "f16", "bf16", "i16b"):
            for spp in (1, 2):
                E, B, tr = gpu_run(p, st, steps_per_pass=spp)
                _CROP_REPORT[(st, spp)] = (rel(E, oE), rel(B, oB), rel(tr, otr))
        print("512^2 crop x 5000 rel-L2 (E, B, traces) by (storage, steps per launch):",
              {f"{k[0]}/{k[1]}": tuple(f"{x:.2e}" for x in v) for k, v in _CROP_REPORT.items()})
    return _CROP_REPORT


def test_storage_forms_5000_steps_on_512_crop_of_4096_medium(lbem):
    """The 4096^2 (seed 2) medium's central 512^2 crop run in FP64 (oracle) and on the GPU in every storage form for
    5000 steps, Ricker source at the crop centre (config 2, reading R11).  FP32 must meet the benchmark spec's 1e-4 and
    block-int16 its reduced-precision bar 1e-3, on E, B and the receiver traces, in single- and two-step launches.
    FP16 and BF16 miss 1e-3 (see the strict xfail below); here they are only held to the rounding-walk model of a
    neutral scheme, 2 u sqrt(N/3), which catches a broken codec."""
    report = _crop512_report()
    u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
    for spp in (1, 2):
        assert max(report[("f32", spp)]) < 1e-4, report[("f32", spp)]
        assert max(report[("i16b", spp)]) < 1e-3, report[("i16b", spp)]
        for st in ("f16", "bf16"):
            assert max(report[(st, spp)]) < 2 * u[st] * np.sqrt(5000 / 3), (st, spp, report[(st, spp)])


@pytest.mark.xfail(strict=True, reason="known miss: FP16 and BF16 storage round every stored value to 11 / 8 "
                   "significant bits and the neutral scheme lets those errors random-walk (~u sqrt(N)); at 5000 steps "
                   "they reach 7.5e-3 (FP16) and 6.0e-2 (BF16) against the 1e-3 bar")
@pytest.mark.parametrize("st", ["f16", "bf16"])
def test_f16_bf16_storage_meet_reduced_precision_bar(lbem, st):
    """The benchmark spec's reduced-precision bar, 1e-3 relative L2 on E and B after 5000 steps, asserted as it stands
    for FP16 and BF16 storage: a documented miss, reported as xfail (an unexpected pass fails the suite)."""
    report = _crop512_report()
    assert max(max(report[(st, 1)][:2]), max(report[(st, 2)][:2])) <= 1e-3, report


def test_mu_heterogeneous_256_1000_steps(lbem):
    """Heterogeneous permeability (the B x grad ln mu source of Eq. 3 acts at every site): 256^2 medium with the
    headline recipe's refractive index and mu_r = 1 + s2, 1000 steps, FP32 against the oracle."""
    p = W.heterogeneous_2d_mu(256, seed=1, nsteps=1000, sigma=12.0)
    eE, eB = _check(p, tol=1e-4)
    print(f"mu-heterogeneous 256^2 x 1000 FP32: rel-L2 E {eE:.2e} B {eB:.2e}")


@pytest.mark.slow
def test_1024_heterogeneous_5000_steps_64_receivers_elementwise(lbem):
    """1024^2 heterogeneous medium (seed 1), Ricker point source, 64 receivers, 5000 steps, FP32: every field
    value and every trace sample against the FP64 oracle (about a minute of oracle time on 16 cores)."""
    p = W.heterogeneous_2d(1024, seed=1, nsteps=5000)
    eE, eB = _check(p, tol=1e-4)
    print(f"1024^2 x 5000 FP32: rel-L2 E {eE:.2e} B {eB:.2e}")


def test_3d_48_cubed_1000_steps_forward(lbem):
    """3D heterogeneous medium (48^3, n in [1, 3]), Ricker j_z, 1000 steps, FP32 vs the FP64 oracle."""
    p = W.heterogeneous_3d(48, seed=4, nsteps=1000, sigma=4.0, plane_dz=12, rec_grid=(4, 4))
    eE, eB = _check(p, tol=1e-4)
    print(f"48^3 x 1000 FP32: rel-L2 E {eE:.2e} B {eB:.2e}")


def test_watchdog_passes_stable_runs_and_stops_overflow(lbem):
    p = W.heterogeneous_2d(128, seed=3, nsteps=300, sigma=6.0, nrec=4, rec_radius=30)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    lbem.lbem_set_watchdog(s.h, 50, 1e6)
    s.step(300)  # a stable run is not stopped
    assert lbem.lbem_time(s.h) == 300
    # an over-driven source overflows the FP32 state (inf, then nan): the watchdog stops the run
    p.src_amp = np.full_like(p.src_amp, 3e38)
    lbem.lbem_set_sources(s.h, p.src_site, p.src_comp, p.src_amp)
    lbem.lbem_set_fields(s.h)
    with pytest.raises(lbem.LbemError) as e:
        s.step(300)
    assert e.value.status == 4
    assert lbem.lbem_time(s.h) % 50 == 0 and lbem.lbem_time(s.h) < 300
    s.close()


@pytest.mark.parametrize("D,shape", [(2, (37, 50)), (3, (7, 9, 11))])
def test_energy_density_and_poynting_vector(lbem, D, shape):
    """u = |B|^2 + |E|^2/c^2 and P = E x B (paper, Sec. "Heterogeneous media") against the oracle's fields;
    u summed over the grid equals the FP64 energy diagnostic."""
    import torch

    p = _problem_small(D, shape, 81, 25, mu=False)
    s = lbem.Solver(p.shape)
    s.set_problem(p)
    s.step(25)
    n = s.nsite
    u = torch.empty(n, device="cuda")
    P = torch.empty(3 * n, device="cuda")
    lbem.lbem_energy_flux(s.h, u, P)
    d = s.diagnostics()
    torch.cuda.synchronize()
    s.close()
    oE, oB, _, m, _ = oracle_run(p)
    ou = (oB ** 2).sum(-1) + (oE ** 2).sum(-1) / m.ceff2
    oP = np.cross(oE, oB)
    gu = u.cpu().double().numpy().reshape(shape)
    gP = np.moveaxis(P.cpu().double().numpy().reshape((3,) + shape), 0, -1)
    assert rel(gu, ou) < 1e-5 and rel(gP, oP) < 1e-5
    assert abs(gu.sum() - d[0]) < 1e-5 * d[0]


def test_extreme_index_contrast(lbem):
    """Degenerate weights: refractive index from 1 (rest weight 0) to 100 (rest weight 1 - 1e-4)."""
    shape = (40, 44)
    rng = np.random.default_rng(90)
    n_idx = np.exp(rng.uniform(0.0, np.log(100.0), shape))
    n_idx[0, 0] = 1.0
    p = W.Problem("contrast", 2, shape, n_idx ** 2, None, 60)
    p.E0, p.B0 = W.random_fields(shape, 91, 0.3)
    p.E0[..., :2] = 0
    p.B0[..., 2] = 0
    _check(p, tol=1e-5)


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 45), (16, 128), (33, 257), (70, 300), (130, 131),
                                   (9, 1), (200, 7), (301, 777), (40, 4), (50, 264)])
def test_two_step_blocking_is_bitwise_identical(lbem, shape):
    """Two steps per pass through a shared-memory tile give the same bits as single steps, for every tile
    shape, with sources and receivers anywhere (including tile edges and periodic wraps), odd step counts
    and graphs."""
    p = _problem_small(2, shape, 95, 41, mu=False, nsrc=7, nrec=15)
    ref = gpu_run(p, steps_per_pass=1)
    import torch

    probe = lbem.Solver((4, 4))
    # FP32: tile shapes 0-6, the register-streaming kernel 7-8, the strip-streaming kernel 9-14
    nsh = lbem.lbem_get_temporal_blocking(probe.h)[2]
    probe.close()
    assert nsh == 15
    for tile_shape, graphs in [(k, g) for k in range(nsh) for g in (False, True)]:
        stream = torch.cuda.Stream() if graphs else None
        s = lbem.Solver(p.shape, stream=stream.cuda_stream if stream else None)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, 2, tile_shape)
        if graphs:
            lbem.lbem_set_graphs(s.h, True)
        s.step(20)
        s.step(21)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_check_guards(s.h)
        s.close()
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
        np.testing.assert_array_equal(tr.cpu().double().numpy(), ref[2])


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 45), (16, 128), (33, 257), (70, 300), (130, 131),
                                   (9, 1), (200, 7), (301, 777), (40, 4), (50, 264)])
def test_three_step_blocking_is_bitwise_identical(lbem, shape):
    """Three steps per launch (FP32): the same bits as single steps, for every tile shape, with sources and
    receivers anywhere, step counts that leave a pair or a single step over, and graphs."""
    p = _problem_small(2, shape, 96, 41, mu=False, nsrc=7, nrec=15)
    ref = gpu_run(p, steps_per_pass=1)
    import torch

    nsh = None
    for tile_shape, graphs in [(k, g) for k in range(3) for g in (False, True)]:
        stream = torch.cuda.Stream() if graphs else None
        s = lbem.Solver(p.shape, stream=stream.cuda_stream if stream else None)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, 3, tile_shape)
        spp, _, nsh = lbem.lbem_get_temporal_blocking(s.h)
        assert spp == 3
        if graphs:
            lbem.lbem_set_graphs(s.h, True)
        s.step(20)
        s.step(19)
        s.step(2)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_sync(s.h)
        lbem.lbem_check_guards(s.h)
        s.close()
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
        np.testing.assert_array_equal(tr.cpu().double().numpy(), ref[2])
    assert nsh == 3


def test_three_step_blocking_full_size_matches_oracle(lbem):
    """4096^2 heterogeneous medium, 21 steps: every three-step tile shape gives the bits of single steps'
    two-step equivalent, and the result matches the oracle."""
    p = W.heterogeneous_2d(4096, seed=2, nsteps=21)
    import torch

    res = []
    for spp, tile_shape in ((2, 0), (3, 0), (3, 1), (3, 2)):
        s = lbem.Solver(p.shape)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, spp, tile_shape)
        s.step(21)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        s.close()
        res.append((E.cpu(), B.cpu(), tr.cpu()))
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert torch.equal(a, b)
    E, B, tr = res[1]
    oE, oB, otr, _, _ = oracle_run(p)
    assert rel(np.moveaxis(E.cpu().double().numpy(), 0, -1), oE) < 1e-5
    assert rel(np.moveaxis(B.cpu().double().numpy(), 0, -1), oB) < 1e-5
    assert rel(tr.cpu().double().numpy(), otr) < 1e-5


@pytest.mark.parametrize("spp", [2, 3])
def test_autotuned_stepping_is_bitwise_identical(lbem, spp):
    """lbem_autotune picks among single steps and every two- (three-) step tile shape; whatever it keeps, the
    results are those of single steps, and the state it timed on is restored."""
    p = _problem_small(2, (150, 390), 97, 33, mu=False, nsrc=5, nrec=9)
    ref = gpu_run(p, steps_per_pass=1)
    import torch

    s = lbem.Solver(p.shape)
    s.set_problem(p)
    lbem.lbem_set_temporal_blocking(s.h, spp, -1)
    lbem.lbem_autotune(s.h, 6)
    got_spp, shape, nsh = lbem.lbem_get_temporal_blocking(s.h)
    assert 1 <= got_spp <= spp and 0 <= shape < max(nsh, 1)
    assert lbem.lbem_time(s.h) == 0
    s.step(33)
    E, B = s.fields()
    tr = s.traces(p.rec_site.size)
    torch.cuda.synchronize()
    s.close()
    np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
    np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
    np.testing.assert_array_equal(tr.cpu().double().numpy(), ref[2])


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (17, 45), (16, 128), (33, 257), (70, 300), (130, 131),
                                   (9, 1), (200, 7), (301, 777), (40, 4), (50, 264)])
def test_two_step_blocking_heterogeneous_mu_is_bitwise_identical(lbem, shape):
    """Two steps per launch with a heterogeneous permeability (the grad ln mu planes staged beside c_L^2): the
    same bits as single steps for both tile shapes and the strip kernel, with sources and receivers anywhere, odd
    step counts and graphs; a fourth shape does not exist for such a medium, and three steps per launch fall back
    to two (uniform mu only), as does a shape set before the medium."""
    p = _problem_small(2, shape, 98, 41, mu=True, nsrc=7, nrec=15)
    ref = gpu_run(p, steps_per_pass=1)
    import torch

    for spp_set, tile_shape, graphs in [(2, k, g) for k in range(3) for g in (False, True)] + [(3, 0, False),
                                                                                              (2, 8, False)]:
        stream = torch.cuda.Stream() if graphs else None
        s = lbem.Solver(p.shape, stream=stream.cuda_stream if stream else None)
        if tile_shape < 3:
            s.set_problem(p)
            lbem.lbem_set_temporal_blocking(s.h, spp_set, tile_shape)
        else:
            lbem.lbem_set_temporal_blocking(s.h, spp_set, tile_shape)
            s.set_problem(p)
        spp, _, nsh = lbem.lbem_get_temporal_blocking(s.h)
        assert spp == 2 and nsh == 3
        with pytest.raises(lbem.LbemError):
            lbem.lbem_set_temporal_blocking(s.h, 2, 3)
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
        np.testing.assert_array_equal(np.moveaxis(E.cpu().double().numpy(), 0, -1), ref[0])
        np.testing.assert_array_equal(np.moveaxis(B.cpu().double().numpy(), 0, -1), ref[1])
        np.testing.assert_array_equal(tr.cpu().double().numpy(), ref[2])


def test_default_two_step_shape_follows_grid_size(lbem):
    """An FP32 grid of uniform mu with at least 12M sites launches the strip-streaming kernel (shape 10) unless a
    shape is set; smaller grids, and any grid once a shape is set, launch that shape (0 by default)."""
    for shape, want in (((3000, 4096), 10), ((2048, 2048), 0)):
        s = lbem.Solver(shape)
        assert lbem.lbem_get_temporal_blocking(s.h)[:2] == (2, want)
        lbem.lbem_set_temporal_blocking(s.h, 2, 0)
        assert lbem.lbem_get_temporal_blocking(s.h)[:2] == (2, 0)
        lbem.lbem_set_temporal_blocking(s.h, 2, -1)
        assert lbem.lbem_get_temporal_blocking(s.h)[:2] == (2, want)
        s.close()


def test_two_step_blocking_rejects_bad_arguments(lbem):
    s = lbem.Solver((16, 16))
    for steps, shape in ((0, 0), (4, 0), (2, 15), (3, 3), (2, -2)):
        with pytest.raises(lbem.LbemError) as e:
            lbem.lbem_set_temporal_blocking(s.h, steps, shape)
        assert e.value.status == 1
    s.close()


def test_two_step_blocking_full_size_matches_oracle(lbem):
    """4096^2 heterogeneous medium (the benchmark's launch configuration), 20 steps: every tile shape gives
    the same bits, and the result matches the oracle."""
    p = W.heterogeneous_2d(4096, seed=2, nsteps=20)
    import torch

    res = []
    for tile_shape in range(15):
        s = lbem.Solver(p.shape)
        s.set_problem(p)
        lbem.lbem_set_temporal_blocking(s.h, 2, tile_shape)
        s.step(20)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        s.close()
        res.append((E.cpu(), B.cpu(), tr.cpu()))
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            assert torch.equal(a, b)
    E, B, tr = res[0]
    oE, oB, otr, _, _ = oracle_run(p)
    assert rel(np.moveaxis(E.cpu().double().numpy(), 0, -1), oE) < 1e-5
    assert rel(np.moveaxis(B.cpu().double().numpy(), 0, -1), oB) < 1e-5
    assert rel(tr.cpu().double().numpy(), otr) < 1e-5
