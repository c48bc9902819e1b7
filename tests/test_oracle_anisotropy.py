"""Pins of the oracle's anisotropic media (different weights per axis, 2D).

The paper says only that choosing different weights for particles moving along different axes models anisotropic
media.  The oracle's reading: a uniform in-plane relative permeability tensor diag(mu_xx, mu_yy) and a
heterogeneous eps_r; axis a moves at c_a^2 = f_a cbar^2 (f_x = r, f_y = 1/r, r = sqrt(mu_xx/mu_yy),
cbar^2 = c_ref^2/(eps_r sqrt(mu_xx mu_yy))), so c_x^2 = c_ref^2/(eps_r mu_yy) is the speed along x, as TM
Maxwell with that tensor has it; E_z = -cbar^2 sigma and B_x = r (g_4 - g_2), B_y = (g_1 - g_3)/r.

What pins it, other than the oracle itself: r = 1 is the isotropic scheme (pinned by test_oracle_pins); the
discrete dispersion relation of per-axis speeds, sin^2(omega/2) = c_x^2 sin^2(kx/2) + c_y^2 sin^2(ky/2) (the
scheme's finite-difference form with the 5-point Laplacian split by axis); the ratio |B|/|E_z| of plane waves
tends to 1/c along the direction of travel (the field scaling, second order); the invariant sum g^2/w with
per-axis weights is exact; and 2D TM Maxwell with the tensor, solved by an independent staggered-grid program,
agrees at second order on a heterogeneous medium.
"""
import numpy as np
import pytest

import oracle as O

C2 = 0.5  # c_ref^2 in 2D


def _plane(w_eps, aniso, mode, N=24, T=60):
    m = O.medium(2, np.full((N, N), w_eps), aniso=aniso)
    kx, ky = 2 * np.pi * mode[0] / N, 2 * np.pi * mode[1] / N
    y, x = np.mgrid[0:N, 0:N]
    E = np.zeros((N, N, 3))
    E[..., 2] = np.cos(kx * x + ky * y)
    g = O.init_state(m, E=E)
    basis = np.exp(-1j * (kx * x + ky * y))
    amp = []
    for _ in range(T):
        Ef, _ = O.fields(m, g)
        amp.append(np.real((Ef[..., 2] * basis).sum()) / (N * N / 2))
        O.run(m, g, 1)
    return np.array(amp), kx, ky


def test_isotropic_tensor_is_the_plain_scheme_with_uniform_mu():
    rng = np.random.default_rng(5)
    shape = (11, 13)
    eps = 1.5 + 2 * rng.random(shape)
    E = np.zeros(shape + (3,))
    B = np.zeros_like(E)
    E[..., 2] = rng.standard_normal(shape)
    B[..., :2] = rng.standard_normal(shape + (2,))
    src = dict(site=np.array([0, 40, 142]), comp=np.full(3, 2), amp=rng.standard_normal((3, 30)))
    rec = dict(site=np.array([3, 77, 142]), comp=np.array([2, 3, 4]))
    for mu in (1.0, 1.7):
        m0 = O.medium(2, eps, np.full(shape, mu))
        m1 = O.medium(2, eps, aniso=(mu, mu))
        assert m1.aniso_r == 1.0
        g0, g1 = O.init_state(m0, E, B), O.init_state(m1, E, B)
        t0 = O.run(m0, g0, 30, sources=src, receivers=rec)
        t1 = O.run(m1, g1, 30, sources=src, receivers=rec)
        np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-13)
        np.testing.assert_allclose(t1, t0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("aniso", [(1.0, 2.0), (3.0, 1.5), (0.8, 1.9)])
@pytest.mark.parametrize("mode", [(3, 0), (0, 4), (2, 5), (7, 7)])
def test_plane_waves_follow_the_per_axis_dispersion(aniso, mode):
    w_eps = 1.6
    amp, kx, ky = _plane(w_eps, aniso, mode)
    cx2, cy2 = C2 / (w_eps * aniso[1]), C2 / (w_eps * aniso[0])
    om = 2 * np.arcsin(np.sqrt(cx2 * np.sin(kx / 2) ** 2 + cy2 * np.sin(ky / 2) ** 2))
    t = np.arange(amp.size)
    b = (amp[1] - amp[0] * np.cos(om)) / np.sin(om)
    np.testing.assert_allclose(amp, amp[0] * np.cos(om * t) + b * np.sin(om * t), rtol=0, atol=1e-12)


def test_field_ratio_of_travelling_waves_tends_to_one_over_the_axis_speed():
    """A wave travelling along x (E_z = cos(kx - w t), B_y from the equilibrium of the travelling wave) keeps
    |B_y| / |E_z| -> 1/c_x; along y, |B_x| / |E_z| -> 1/c_y; error falling ~4x per halving of k."""
    w_eps, aniso = 1.3, (2.5, 1.2)
    cx, cy = np.sqrt(C2 / (w_eps * aniso[1])), np.sqrt(C2 / (w_eps * aniso[0]))
    for axis, c in ((0, cx), (1, cy)):
        errs = []
        for N in (32, 64, 128):
            k = 2 * np.pi / N
            shape = (N, 4) if axis == 1 else (4, N)
            m = O.medium(2, np.full(shape, w_eps), aniso=aniso)
            y, x = np.mgrid[0:shape[0], 0:shape[1]]
            ph = k * (x if axis == 0 else y)
            E = np.zeros(shape + (3,))
            B = np.zeros_like(E)
            E[..., 2] = np.cos(ph)
            if axis == 0:
                B[..., 1] = -np.cos(ph) / c  # a wave moving towards +x: B_y = -E_z / c
            else:
                B[..., 0] = np.cos(ph) / c  # towards +y: B_x = E_z / c
            g = O.init_state(m, E, B)
            O.run(m, g, N // 2)  # half a period
            Ef, Bf = O.fields(m, g)
            e = np.abs(np.fft.fft(Ef[..., 2].mean(axis=axis))[1])
            bcomp = Bf[..., 1] if axis == 0 else Bf[..., 0]
            bb = np.abs(np.fft.fft(bcomp.mean(axis=axis))[1])
            errs.append(abs(bb / e * c - 1))
        assert errs[2] < 2e-3 and 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, errs


def test_invariant_with_per_axis_weights_is_exact():
    rng = np.random.default_rng(9)
    shape = (14, 17)
    E = np.zeros(shape + (3,))
    B = np.zeros_like(E)
    E[..., 2] = rng.standard_normal(shape)
    B[..., :2] = rng.standard_normal(shape + (2,))
    m = O.medium(2, np.full(shape, 1.4), aniso=(1.1, 2.3))
    g = O.init_state(m, E, B)
    inv0 = O.diagnostics(m, g)[1]
    O.run(m, g, 200)
    assert abs(O.diagnostics(m, g)[1] / inv0 - 1) < 1e-13


def _yee_tm(eps, mxx, myy, Ez0, T, dt):
    """2D TM Maxwell with diag(mu_xx, mu_yy) on a periodic unit-spaced staggered grid (E_z at nodes, H_x at
    y + 1/2, H_y at x + 1/2), leapfrog in time; units with c_ref^2 = C2: eps_r / C2 and mu as given."""
    e = eps / C2
    Ez = Ez0.copy()
    Hx = np.zeros_like(Ez)
    Hy = np.zeros_like(Ez)
    # start H at -dt/2 consistent with E at 0 at rest: first half step
    Hx -= 0.5 * dt / mxx * (np.roll(Ez, -1, 0) - Ez)
    Hy += 0.5 * dt / myy * (np.roll(Ez, -1, 1) - Ez)
    nstep = int(round(T / dt))
    for _ in range(nstep):
        Ez += dt / e * ((Hy - np.roll(Hy, 1, 1)) - (Hx - np.roll(Hx, 1, 0)))
        Hx -= dt / mxx * (np.roll(Ez, -1, 0) - Ez)
        Hy += dt / myy * (np.roll(Ez, -1, 1) - Ez)
    return Ez


def test_agrees_with_an_independent_staggered_grid_maxwell_solver():
    """A smooth pulse in a smooth heterogeneous eps_r with mu = diag(2, 1): the oracle's E_z after T steps and a
    fine-time-step Yee solution on the same grid agree; refining the grid by 2 (and scaling the medium and pulse
    with it) shrinks the difference ~4x."""
    diffs = []
    for N in (48, 96):
        h = 48 / N
        y, x = np.mgrid[0:N, 0:N] * h
        eps = 2.0 + 0.5 * np.sin(2 * np.pi * x / 48) * np.cos(2 * np.pi * y / 48)
        Ez0 = np.exp(-((x - 24) ** 2 + (y - 24) ** 2) / (2 * 4.0 ** 2))
        m = O.medium(2, eps, aniso=(2.0, 1.0))
        E = np.zeros((N, N, 3))
        E[..., 2] = Ez0
        g = O.init_state(m, E)
        steps = int(24 / h)
        O.run(m, g, steps)
        lb = O.fields(m, g)[0][..., 2]
        yee = _yee_tm(eps, 2.0, 1.0, Ez0, steps, 0.05)
        diffs.append(np.sqrt(np.mean((lb - yee) ** 2)) / np.sqrt(np.mean(yee ** 2)))
    assert diffs[1] < 0.02 and diffs[0] / diffs[1] > 3.0, diffs
