"""Pins of the oracle's frequency-dispersive permittivity (one Drude-Lorentz pole per site).

Eq. 3 carries a polarization term (a convolution with the time derivative of the permittivity) that the paper
leaves to auxiliary differential equations and does not treat.  The oracle's reading: d_t J + gamma J + wr^2 P =
wp^2 E with J = d_t P; the lattice's zeroth moment carries D/eps_inf, the field is E = D/eps_inf - P, and P enters
the equilibrium's second moment; J at half steps, P at whole ones (time-centred).

What pins it, other than the oracle itself, is the discrete dispersion relation that this reading implies for a
homogeneous medium, derived by hand from the finite-difference form of the scheme: with zeta = exp(-i omega),
A = zeta - 2 + 1/zeta (= -4 sin^2(omega/2)), q = sin^2(kx/2) + sin^2(ky/2),
    A (1 + wp^2 / Q) = -4 c^2 q,   Q = A + (gamma/2)(zeta - 1/zeta) + wr^2,
the discrete counterpart of eps(omega) = 1 + wp^2 / (wr^2 - omega^2 - i gamma omega).  So the Fourier amplitude of
E_z obeys the 4th-order linear recurrence whose characteristic polynomial is zeta^2 [A (Q + wp^2) + 4 c^2 q Q]; for
a lossless Drude medium (wr = gamma = 0) it is a single pair, 4 sin^2(omega/2) = 4 c^2 q + wp^2, the lattice form
of omega^2 = wp^2 + c^2 k^2 (plasma waves).  Plus: no pole (wp = 0) is the plain scheme; a uniform field in a
lossless Drude medium oscillates at 2 sin(omega/2) = wp with D constant; the stability bound wp^2 + wr^2 <= 4 w0.
With an anisotropic tensor (per-axis speeds) the lattice's Laplacian splits by axis, so 4 c^2 q becomes
4 (c_x^2 sin^2(kx/2) + c_y^2 sin^2(ky/2)) in the same relation.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as Pn

import oracle as O

N = 24


def _amplitudes(w_eps, mode, disp, T=60, aniso=None):
    """Fourier amplitude of E_z(t) for the plane wave E_z = cos(k.x) released from equilibrium at rest."""
    m = O.medium(2, np.full((N, N), w_eps), dispersion=disp, aniso=aniso)
    kx, ky = 2 * np.pi * mode[0] / N, 2 * np.pi * mode[1] / N
    y, x = np.mgrid[0:N, 0:N]
    E = np.zeros((N, N, 3))
    E[..., 2] = np.cos(kx * x + ky * y)
    g = O.init_state(m, E=E)
    pole = O.pole_state(m)
    basis = np.exp(-1j * (kx * x + ky * y))
    norm = N * N / (1 if mode == (0, 0) else 2)
    amp = []
    for _ in range(T):
        Ef, _ = O.fields(m, g, pole)
        amp.append(np.real((Ef[..., 2] * basis).sum()) / norm)
        O.run(m, g, 1, pole=pole)
    return np.array(amp), 0.5 / w_eps, np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2


def _charpoly(c2, q, wp2, wr2, gamma):
    """Ascending coefficients of zeta^2 [A (Q + wp^2) + 4 c^2 q Q] (see the module docstring)."""
    zA = np.array([1.0, -2.0, 1.0])  # zeta A
    zQ = zA + 0.5 * gamma * np.array([-1.0, 0.0, 1.0]) + wr2 * np.array([0.0, 1.0, 0.0])  # zeta Q
    p = Pn.polymul(zA, Pn.polyadd(zQ, wp2 * np.array([0.0, 1.0])))
    return Pn.polyadd(p, 4 * c2 * q * Pn.polymul(np.array([0.0, 1.0]), zQ))


@pytest.mark.parametrize("w_eps,mode,wp2", [(1.6, (2, 5), 0.2), (4.0, (1, 11), 0.5), (1.0, (3, 0), 0.05),
                                            (2.5, (7, 7), 1.0), (1.6, (0, 0), 0.3)])
def test_drude_plane_waves_follow_the_lattice_plasma_dispersion(w_eps, mode, wp2):
    amp, c2, q = _amplitudes(w_eps, mode, dict(wp2=wp2))
    om = 2 * np.arcsin(np.sqrt(c2 * q + wp2 / 4))
    t = np.arange(amp.size)
    b = (amp[1] - amp[0] * np.cos(om)) / np.sin(om)
    np.testing.assert_allclose(amp, amp[0] * np.cos(om * t) + b * np.sin(om * t), rtol=0, atol=1e-12)


@pytest.mark.parametrize("w_eps,mode,wp2,wr2,gamma", [(1.6, (2, 5), 0.2, 0.1, 0.0), (1.6, (2, 5), 0.2, 0.1, 0.2),
                                                      (1.0, (3, 0), 0.3, 0.0, 0.1), (4.0, (1, 11), 0.5, 0.7, 0.05),
                                                      (2.0, (0, 0), 0.4, 0.3, 0.3)])
def test_lorentz_pole_with_damping_follows_the_discrete_permittivity(w_eps, mode, wp2, wr2, gamma):
    amp, c2, q = _amplitudes(w_eps, mode, dict(wp2=wp2, wr2=wr2, gamma=gamma))
    p = _charpoly(c2, q, wp2, wr2, gamma)
    res = np.array([np.dot(p, amp[t:t + p.size]) for t in range(amp.size - p.size + 1)])
    assert np.abs(res).max() < 1e-13
    assert np.abs(Pn.polyroots(p)).max() <= 1 + 1e-6  # no growing mode (double roots at zeta = 1 when k = 0)
    if gamma > 0:
        assert np.abs(amp[-8:]).max() < np.abs(amp[:8]).max()


def test_continuum_limit_is_omega_squared_equals_wp_squared_plus_c_squared_k_squared():
    """The lattice relation tends to omega^2 = wp^2 + c^2 k^2 at second order as k and wp shrink together."""
    c2 = 0.3
    errs = []
    for h in (0.2, 0.1, 0.05):
        k, wp = 2.0 * h, 1.5 * h
        om = 2 * np.arcsin(np.sqrt(c2 * np.sin(k / 2) ** 2 + wp ** 2 / 4))
        errs.append(abs(om / np.sqrt(wp ** 2 + c2 * k ** 2) - 1))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_no_pole_is_the_plain_scheme_and_a_uniform_field_rings_at_the_plasma_frequency():
    rng = np.random.default_rng(3)
    eps = 1.5 + rng.random((12, 14))
    E = np.zeros((12, 14, 3))
    B = np.zeros_like(E)
    E[..., 2] = rng.standard_normal((12, 14))
    B[..., :2] = rng.standard_normal((12, 14, 2))
    m0, m1 = O.medium(2, eps), O.medium(2, eps, dispersion=dict(wp2=0.0))
    g0, g1 = O.init_state(m0, E, B), O.init_state(m1, E, B)
    pole = O.pole_state(m1)
    O.run(m0, g0, 30)
    O.run(m1, g1, 30, pole=pole)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-13)
    # uniform E_z in a lossless Drude medium: D stays constant, E = D - P rings at 2 sin(omega/2) = wp
    wp2 = 0.3
    m = O.medium(2, np.full((4, 4), 2.0), dispersion=dict(wp2=wp2))
    Eu = np.zeros((4, 4, 3))
    Eu[..., 2] = 1.0
    g = O.init_state(m, Eu)
    pole = O.pole_state(m)
    ez = []
    for _ in range(50):
        ez.append(O.fields(m, g, pole)[0][0, 0, 2])
        O.run(m, g, 1, pole=pole)
    om = 2 * np.arcsin(np.sqrt(wp2) / 2)
    t = np.arange(50)
    # E(t) = cos(omega (t + 1/2)) / cos(omega / 2) for E(0) = 1 and J(-1/2) = 0 (leapfrog start)
    np.testing.assert_allclose(ez, np.cos(om * (t + 0.5)) / np.cos(om / 2), rtol=0, atol=1e-12)
    D = O.fields(m, g)[0][..., 2]  # the lattice's moment: D / eps_inf
    np.testing.assert_allclose(D, 1.0, rtol=0, atol=1e-12)


def test_stability_bound():
    """wp^2 + wr^2 <= 4 w0 keeps every Fourier mode bounded (checked on the checkerboard mode, the worst case);
    beyond it that mode grows."""
    for w_eps, wp2, grows in ((1.25, 0.8, False), (1.25, 0.79, False), (1.25, 0.9, True)):
        c2 = 0.5 / w_eps  # w0 = 1 - 2 c2 = 0.2: bound wp2 <= 0.8
        q = 2.0
        p = _charpoly(c2, q, wp2, 0.0, 0.0)
        assert (np.abs(Pn.polyroots(p)).max() > 1 + 1e-6) == grows


@pytest.mark.parametrize("aniso,mode,disp", [((2.0, 1.0), (2, 5), dict(wp2=0.2)), ((3.0, 1.5), (0, 4), dict(wp2=0.5)),
                                             ((1.2, 2.5), (3, 1), dict(wp2=0.3, wr2=0.2, gamma=0.1)),
                                             ((3.0, 1.5), (5, 2), dict(wp2=0.1, wr2=0.05))])
def test_pole_in_an_anisotropic_medium_follows_the_per_axis_discrete_permittivity(aniso, mode, disp):
    """The pole and the anisotropic tensor together.  E = D/eps_inf - P enters the second moment per axis, so
    with u = D/eps_inf the lattice gives A u = -L (u - P) and the pole A P = wp^2 (u - P) (lossless Drude),
    L = 4 (c_x^2 sin^2(kx/2) + c_y^2 sin^2(ky/2)), c_x^2 = c^2/(eps mu_yy), c_y^2 = c^2/(eps mu_xx); hence
    4 sin^2(omega/2) = L + wp^2, and with wr, gamma the same recurrence as the isotropic pole with 4 c^2 q -> L."""
    w_eps = 1.6
    amp, _, _ = _amplitudes(w_eps, mode, disp, aniso=aniso)
    kx, ky = 2 * np.pi * mode[0] / N, 2 * np.pi * mode[1] / N
    cq = 0.5 / (w_eps * aniso[1]) * np.sin(kx / 2) ** 2 + 0.5 / (w_eps * aniso[0]) * np.sin(ky / 2) ** 2
    if set(disp) == {"wp2"}:
        om = 2 * np.arcsin(np.sqrt(cq + disp["wp2"] / 4))
        t = np.arange(amp.size)
        b = (amp[1] - amp[0] * np.cos(om)) / np.sin(om)
        np.testing.assert_allclose(amp, amp[0] * np.cos(om * t) + b * np.sin(om * t), rtol=0, atol=1e-12)
    p = _charpoly(cq, 1.0, disp["wp2"], disp.get("wr2", 0.0), disp.get("gamma", 0.0))
    res = np.array([np.dot(p, amp[t:t + p.size]) for t in range(amp.size - p.size + 1)])
    assert np.abs(res).max() < 1e-13
    # a plausible mistake, the isotropic c^2 (mean of the axes) in place of the per-axis split, fails the recurrence
    cbar = 0.25 / w_eps * (1 / aniso[0] + 1 / aniso[1]) * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2)
    if abs(cbar - cq) > 1e-3:
        pw = _charpoly(cbar, 1.0, disp["wp2"], disp.get("wr2", 0.0), disp.get("gamma", 0.0))
        assert np.abs([np.dot(pw, amp[t:t + pw.size]) for t in range(amp.size - pw.size + 1)]).max() > 1e-6
