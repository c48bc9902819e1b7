"""Pins of the oracle's heterogeneous-permeability source term (CPU).

Eq. 3 of the paper collects a spatially varying permeability into the source
S = c^2 (B x grad ln mu0) of the E equation.  The other pins run with mu = 1,
so this term is checked here against what the mathematics fixes without it:

* Fresnel reflection.  A smooth step in mu with eps*mu held fixed keeps the
  wave speed constant; only the impedance Z = sqrt(mu/eps) changes, so the
  whole reflection comes from the B x grad ln mu term.  The integral of E over
  the reflected (transmitted) pulse is the zero-frequency content of the pulse
  times r (t c2/c1), and at zero frequency any finite transition is a sharp
  interface: r = (Z2 - Z1)/(Z2 + Z1), t = 2 Z2/(Z2 + Z1) exactly in the
  continuum.  A step with matched impedance but a 2:1 speed contrast must not
  reflect at all.  2D TM along x, and 3D along every axis in both
  polarisations (each sign and index of the cross product).
* Pseudo-spectral Maxwell in the H form (eps dE/dt = curl(B/mu), no gradient of
  ln mu formed), the paper's own kind of validation: the LB - PS difference
  with smooth heterogeneous eps and mu falls at second order.

Negative controls plant the plausible mistakes in the oracle's input on the
CPU (the gradient of ln mu negated: the cross product reversed; or zeroed: the
term dropped) and check that each pin then fails.
"""
import numpy as np
import pytest

import crosscheck as X
import oracle as O


def _tanh_box(n, w):
    """0 on the first half of a periodic line of n sites, 1 on the second, smooth steps of width w at n/2 and n."""
    x = np.arange(n, dtype=np.float64)
    return 0.25 * (np.tanh((x - n / 2) / w) + 1) * (1 - np.tanh((x - n) / w))


def _line_pulse(D, axis, n, eps, mu, pol=0, sigma=30.0, mistake=None):
    """A right-moving Gaussian pulse on a periodic line of n sites along `axis` (other axes 1 site), started in
    the first half at n/4 and stepped until the reflected and transmitted pulses are clear of the interface at
    n/2.  In 2D the fields are E_z, B_y (axis x); in 3D E along p = axis+1 and B along q = axis+2 (pol 0), or E
    along q and B along p (pol 1).  Returns (integral of E over the first half, over the second half), both
    divided by the integral of the incident E."""
    shape = [1] * D
    shape[D - 1 - axis] = n  # grids are [y, x] / [z, y, x]
    m = O.medium(D, eps.reshape(shape), mu.reshape(shape))
    if mistake == "reversed":
        m.dlnmu = -m.dlnmu
    elif mistake == "dropped":
        m.dlnmu = np.zeros_like(m.dlnmu)
    c1 = np.sqrt(m.ceff2.ravel()[0])
    x = np.arange(n, dtype=np.float64)
    f = np.exp(-(x - n / 4) ** 2 / (2 * sigma ** 2))
    E = np.zeros(tuple(shape) + (3,))
    B = np.zeros(tuple(shape) + (3,))
    if D == 2:
        ce, cb, sb = 2, 1, -1.0  # dB_y/dt = dE_z/dx: B_y = -E_z/c for E_z = f(x - ct)
    else:
        p, q = (axis + 1) % 3, (axis + 2) % 3
        # dB/dt = -curl E: eps_{q,axis,p} = +1, eps_{p,axis,q} = -1
        ce, cb, sb = (p, q, 1.0) if pol == 0 else (q, p, -1.0)
    E[..., ce] = f.reshape(shape)
    B[..., cb] = sb * f.reshape(shape) / c1
    g = O.init_state(m, E=E, B=B)
    steps = int(round(3 * n / 8 / c1))
    steps += steps % 2  # even steps: the period-2 mode of tau = dt/2 offsets B at odd ones
    O.run(m, g, steps)
    Ef, _ = O.fields(m, g)
    e = Ef[..., ce].ravel()
    return e[: n // 2].sum() / f.sum(), e[n // 2:].sum() / f.sum()


def _speed_ratio(eps1, mu1, eps2, mu2):
    return np.sqrt((eps1 * mu1) / (eps2 * mu2))


# (eps, mu) of the first and second half: impedance steps at constant speed (up and down), and a matched
# impedance with a 2:1 speed contrast
CASES = [((2.0, 1.0), (0.5, 4.0)), ((2.0, 1.0), (8.0, 0.25)), ((2.0, 1.0), (4.0, 2.0))]


@pytest.mark.parametrize("case", CASES, ids=["Z_up_4x", "Z_down_4x", "Z_matched_slow"])
def test_mu_step_reflects_as_fresnel_2d(case):
    """2D TM pulse along x across a smooth (width 8 sites) step of mu: the reflected and transmitted integrals of
    E_z follow r = (Z2 - Z1)/(Z2 + Z1) and t c2/c1 to 1e-3, with r = 0 for a matched impedance."""
    (e1, m1), (e2, m2) = case
    n = 2048
    s = _tanh_box(n, 8.0)
    eps = np.exp(np.log(e1) + s * np.log(e2 / e1))
    mu = np.exp(np.log(m1) + s * np.log(m2 / m1))
    refl, tran = _line_pulse(2, 0, n, eps, mu)
    r, t = X.fresnel(e1, m1, e2, m2)
    assert abs(refl - r) < 1e-3, (refl, r)
    assert abs(tran - t * _speed_ratio(e1, m1, e2, m2)) < 1e-3, (tran, t)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("pol", [0, 1])
def test_mu_step_reflects_as_fresnel_3d(axis, pol):
    """3D (reading R2's c_eff^2 = c_L^2 / 2): a pulse along each axis in both transverse polarisations across a
    constant-speed impedance step (Z2/Z1 = 4) and a matched one with a 2:1 speed contrast."""
    n = 1024
    s = _tanh_box(n, 8.0)
    for (e1, m1), (e2, m2) in (CASES[0], CASES[2]):
        eps = np.exp(np.log(e1) + s * np.log(e2 / e1))
        mu = np.exp(np.log(m1) + s * np.log(m2 / m1))
        refl, tran = _line_pulse(3, axis, n, eps, mu, pol=pol)
        r, t = X.fresnel(e1, m1, e2, m2)
        assert abs(refl - r) < 1e-3, (axis, pol, refl, r)
        assert abs(tran - t * _speed_ratio(e1, m1, e2, m2)) < 1e-3, (axis, pol, tran, t)


@pytest.mark.parametrize("D", [2, 3])
def test_fresnel_pin_catches_a_reversed_or_dropped_mu_term(D):
    """Negative control: with the gradient of ln mu negated (B x grad ln mu replaced by grad ln mu x B) the
    constant-speed step reflects -0.6 instead of +0.6; with the term dropped it does not reflect at all."""
    n = 2048 if D == 2 else 1024
    s = _tanh_box(n, 8.0)
    (e1, m1), (e2, m2) = CASES[0]
    eps = np.exp(np.log(e1) + s * np.log(e2 / e1))
    mu = np.exp(np.log(m1) + s * np.log(m2 / m1))
    r, _ = X.fresnel(e1, m1, e2, m2)
    rev, _ = _line_pulse(D, 0, n, eps, mu, mistake="reversed")
    drop, _ = _line_pulse(D, 0, n, eps, mu, mistake="dropped")
    assert abs(rev + r) < 1e-3 and abs(drop) < 1e-4, (rev, drop)
    assert abs(rev - r) > 1.0 and abs(drop - r) > 0.5


def _smooth_medium_2d(N):
    x = np.arange(N) / N
    X_, Y_ = np.meshgrid(x, x, indexing="xy")  # [y, x]
    n_idx = 1.0 + 0.5 * (1 + np.sin(2 * np.pi * X_) * np.cos(2 * np.pi * Y_))
    mu = 1.0 + 0.6 * (1 + np.cos(2 * np.pi * X_ + 0.3) * np.sin(2 * np.pi * Y_))
    # divergence-free initial B of the paper's heterogeneous test (Sec. "Heterogeneous media")
    f = 10.0 * np.exp(-((X_ - 0.5) ** 2 + (Y_ - 0.35) ** 2) / (2 * 0.04 ** 2))
    return n_idx ** 2 / mu, mu, (Y_ - 0.35) * f, -(X_ - 0.5) * f


def _lb_vs_ps_2d(N, ps, mistake=None):
    eps, mu, Bx, By = _smooth_medium_2d(N)
    m = O.medium(2, eps, mu)
    if mistake == "reversed":
        m.dlnmu = -m.dlnmu
    elif mistake == "dropped":
        m.dlnmu = np.zeros_like(m.dlnmu)
    B = np.zeros((N, N, 3))
    B[..., 0], B[..., 1] = Bx, By
    g = O.init_state(m, B=B)
    O.run(m, g, int(round(0.25 * N)))
    Ef, Bf = O.fields(m, g)
    e, bx, by = ps
    num = np.sqrt(((Ef[..., 2] - e) ** 2).sum() + ((Bf[..., 0] - bx) ** 2).sum() + ((Bf[..., 1] - by) ** 2).sum())
    return num / np.sqrt((e ** 2).sum() + (bx ** 2).sum() + (by ** 2).sum())


def test_lb_with_mu_converges_to_h_form_pseudo_spectral_2d():
    """Smooth heterogeneous eps and mu (mu from 1 to 2.2, refractive index 1 to 2), the paper's divergence-free
    initial B: the LB - PS(H form) difference at t = 1/4 falls about 4x per grid doubling (second order, 0.5 %
    at 256^2), while the same runs with the mu term reversed or dropped stall (ratio < 1.5, error > 8 %).  mu
    alone moves the solution by 8 % of its norm (PS with mu = 1 at the same speed), so the pin is not idle."""
    errs, rev, drop = [], [], []
    for N in (64, 128, 256):
        eps, mu, Bx, By = _smooth_medium_2d(N)
        steps = int(round(0.25 * N))
        ps = X.maxwell_ps_2d_h(0.5 / eps, mu, np.zeros((N, N)), Bx, By, steps / N, 0.25 / N)
        errs.append(_lb_vs_ps_2d(N, ps))
        if N < 256:
            rev.append(_lb_vs_ps_2d(N, ps, "reversed"))
            drop.append(_lb_vs_ps_2d(N, ps, "dropped"))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5 and errs[2] < 0.01, errs
    assert rev[0] / rev[1] < 1.5 and min(rev) > 0.08, rev
    assert drop[0] / drop[1] < 1.5 and min(drop) > 0.08, drop


def test_lb_with_mu_converges_to_h_form_pseudo_spectral_3d():
    """3D with heterogeneous eps and mu (reading R2): LB - PS(H form) falls at about second order; with the
    mu term reversed the difference does not fall."""
    errs, rev = [], []
    for N in (16, 32):
        z, y, x = np.meshgrid(*(np.arange(N) / N,) * 3, indexing="ij")
        n_idx = 1.0 + 0.3 * (1 + np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.cos(2 * np.pi * z))
        mu = 1.0 + 0.5 * (1 + np.cos(2 * np.pi * y + 0.4) * np.sin(2 * np.pi * z) * np.cos(2 * np.pi * x))
        eps = n_idx ** 2 / mu
        psi = np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / (2 * 0.12 ** 2))
        kz, ky, kx = np.meshgrid(*(2 * np.pi * np.fft.fftfreq(N, 1 / N),) * 3, indexing="ij")
        dpsi = lambda k: np.real(np.fft.ifftn(1j * k * np.fft.fftn(psi)))
        Bv = np.array([dpsi(ky), dpsi(kz) - dpsi(kx), -dpsi(ky)])  # curl of (psi, 0, psi): divergence-free
        steps = int(round(0.25 * N))
        m = O.medium(3, eps, mu)
        e, b = X.maxwell_ps_3d_h(m.ceff2 * mu, mu, np.zeros_like(Bv), Bv, steps / N, 0.25 / N)
        den = np.sqrt((e ** 2).sum() + (b ** 2).sum())
        for out, flip in ((errs, False), (rev, True)):
            mm = O.medium(3, eps, mu)
            if flip:
                mm.dlnmu = -mm.dlnmu
            g = O.init_state(mm, B=np.moveaxis(Bv, 0, -1))
            O.run(mm, g, steps)
            Ef, Bf = O.fields(mm, g)
            num = np.sqrt(((np.moveaxis(Ef, -1, 0) - e) ** 2).sum() + ((np.moveaxis(Bf, -1, 0) - b) ** 2).sum())
            out.append(num / den)
    assert errs[0] / errs[1] > 3.0, errs
    assert rev[0] / rev[1] < 2.0 and rev[1] > 3 * errs[1], (rev, errs)
