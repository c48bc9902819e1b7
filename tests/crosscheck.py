"""Independent solvers and closed forms that pin the FP64 oracle.

Nothing here calls the oracle or the GPU library: these are separate
statements of what the paper fixes, written from the mathematics.

* leapfrog_2d: the exact finite-difference form of the 2D scheme.  At
  tau = 1/2 the lattice update of the paper's Eqs. 17-18 on the D2Q5 lattice
  eliminates to a three-level scheme in E_z and a two-level one in B (the
  paper's closing remark that the method is a special finite-difference
  method, made concrete).  With Lap5 the 5-point Laplacian, c2 = c_L^2(x) and
  S = S_z(x, t) of Eq. 3:
      E^{t+1} - 2E^t + E^{t-1} = c2 Lap5 E^t + S^t + (c2/2) Lap5 S^t - S^{t-1}
      B_y^{t+1} - B_y^{t-1} = D_x E^t + (1/2) D_x S^t
      B_x^{t+1} - B_x^{t-1} = -D_y E^t - (1/2) D_y S^t
  with D_x u = u(x+1) - u(x-1).  Derivation: substitute the collision into the
  streaming twice and use that the weights of moving particles over c_L^2
  equal 1/2 and sum_i w_i = 1.
* omega_2d: its plane-wave dispersion relation
      sin^2(omega/2) = c2 (sin^2(kx/2) + sin^2(ky/2)).
* maxwell_ps_2d / maxwell_ps_3d: pseudo-spectral Maxwell solvers with
  classical RK4 (the paper validates against a pseudo-spectral solver with an
  optimised Runge-Kutta scheme whose coefficients it does not give).
* maxwell_ps_2d_h / maxwell_ps_3d_h: the same in the H form for a medium with
  heterogeneous eps and mu, d_t B = -curl E, d_t E = (c_ref^2/eps_r) curl(B/mu_r).
  No gradient of ln mu appears: the permeability enters only through H = B/mu,
  differentiated spectrally, so these solvers pin the paper's Eq. 3 source
  c^2 (B x grad ln mu) without restating it.
* fresnel: normal-incidence reflection and transmission of E at an impedance
  step, Z = sqrt(mu/eps).
* spectral_divb_error: Eq. 19 with F = 1.
"""
import numpy as np


def lap5(u):
    """Periodic 5-point Laplacian on a [y, x] grid."""
    return np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1) - 4.0 * u


def dx_c(u):
    """u(x+1) - u(x-1) on a [y, x] grid (periodic)."""
    return np.roll(u, -1, 1) - np.roll(u, 1, 1)


def dy_c(u):
    """u(y+1) - u(y-1) on a [y, x] grid (periodic)."""
    return np.roll(u, -1, 0) - np.roll(u, 1, 0)


def leapfrog_2d(c2, E0, E1, Bx0, Bx1, By0, By1, S, nsteps):
    """Advance the exact FD form from levels 0 and 1 to level nsteps-1.

    S is a list/array of S_z^t for t = 0..nsteps-1.  Returns arrays E, Bx, By
    of shape (nsteps,) + grid.
    """
    E = [E0, E1]
    Bx = [Bx0, Bx1]
    By = [By0, By1]
    for t in range(1, nsteps - 1):
        E.append(2 * E[t] - E[t - 1] + c2 * lap5(E[t]) + S[t] + 0.5 * c2 * lap5(S[t]) - S[t - 1])
        By.append(By[t - 1] + dx_c(E[t]) + 0.5 * dx_c(S[t]))
        Bx.append(Bx[t - 1] - dy_c(E[t]) - 0.5 * dy_c(S[t]))
    return np.array(E), np.array(Bx), np.array(By)


def omega_2d(c2, kx, ky):
    """Angular frequency of the exact FD form for wavevector (kx, ky), 0 <= omega <= pi."""
    s = c2 * (np.sin(kx / 2) ** 2 + np.sin(ky / 2) ** 2)
    return 2.0 * np.arcsin(np.sqrt(s))


def _kgrid(shape, L):
    ks = [2.0 * np.pi * np.fft.fftfreq(n, d=L / n) for n in shape]
    return np.meshgrid(*ks, indexing="ij")


def _deriv(u, k):
    return np.real(np.fft.ifftn(1j * k * np.fft.fftn(u)))


def maxwell_ps_2d(c2, E, Bx, By, t_end, dt, S=None, L=1.0):
    """TM Maxwell on a periodic [y, x] grid of side L:
        dBx/dt = -dE/dy, dBy/dt = dE/dx, dE/dt = c2 (dBy/dx - dBx/dy) + S(t).
    Spectral derivatives, classical RK4 with step <= dt.  S: callable t -> grid or None."""
    ky, kx = _kgrid(E.shape, L)
    nst = int(np.ceil(t_end / dt - 1e-12))
    h = t_end / nst

    def rhs(t, y):
        e, bx, by = y
        de = c2 * (_deriv(by, kx) - _deriv(bx, ky))
        if S is not None:
            de = de + S(t)
        return np.array([de, -_deriv(e, ky), _deriv(e, kx)])

    y = np.array([E, Bx, By], dtype=np.float64)
    t = 0.0
    for _ in range(nst):
        k1 = rhs(t, y)
        k2 = rhs(t + h / 2, y + h / 2 * k1)
        k3 = rhs(t + h / 2, y + h / 2 * k2)
        k4 = rhs(t + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += h
    return y


def maxwell_ps_3d(c2, E, B, t_end, dt, L=1.0):
    """dB/dt = -curl E, dE/dt = c2 curl B on a periodic [z, y, x] grid; E, B of shape (3,) + grid
    (components x, y, z).  Spectral derivatives, classical RK4."""
    kz, ky, kx = _kgrid(E.shape[1:], L)
    K = (kx, ky, kz)
    nst = int(np.ceil(t_end / dt - 1e-12))
    h = t_end / nst

    def curl(v):
        d = [[_deriv(v[a], K[b]) for b in range(3)] for a in range(3)]  # d[a][b] = d_b v_a
        return np.array([d[2][1] - d[1][2], d[0][2] - d[2][0], d[1][0] - d[0][1]])

    def rhs(y):
        e, b = y[:3], y[3:]
        return np.concatenate([c2 * curl(b), -curl(e)])

    y = np.concatenate([E, B]).astype(np.float64)
    for _ in range(nst):
        k1 = rhs(y)
        k2 = rhs(y + h / 2 * k1)
        k3 = rhs(y + h / 2 * k2)
        k4 = rhs(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y[:3], y[3:]


def maxwell_ps_2d_h(ceps2, mu, E, Bx, By, t_end, dt, L=1.0):
    """TM Maxwell in the H form on a periodic [y, x] grid of side L, for eps and mu that vary in space:
        dBx/dt = -dE/dy, dBy/dt = dE/dx, dE/dt = ceps2 (d(By/mu)/dx - d(Bx/mu)/dy),
    ceps2 = c_ref^2 / eps_r (so that the local wave speed squared is ceps2 / mu).  This is the form
    eps dE/dt = curl H with H = B/mu; expanding curl(B/mu) gives the c^2 (B x grad ln mu) source of Eq. 3,
    which is never formed here.  Spectral derivatives, classical RK4 with step <= dt."""
    ky, kx = _kgrid(E.shape, L)
    nst = int(np.ceil(t_end / dt - 1e-12))
    h = t_end / nst

    def rhs(y):
        e, bx, by = y
        de = ceps2 * (_deriv(by / mu, kx) - _deriv(bx / mu, ky))
        return np.array([de, -_deriv(e, ky), _deriv(e, kx)])

    y = np.array([E, Bx, By], dtype=np.float64)
    for _ in range(nst):
        k1 = rhs(y)
        k2 = rhs(y + h / 2 * k1)
        k3 = rhs(y + h / 2 * k2)
        k4 = rhs(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def maxwell_ps_3d_h(ceps2, mu, E, B, t_end, dt, L=1.0):
    """dB/dt = -curl E, dE/dt = ceps2 curl(B/mu) on a periodic [z, y, x] grid (the H form in 3D); E, B of
    shape (3,) + grid.  Spectral derivatives, classical RK4."""
    kz, ky, kx = _kgrid(E.shape[1:], L)
    K = (kx, ky, kz)
    nst = int(np.ceil(t_end / dt - 1e-12))
    h = t_end / nst

    def curl(v):
        d = [[_deriv(v[a], K[b]) for b in range(3)] for a in range(3)]  # d[a][b] = d_b v_a
        return np.array([d[2][1] - d[1][2], d[0][2] - d[2][0], d[1][0] - d[0][1]])

    def rhs(y):
        e, b = y[:3], y[3:]
        return np.concatenate([ceps2 * curl(b / mu), -curl(e)])

    y = np.concatenate([E, B]).astype(np.float64)
    for _ in range(nst):
        k1 = rhs(y)
        k2 = rhs(y + h / 2 * k1)
        k3 = rhs(y + h / 2 * k2)
        k4 = rhs(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y[:3], y[3:]


def fresnel(eps1, mu1, eps2, mu2):
    """Reflection and transmission coefficients of E for a plane wave at normal incidence on the interface
    between two uniform media (continuity of tangential E and H = B/mu):
        r = (Z2 - Z1)/(Z2 + Z1), t = 1 + r = 2 Z2/(Z2 + Z1), Z = sqrt(mu/eps)."""
    z1, z2 = np.sqrt(mu1 / eps1), np.sqrt(mu2 / eps2)
    return (z2 - z1) / (z2 + z1), 2 * z2 / (z2 + z1)


def spectral_divb_error(Bx, By, L=1.0):
    """Eq. 19 with F = 1: sum_k |i k . B(k)| / sum_k |B(k)| on a [y, x] grid."""
    ky, kx = _kgrid(Bx.shape, L)
    bx, by = np.fft.fft2(Bx), np.fft.fft2(By)
    num = np.abs(1j * (kx * bx + ky * by)).sum()
    den = np.sqrt(np.abs(bx) ** 2 + np.abs(by) ** 2).sum()
    return num / den
