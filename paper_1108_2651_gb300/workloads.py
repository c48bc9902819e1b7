"""Seeded synthetic inputs for the lattice-Boltzmann Maxwell solver.

This module only draws inputs: media (relative permittivity eps_r and
permeability mu_r), initial fields, source time series and receiver positions.
It holds none of the scheme's arithmetic, so that the GPU library and the FP64
oracle can both be fed from it.  Every array is numpy; grids are indexed
[y, x] in 2D and [z, y, x] in 3D (flat index x + nx*(y + ny*z)).

The paper's own heterogeneous medium is only shown in a figure (Sec.
"Heterogeneous media"), so the heterogeneous media here are seeded smoothed
random fields with the paper's kind of contrast (refractive index varying by
a factor of up to 3).
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# Reference (vacuum) wave speed squared in lattice units: the largest speed the
# lattice can carry with a non-negative rest weight.  2D: 1/2, 3D: 1/6.
C_REF2 = {2: 0.5, 3: 1.0 / 6.0}


def smoothed_unit_field(shape, sigma, seed):
    """u ~ U[0,1) from PCG64(seed), periodic Gaussian smoothing (std sigma cells) by FFT, min-max to [0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(shape)
    k2 = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[ax] = n
        k2 = k2 + (k.reshape(sh)) ** 2
    s = np.real(np.fft.ifftn(np.fft.fftn(u) * np.exp(-2.0 * np.pi ** 2 * sigma ** 2 * k2)))
    s = (s - s.min()) / (s.max() - s.min())
    return s


def refractive_index(shape, sigma, seed, contrast=2.0):
    """n = 1 + contrast * s, s a smoothed unit field (n in [1, 1 + contrast])."""
    return 1.0 + contrast * smoothed_unit_field(shape, sigma, seed)


def ricker(nt, f, t0=None, amp=1.0):
    """Ricker wavelet r(t) = amp (1 - 2a) exp(-a), a = (pi f (t - t0))^2, t = 0..nt-1, t0 = 1.5/f."""
    if t0 is None:
        t0 = 1.5 / f
    t = np.arange(nt, dtype=np.float64)
    a = (np.pi * f * (t - t0)) ** 2
    return amp * (1.0 - 2.0 * a) * np.exp(-a)


def gaussian_pulse(shape, center, sigma):
    """exp(-|x - center|^2 / (2 sigma^2)) on the grid (axes as the grid's)."""
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    r2 = sum((g - c) ** 2 for g, c in zip(grids, center))
    return np.exp(-r2 / (2.0 * sigma ** 2))


def flat_index(shape, pos):
    """Flat C-order index of grid position pos (same axis order as shape)."""
    return int(np.ravel_multi_index(tuple(int(p) % n for p, n in zip(pos, shape)), shape))


@dataclass
class Problem:
    """One simulation: medium, initial fields, sources, receivers, number of steps."""

    name: str
    D: int
    shape: tuple
    eps_r: np.ndarray
    mu_r: Optional[np.ndarray]
    nsteps: int
    E0: Optional[np.ndarray] = None  # grid + (3,)
    B0: Optional[np.ndarray] = None
    src_site: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    src_comp: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    src_amp: np.ndarray = field(default_factory=lambda: np.zeros((0, 1)))
    rec_site: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    rec_comp: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    bc: tuple = (0, 0, 0)  # boundary per axis x, y, z: 0 periodic, 1 PEC wall, 2 PMC wall (2D)
    layer: int = 0  # absorbing layer inside the walls (sites)
    gamma_max: float = 0.0  # its damping at the wall-adjacent site
    wp2: Optional[np.ndarray] = None  # dispersive pole per site (grid): plasma frequency squared, or None
    wr2: Optional[np.ndarray] = None  # its resonance frequency squared
    gamma: Optional[np.ndarray] = None  # its damping rate
    aniso: Optional[tuple] = None  # (mu_xx, mu_yy): a uniform in-plane permeability tensor (2D; mu_r must be None)

    @property
    def c_ref2(self):
        return C_REF2[self.D]

    @property
    def nsite(self):
        return int(np.prod(self.shape))

    def sources(self):
        if self.src_site.size == 0:
            return None
        return dict(site=self.src_site, comp=self.src_comp, amp=self.src_amp)

    def receivers(self):
        if self.rec_site.size == 0:
            return None
        return dict(site=self.rec_site, comp=self.rec_comp)


def homogeneous_pulse(n=128, sigma=6.0, nsteps=500):
    """2D homogeneous medium (n = mu = 1), periodic n x n grid, Gaussian pulse (std sigma cells) in E_z, B = 0."""
    shape = (n, n)
    E0 = np.zeros(shape + (3,))
    E0[..., 2] = gaussian_pulse(shape, (n // 2, n // 2), sigma)
    return Problem("homogeneous_pulse", 2, shape, np.ones(shape), None, nsteps, E0=E0)


def point_source_problem(D, shape, n_index, nsteps, src_pos, nrec, rec_positions, ppw=20.0, comp=2, name="point"):
    """A medium n(x), eps_r = n^2, mu = 1; Ricker j_comp at src_pos, peak at ppw cells per local wavelength."""
    eps = n_index ** 2
    n_src = n_index[tuple(src_pos)]
    f = np.sqrt(C_REF2[D]) / n_src / ppw
    p = Problem(name, D, shape, eps, None, nsteps)
    p.src_site = np.array([flat_index(shape, src_pos)], np.int64)
    p.src_comp = np.array([comp], np.int32)
    p.src_amp = ricker(nsteps, f)[None, :]
    p.rec_site = np.array([flat_index(shape, r) for r in rec_positions], np.int64)
    p.rec_comp = np.full(len(rec_positions), 2 if D == 2 else comp, np.int32)
    return p


def circle_receivers(center, radius, count):
    """count positions at angles 2 pi k / count on a circle, rounded to cells; returned as (y, x)."""
    out = []
    for k in range(count):
        th = 2.0 * np.pi * k / count
        out.append((int(round(center[0] + radius * np.sin(th))), int(round(center[1] + radius * np.cos(th)))))
    return out


def heterogeneous_2d(n=1024, seed=1, nsteps=5000, sigma=20.0, nrec=64, rec_radius=None, name=None):
    """2D heterogeneous medium n = 1 + 2 s (s smoothed, sigma cells), Ricker j_z at the centre, receivers on a circle."""
    shape = (n, n)
    nidx = refractive_index(shape, sigma, seed)
    c = (n // 2, n // 2)
    if rec_radius is None:
        rec_radius = min(256, n // 4)
    recs = circle_receivers(c, rec_radius, nrec)
    return point_source_problem(2, shape, nidx, nsteps, c, nrec, recs, name=name or f"het2d_{n}")


def heterogeneous_2d_mu(n=1024, seed=1, nsteps=5000, sigma=20.0, nrec=64, rec_radius=None, mu_contrast=1.0,
                        mu_seed=None, name=None):
    """heterogeneous_2d with the same refractive index n = 1 + 2 s but a heterogeneous permeability:
    mu_r = 1 + mu_contrast * s2 (s2 a second smoothed unit field, seed mu_seed, default seed + 7919) and
    eps_r = n^2 / mu_r, so the wave speed c/n is unchanged while the impedance varies and the B x grad ln mu
    source term (Eq. 3) acts everywhere."""
    p = heterogeneous_2d(n, seed, nsteps, sigma, nrec, rec_radius, name=name or f"het2d_mu_{n}")
    n2 = p.eps_r
    mu = np.float32(1.0 + mu_contrast * smoothed_unit_field(p.shape, sigma, seed + 7919 if mu_seed is None else mu_seed))
    eps = np.float32(n2 / mu.astype(np.float64))
    # the media are given to the solver in FP32: where rounding made eps_r mu_r < n^2 (which at n = 1 would put the
    # medium above the reference speed), step eps_r up by one unit in the last place
    low = eps.astype(np.float64) * mu.astype(np.float64) < n2
    eps[low] = np.nextafter(eps[low], np.float32(np.inf))
    p.eps_r = eps.astype(np.float64)
    p.mu_r = mu.astype(np.float64)
    return p


def heterogeneous_2d_walls(n=1024, seed=1, nsteps=5000, sigma=20.0, nrec=64, rec_radius=None, bc=(1, 1, 0),
                           layer=32, gamma_max=0.2, name=None):
    """heterogeneous_2d in a box: walls on x and y (default PEC) with an absorbing layer of `layer` sites inside
    them (damping gamma_max at the wall-adjacent site), so the waves leave the domain instead of wrapping."""
    p = heterogeneous_2d(n, seed, nsteps, sigma, nrec, rec_radius, name=name or f"het2d_walls_{n}")
    p.bc = tuple(bc) + (0,) * (3 - len(bc))
    p.layer = int(layer)
    p.gamma_max = float(gamma_max)
    return p


def heterogeneous_2d_drude(n=1024, seed=1, nsteps=5000, sigma=20.0, nrec=64, rec_radius=None, wp2=0.5, gamma=0.01,
                           name=None):
    """heterogeneous_2d with a lossy Drude cylinder (a plasmonic scatterer): inside the disk of radius n/8 centred
    n/4 from the source along x, eps_r (eps_infinity) is raised to at least 2.25 and the pole has wp^2 = wp2,
    damping gamma (wr = 0); zero elsewhere.  At eps_r >= 2.25 the rest weight is >= 0.55, so wp2 <= 2.2 keeps the
    pole within its stability bound wp^2 <= 4 w0."""
    p = heterogeneous_2d(n, seed, nsteps, sigma, nrec, rec_radius, name=name or f"het2d_drude_{n}")
    y, x = np.mgrid[0:n, 0:n]
    disk = (x - (n // 2 + n // 4)) ** 2 + (y - n // 2) ** 2 <= (n / 8) ** 2
    p.eps_r = np.where(disk, np.maximum(p.eps_r, 2.25), p.eps_r)
    p.wp2 = np.where(disk, wp2, 0.0)
    p.wr2 = np.zeros(p.shape)
    p.gamma = np.where(disk, gamma, 0.0)
    return p


def heterogeneous_2d_aniso(n=1024, seed=1, nsteps=5000, sigma=20.0, nrec=64, rec_radius=None, mu_xx=2.0, mu_yy=1.0,
                           name=None):
    """heterogeneous_2d in a uniaxial medium: the same eps_r with a uniform permeability tensor diag(mu_xx, mu_yy),
    so waves move sqrt(mu_xx / mu_yy) times faster along x than along y.  The lattice needs
    c_ref^2 (1/mu_xx + 1/mu_yy) <= eps_r (rest weight >= 0): eps_r is raised to at least that."""
    p = heterogeneous_2d(n, seed, nsteps, sigma, nrec, rec_radius, name=name or f"het2d_aniso_{n}")
    need = C_REF2[2] * (1.0 / mu_xx + 1.0 / mu_yy)
    p.eps_r = np.maximum(p.eps_r, need)
    p.aniso = (float(mu_xx), float(mu_yy))
    return p


def batch_sizes(count=256, seed=3, lo=64, hi=512):
    """Square grid sizes N_b = round(exp(U(ln lo, ln hi))) from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(count)]


def batch_2d(count=256, nsteps=2000, size_seed=3, sizes=None):
    """Independent 2D heterogeneous media of uneven sizes (seeds 1000 + b), source at each centre, 8 receivers each."""
    if sizes is None:
        sizes = batch_sizes(count, size_seed)
    probs = []
    for b, N in enumerate(sizes):
        sigma = min(20.0, N / 8.0)
        probs.append(heterogeneous_2d(N, seed=1000 + b, nsteps=nsteps, sigma=sigma, nrec=8,
                                      rec_radius=max(1, N // 4), name=f"batch{b}_{N}"))
    return probs


def heterogeneous_3d(n=192, seed=4, nsteps=1000, sigma=12.0, plane_dz=48, rec_grid=(8, 16), ppw=20.0):
    """3D medium n = 1 + 2 s (s smoothed, sigma cells), Ricker j_z at the centre (a point current element),
    receivers on a rec_grid (rows x cols) lattice on the plane z = n/2 + plane_dz, recording E_z."""
    shape = (n, n, n)
    nidx = refractive_index(shape, sigma, seed)
    c = (n // 2, n // 2, n // 2)
    zr = min(n - 1, n // 2 + plane_dz)
    ry, rx = rec_grid
    ys = np.linspace(n // 4, 3 * n // 4, ry).round().astype(int)
    xs = np.linspace(n // 8, 7 * n // 8, rx).round().astype(int)
    recs = [(zr, y, x) for y in ys for x in xs]
    return point_source_problem(3, shape, nidx, nsteps, c, len(recs), recs, ppw=ppw, comp=2, name=f"het3d_{n}")


def smooth_perturbation(shape, seed, sigma, amp=1.0):
    """A mean-zero smoothed random field scaled to max |.| = amp (for gradient checks)."""
    s = smoothed_unit_field(shape, sigma, seed)
    s = s - s.mean()
    return amp * s / np.abs(s).max()


def random_fields(shape, seed, scale=1.0):
    """Random E and B (grid + (3,)) from PCG64(seed), for moment and parity checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape + (3,)), scale * rng.standard_normal(shape + (3,))


def random_medium(shape, seed, lo=1.0, hi=3.0, mu=False):
    """Unsmoothed random eps_r = n^2 with n ~ U[lo, hi] (and mu_r ~ U[1, 2] if mu), for parity on tiny grids."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.uniform(lo, hi, shape)
    mu_r = rng.uniform(1.0, 2.0, shape) if mu else None
    return n ** 2, mu_r
