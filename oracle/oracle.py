"""ctypes wrapper of the FP64 C oracle (lbem_oracle.c).

TEST INFRASTRUCTURE ONLY.  Grids are numpy arrays indexed [y, x] in 2D and
[z, y, x] in 3D, so that the flat C-order index is s = x + nx*(y + ny*z), the
oracle's site index.  The state g has shape grid + (Q, D, D): the full tensor
g_{i,alpha,beta} of the paper's Sec. "Lattice BGK formulation".
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build_oracle import build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        I, D_ = C.c_int, C.c_double
        lib.or_medium.restype = C.c_long
        lib.or_medium.argtypes = [I, I, I, I, D_, dp, C.c_void_p, ip, D_, dp, dp, dp, dp, dp]
        lib.or_init.restype = None
        lib.or_init.argtypes = [I, I, I, I, dp, dp, C.c_void_p, C.c_void_p, dp, D_]
        lib.or_fields.restype = None
        lib.or_fields.argtypes = [I, I, I, I, dp, dp, dp, dp, D_]
        lib.or_run.restype = I
        vp = C.c_void_p
        lib.or_run.argtypes = [I, I, I, I, dp, dp, dp, dp, dp, dp, I, I, I, lp, ip, dp, I, I, lp, ip, dp, ip, I, D_,
                               vp, vp, vp, vp, vp, D_]
        lib.or_diagnostics.restype = None
        lib.or_diagnostics.argtypes = [I, I, I, I, dp, dp, dp, dp, dp, D_]
        lib.or_adjoint.restype = D_
        lib.or_adjoint.argtypes = [I, I, I, I, dp, dp, dp, dp, dp, I, I, I, lp, ip, dp, I, I, lp, ip, dp, dp]
        lib.or_threads.restype = I
        lib.or_threads.argtypes = []
        lib.or_set_threads.restype = I
        lib.or_set_threads.argtypes = [I]
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return _load().or_threads()


def set_threads(n: int) -> int:
    """Set the oracle's OpenMP thread count (timing on fewer cores); returns the count in effect."""
    return _load().or_set_threads(int(n))


_lib32 = None


def time_fp32(eps_r, nsteps, src_site, src_amp, threads_=0):
    """Seconds for nsteps steps of the FP32 build of the same oracle source (2D isotropic periodic medium eps_r,
    point current j_z at flat index src_site with amplitudes src_amp[t]), from a zero state: a like-for-like CPU
    timing figure only; its results are never used as a reference."""
    import time

    global _lib32
    if _lib32 is None:
        lib = C.CDLL(build(fp32=True))
        fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        I, F, vp = C.c_int, C.c_float, C.c_void_p
        lib.or_medium.restype = C.c_long
        lib.or_medium.argtypes = [I, I, I, I, F, fp, vp, ip, F, fp, fp, fp, fp, fp]
        lib.or_run.restype = I
        lib.or_run.argtypes = [I, I, I, I, fp, fp, fp, fp, fp, fp, I, I, I, lp, ip, fp, I, I, lp, ip, fp, ip, I, F,
                               vp, vp, vp, vp, vp, F]
        lib.or_set_threads.restype = I
        lib.or_set_threads.argtypes = [I]
        _lib32 = lib
    lib = _lib32
    eps = np.ascontiguousarray(eps_r, np.float32)
    ny, nx = eps.shape
    n = eps.size
    out = [np.empty(n, np.float32) for _ in range(4)]
    dl = np.empty(3 * n, np.float32)
    bc = np.zeros(3, np.int32)
    lib.or_medium(2, nx, ny, 1, 0.5, eps.ravel(), None, bc, 1.0, *out, dl)
    ceff2, cL2, w0, mu = out
    g = np.zeros(n * 5 * 4, np.float32)
    amp = np.ascontiguousarray(src_amp, np.float32).ravel()
    site = np.array([src_site], np.int64)
    tr = np.zeros(1, np.float32)
    nthr = lib.or_set_threads(int(threads_)) if threads_ else lib.or_set_threads(0)
    t0 = time.perf_counter()
    rc = lib.or_run(2, nx, ny, 1, cL2, w0, ceff2, mu, dl, g, 0, int(nsteps), 1, site, np.array([2], np.int32), amp,
                    amp.size, 0, np.zeros(1, np.int64), np.zeros(1, np.int32), tr, bc, 0, 0.0, None, None, None, None,
                    None, 1.0)
    dt = time.perf_counter() - t0
    assert rc == 0 and np.all(np.isfinite(g))
    return dt, nthr


@dataclass
class Oracle:
    """A medium on a periodic grid, as the oracle sees it (all FP64)."""

    D: int
    shape: tuple  # (ny, nx) or (nz, ny, nx)
    eps_r: np.ndarray
    ceff2: np.ndarray
    cL2: np.ndarray
    w0: np.ndarray
    mu: np.ndarray
    dlnmu: np.ndarray  # grid + (3,)
    bad: int
    bc: tuple = (0, 0, 0)  # per axis x, y, z: 0 periodic, 1 PEC wall, 2 PMC wall
    layer: int = 0  # absorbing layer width inside the walls (sites)
    gamma_max: float = 0.0  # damping of the wall-adjacent site
    wp2: np.ndarray = None  # frequency-dispersive permittivity: one Drude-Lorentz pole per site (grid), or None
    wr2: np.ndarray = None  # its resonance frequency squared (0: Drude)
    gamma: np.ndarray = None  # its damping rate
    aniso_r: float = 1.0  # sqrt(mu_xx / mu_yy) of a uniform in-plane permeability tensor (2D); 1: isotropic

    @property
    def dims(self):
        if self.D == 2:
            ny, nx = self.shape
            return nx, ny, 1
        nz, ny, nx = self.shape
        return nx, ny, nz

    @property
    def Q(self):
        return 2 * self.D + 1


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


PERIODIC, PEC, PMC = 0, 1, 2


def medium(D, eps_r, mu_r=None, c_ref2=None, bc=(0, 0, 0), layer=0, gamma_max=0.0, dispersion=None,
           aniso=None) -> Oracle:
    """Medium upload: eps_r, mu_r -> c_eff^2, c_L^2, w0, grad ln mu (Eq. 3).

    bc (x, y, z): 0 periodic, 1 PEC wall, 2 PMC wall on both ends of that axis; layer > 0 adds an
    absorbing layer of that many sites inside every wall, damping 1 - gamma_max ((L - i)/L)^2 at distance i.
    dispersion: dict(wp2=, wr2=, gamma=) (arrays of the grid's shape or scalars; wr2 and gamma default to 0): one
    Drude-Lorentz pole per site, d_t J + gamma J + wr2 P = wp2 E, J = d_t P; the lattice then carries D/eps_inf
    and the field is E = D/eps_inf - P (the oracle's reading R9).
    aniso: (mu_xx, mu_yy), a uniform in-plane relative permeability tensor (2D, mu_r must be None): per-axis
    lattice speeds c_x^2 = c_ref^2/(eps_r mu_yy), c_y^2 = c_ref^2/(eps_r mu_xx) (the oracle's reading R10)."""
    lib = _load()
    bc = tuple(int(b) for b in bc) + (0,) * (3 - len(bc))
    assert all(b in (PERIODIC, PEC, PMC) for b in bc) and (D == 3 or bc[2] == 0)
    assert layer >= 0 and 0.0 <= gamma_max < 1.0
    eps_r = _f64(eps_r)
    shape = eps_r.shape
    assert len(shape) == D
    if c_ref2 is None:
        c_ref2 = 0.5 if D == 2 else 1.0 / 6.0
    r = 1.0
    if aniso is not None:
        assert D == 2 and mu_r is None
        mxx, myy = float(aniso[0]), float(aniso[1])
        r = float(np.sqrt(mxx / myy))
        mu_r = np.full(shape, np.sqrt(mxx * myy))
    n = eps_r.size
    out = [np.empty(n) for _ in range(4)]
    dl = np.empty(3 * n)
    if mu_r is None:
        mu_ptr = None
    else:
        mu_r = _f64(mu_r)
        assert mu_r.shape == shape
        mu_ptr = mu_r.ctypes.data_as(C.c_void_p)
    nx, ny, nz = (shape[-1], shape[-2], shape[0] if D == 3 else 1)
    if aniso is not None:
        mu_r = _f64(mu_r)
        mu_ptr = mu_r.ctypes.data_as(C.c_void_p)
    bad = lib.or_medium(D, nx, ny, nz, float(c_ref2), eps_r.ravel(), mu_ptr, np.array(bc, np.int32), r, *out, dl)
    ceff2, cL2, w0, mu = (o.reshape(shape) for o in out)
    m = Oracle(D, shape, eps_r, ceff2, cL2, w0, mu, dl.reshape(shape + (3,)), int(bad), bc, int(layer),
               float(gamma_max))
    m.aniso_r = r
    if dispersion is not None:
        full = lambda v: np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), shape))
        m.wp2 = full(dispersion["wp2"])
        m.wr2 = full(dispersion.get("wr2", 0.0))
        m.gamma = full(dispersion.get("gamma", 0.0))
    return m


def pole_state(m: Oracle):
    """Zero state of the dispersive pole: dict(J=, P=), each grid + (3,) (J at t - 1/2, P at t)."""
    return dict(J=np.zeros(m.shape + (3,)), P=np.zeros(m.shape + (3,)))


def init_state(m: Oracle, E=None, B=None) -> np.ndarray:
    """g = g^(0)(E, B) at every site (Eq. 8); E, B have shape grid + (3,)."""
    lib = _load()
    g = np.zeros(m.shape + (m.Q, m.D, m.D))
    Ep = None if E is None else _f64(E, m.shape + (3,))
    Bp = None if B is None else _f64(B, m.shape + (3,))
    lib.or_init(m.D, *m.dims, m.cL2.ravel(), m.w0.ravel(),
                None if Ep is None else Ep.ctypes.data_as(C.c_void_p),
                None if Bp is None else Bp.ctypes.data_as(C.c_void_p), g.reshape(-1), m.aniso_r)
    return g


def _sources(sources, nsite):
    if sources is None:
        return 0, np.zeros(1, np.int64), np.zeros(1, np.int32), np.zeros(1), 1
    site = np.ascontiguousarray(sources["site"], dtype=np.int64).ravel()
    comp = np.ascontiguousarray(sources["comp"], dtype=np.int32).ravel()
    amp = _f64(sources["amp"])
    if amp.ndim == 1:
        amp = amp[None, :]
    assert amp.shape[0] == site.size == comp.size
    assert np.all((site >= 0) & (site < nsite)) and np.all((comp >= 0) & (comp < 3))
    return site.size, site, comp, np.ascontiguousarray(amp).ravel(), amp.shape[1]


def _receivers(receivers, nsite):
    if receivers is None:
        return 0, np.zeros(1, np.int64), np.zeros(1, np.int32)
    site = np.ascontiguousarray(receivers["site"], dtype=np.int64).ravel()
    comp = np.ascontiguousarray(receivers["comp"], dtype=np.int32).ravel()
    assert np.all((site >= 0) & (site < nsite)) and np.all((comp >= 0) & (comp < 6))
    return site.size, site, comp


def run(m: Oracle, g: np.ndarray, nsteps: int, t0: int = 0, sources=None, receivers=None, pole=None) -> np.ndarray:
    """Advance g (in place) by nsteps steps of Eqs. 17-18; returns receiver traces [nrec, nsteps].

    sources: dict(site=flat indices, comp=0..2, amp=[nsrc, nt] current density j(t)).
    receivers: dict(site=flat indices, comp=0..5 for E_x..E_z, B_x..B_z).
    pole: the dispersive pole's state (pole_state), advanced in place; required with a dispersive medium.
    """
    lib = _load()
    assert (m.wp2 is None) == (pole is None)
    vp = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
    if pole is not None:
        assert pole["J"].flags.c_contiguous and pole["P"].flags.c_contiguous
    assert g.dtype == np.float64 and g.flags.c_contiguous and g.shape == m.shape + (m.Q, m.D, m.D)
    n = m.cL2.size
    ns, ss, sc, sa, nt = _sources(sources, n)
    nr, rs, rc = _receivers(receivers, n)
    traces = np.zeros(max(nr, 1) * max(nsteps, 1))
    rc_ = lib.or_run(m.D, *m.dims, m.cL2.ravel(), m.w0.ravel(), m.ceff2.ravel(), m.mu.ravel(), m.dlnmu.reshape(-1),
                     g.reshape(-1), int(t0), int(nsteps), ns, ss, sc, sa, nt, nr, rs, rc, traces,
                     np.array(m.bc, np.int32), m.layer, m.gamma_max, vp(m.wp2), vp(m.wr2), vp(m.gamma),
                     vp(None if pole is None else pole["J"]), vp(None if pole is None else pole["P"]), m.aniso_r)
    assert rc_ == 0
    return traces[: nr * nsteps].reshape(nr, nsteps)


def fields(m: Oracle, g: np.ndarray, pole=None):
    """E, B (each grid + (3,)) from the moments of a pre-collision state (with a dispersive pole's state, E is
    the lattice's D/eps_inf minus P)."""
    lib = _load()
    n = m.cL2.size
    E = np.empty(3 * n)
    B = np.empty(3 * n)
    lib.or_fields(m.D, *m.dims, m.cL2.ravel(), np.ascontiguousarray(g).reshape(-1), E, B, m.aniso_r)
    E = E.reshape(m.shape + (3,))
    if pole is not None:
        E = E - pole["P"]
    return E, B.reshape(m.shape + (3,))


def diagnostics(m: Oracle, g: np.ndarray):
    """(field energy, sum g^2/w invariant, ||div B||_2) of a pre-collision state."""
    lib = _load()
    out = np.zeros(3)
    lib.or_diagnostics(m.D, *m.dims, m.cL2.ravel(), m.w0.ravel(), m.ceff2.ravel(),
                       np.ascontiguousarray(g).reshape(-1), out, m.aniso_r)
    return float(out[0]), float(out[1]), float(out[2])


def adjoint(m: Oracle, g0: np.ndarray, nsteps: int, sources, receivers, obs, t0: int = 0):
    """Misfit 1/2 sum (trace - obs)^2 and its gradient with respect to eps_r (grid shape); periodic only."""
    lib = _load()
    assert not any(m.bc) and m.aniso_r == 1.0 and m.wp2 is None
    n = m.cL2.size
    ns, ss, sc, sa, nt = _sources(sources, n)
    nr, rs, rc = _receivers(receivers, n)
    obs = _f64(obs).reshape(nr, nsteps)
    grad = np.zeros(n)
    mis = lib.or_adjoint(m.D, *m.dims, m.eps_r.ravel(), m.cL2.ravel(), m.mu.ravel(), m.dlnmu.reshape(-1),
                         np.ascontiguousarray(g0).reshape(-1), int(t0), int(nsteps), ns, ss, sc, sa, nt, nr, rs, rc,
                         np.ascontiguousarray(obs).ravel(), grad)
    return float(mis), grad.reshape(m.shape)
