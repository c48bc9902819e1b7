"""Pins of the oracle's walls and absorbing layers (2D).

The paper treats periodic domains only and leaves reflecting and absorbing
boundaries open; the oracle reads them as follows.  A wall half a site beyond
the edge sends a particle that would cross it back into the site it left, in
the opposite direction, times -1 (PEC: E_z = 0 and B_normal = 0 on the wall)
or +1 (PMC: tangential B = 0).  An absorbing layer of L sites inside a wall
multiplies the post-collision populations at distance i from the
wall-adjacent site by 1 - gamma_max ((L - i)/L)^2.

What pins them, other than the oracle itself:
  * the method of images: a domain with walls evolves exactly as the periodic
    domain twice as long (per walled axis) holding the mirror image of medium,
    fields and currents (directions i <-> opposite(i), times the wall sign),
    which the periodic pins tie to the paper;
  * exact conservation of the discrete invariant sum g^2/w with walls (the
    reflection is a signed permutation of post-collision populations);
  * the layer: where each damping factor acts (site the population leaves,
    axis, corner product), that the invariant never grows with it, and that a
    pulse sent into it comes back with a tiny fraction of its energy while
    the bare wall returns all of it.
"""
import numpy as np
import pytest

import oracle as O

PEC, PMC = O.PEC, O.PMC


def _mirror(a, axis, s=1.0):
    """Grid array (ny, nx, ...) doubled along `axis` (0 = y, 1 = x): index n + k holds s * a[n - 1 - k]."""
    return np.concatenate([a, s * np.flip(a, axis=axis)], axis=axis)


def _mirror_g(g, axis, s):
    """Oracle state (ny, nx, 5, 2, 2) doubled along `axis`: the image swaps the two directions along that axis
    (1 <-> 3 for x, 2 <-> 4 for y) and carries the wall sign."""
    gm = np.flip(g, axis=axis).copy()
    a, b = (1, 3) if axis == 1 else (2, 4)
    gm[:, :, [a, b]] = gm[:, :, [b, a]]
    return np.concatenate([g, s * gm], axis=axis)


def _problem(ny, nx, seed, mu=True):
    rng = np.random.default_rng(seed)
    eps = 1.0 + rng.random((ny, nx))
    mur = 1.0 + 0.5 * rng.random((ny, nx)) if mu else None
    E = np.zeros((ny, nx, 3))
    B = np.zeros((ny, nx, 3))
    E[..., 2] = rng.standard_normal((ny, nx))
    B[..., :2] = rng.standard_normal((ny, nx, 2))
    site = np.unique(np.concatenate([[0, nx - 1, (ny - 1) * nx], rng.integers(0, ny * nx, 3)]))
    amp = rng.standard_normal((site.size, 60))
    return eps, mur, E, B, site, amp


@pytest.mark.parametrize("bc", [(PEC, 0), (PMC, 0), (0, PEC), (0, PMC), (PEC, PEC), (PEC, PMC), (PMC, PMC)])
def test_walls_equal_the_mirror_image_on_a_doubled_periodic_domain(bc):
    ny, nx, nsteps = 9, 11, 60
    eps, mur, E, B, site, amp = _problem(ny, nx, 3 + bc[0] + 3 * bc[1])
    m = O.medium(2, eps, mur, bc=bc)
    g = O.init_state(m, E, B)
    recs = dict(site=site, comp=np.arange(site.size) % 6)
    tr = O.run(m, g, nsteps, sources=dict(site=site, comp=np.full(site.size, 2), amp=amp), receivers=recs)
    Ew, Bw = O.fields(m, g)

    # the image: mirror along every walled axis; currents carry the wall sign (j_z odd about a PEC wall)
    ebig, mbig = eps, mur
    g0 = O.init_state(m, E, B)
    Y, X = np.divmod(site, nx)
    for axis, kind in ((1, bc[0]), (0, bc[1])):
        if not kind:
            continue
        s = -1.0 if kind == PEC else 1.0
        ebig = _mirror(ebig, axis)
        mbig = _mirror(mbig, axis)
        g0 = _mirror_g(g0, axis, s)
    NY, NX = ebig.shape
    # sources: one per image, amplitude times the product of the wall signs it was reflected through
    bsite, bamp = [], []
    for yy, xx, a in zip(Y, X, amp):
        for fy in ((0, 1) if bc[1] else (0,)):
            for fx in ((0, 1) if bc[0] else (0,)):
                sgn = (-1.0 if (fx and bc[0] == PEC) else 1.0) * (-1.0 if (fy and bc[1] == PEC) else 1.0)
                by = 2 * ny - 1 - yy if fy else yy
                bx = 2 * nx - 1 - xx if fx else xx
                bsite.append(by * NX + bx)
                bamp.append(sgn * a)
    mb = O.medium(2, ebig, mbig)
    assert not np.any(mb.bc)
    brec = dict(site=(Y * NX + X), comp=recs["comp"])
    trb = O.run(mb, g0, nsteps, sources=dict(site=np.array(bsite), comp=np.full(len(bsite), 2),
                                              amp=np.array(bamp)), receivers=brec)
    Eb, Bb = O.fields(mb, g0)
    scale = max(np.abs(Ew).max(), np.abs(Bw).max())
    np.testing.assert_allclose(Eb[:ny, :nx], Ew, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(Bb[:ny, :nx], Bw, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(trb, tr, rtol=0, atol=1e-12 * max(1.0, np.abs(tr).max()))
    # grad ln mu at the edge sites is that of the mirror image
    np.testing.assert_allclose(m.dlnmu, mb.dlnmu[:ny, :nx], rtol=0, atol=1e-15)


def test_walls_keep_the_discrete_invariant_exactly():
    """Homogeneous medium (the weights w_i are then the same at every site): the invariant is exact."""
    ny, nx = 14, 17
    _, _, E, B, _, _ = _problem(ny, nx, 7, mu=False)
    eps = np.full((ny, nx), 1.7)
    for bc in ((PEC, PMC), (PMC, PEC), (PEC, PEC)):
        m = O.medium(2, eps, bc=bc)
        g = O.init_state(m, E, B)
        inv0 = O.diagnostics(m, g)[1]
        for _ in range(5):
            O.run(m, g, 40)
            assert abs(O.diagnostics(m, g)[1] / inv0 - 1) < 1e-13


def _layer_factor(v, n, L, gmax):
    i = min(v, n - 1 - v)
    return 1.0 - gmax * ((L - i) / L) ** 2 if i < L else 1.0


def test_layer_damps_each_population_by_the_factor_of_the_site_it_leaves():
    """One step from a random state with and without the layer: every population of the new state is the
    undamped one times the layer factor of the site it was collided at (its upwind neighbour, or the site
    itself after a wall reflection), the two axes' factors multiplied at corners."""
    ny, nx, L, gmax = 13, 16, 5, 0.3
    eps, _, E, B, _, _ = _problem(ny, nx, 9, mu=False)
    for bc in ((PEC, 0), (0, PMC), (PEC, PMC)):
        m0 = O.medium(2, eps, bc=bc)
        m1 = O.medium(2, eps, bc=bc, layer=L, gamma_max=gmax)
        g0 = O.init_state(m0, E, B)
        g1 = g0.copy()
        O.run(m0, g0, 1)
        O.run(m1, g1, 1)
        c = {1: (1, 0), 2: (0, 1), 3: (-1, 0), 4: (0, -1)}
        for y in range(ny):
            for x in range(nx):
                for i in range(5):
                    dx, dy = c.get(i, (0, 0))
                    sx, sy = x - dx, y - dy
                    if (bc[0] and not 0 <= sx < nx) or (bc[1] and not 0 <= sy < ny):
                        sx, sy = x, y  # reflected at a wall: it left this site
                    sx, sy = sx % nx, sy % ny
                    f = (_layer_factor(sx, nx, L, gmax) if bc[0] else 1.0) * \
                        (_layer_factor(sy, ny, L, gmax) if bc[1] else 1.0)
                    np.testing.assert_allclose(g1[y, x, i], f * g0[y, x, i], rtol=1e-14, atol=1e-15)


def test_layer_never_increases_the_invariant_and_zero_strength_changes_nothing():
    ny, nx = 20, 24
    _, _, E, B, _, _ = _problem(ny, nx, 11, mu=False)
    eps = np.full((ny, nx), 1.3)
    m = O.medium(2, eps, bc=(PEC, PMC), layer=6, gamma_max=0.25)
    g = O.init_state(m, E, B)
    prev = O.diagnostics(m, g)[1]
    for _ in range(30):
        O.run(m, g, 3)
        cur = O.diagnostics(m, g)[1]
        assert cur <= prev * (1 + 1e-14)
        prev = cur
    assert prev < 0.5 * O.diagnostics(m, O.init_state(m, E, B))[1]
    ma = O.medium(2, eps, bc=(PEC, PMC))
    mb = O.medium(2, eps, bc=(PEC, PMC), layer=6, gamma_max=0.0)
    ga, gb = O.init_state(ma, E, B), O.init_state(mb, E, B)
    O.run(ma, ga, 25)
    O.run(mb, gb, 25)
    np.testing.assert_array_equal(ga, gb)


@pytest.mark.parametrize("kind", [PEC, PMC])
def test_layer_absorbs_a_pulse_the_bare_wall_returns(kind):
    """A Gaussian E_z slab between two walls, long enough for both halves to reach a wall and come back: the
    bare walls return all of the field energy; a 32-site layer (gamma_max = 0.2) leaves less than 1e-5 of it."""
    ny, nx = 4, 600
    x = np.arange(nx)
    E = np.zeros((ny, nx, 3))
    E[..., 2] = np.exp(-((x - nx / 2) / 6.0) ** 2)[None, :]
    B = np.zeros_like(E)
    T = int(nx / 2 / np.sqrt(0.5)) + 50
    left = []
    for L, gmax in ((0, 0.0), (32, 0.2)):
        m = O.medium(2, np.ones((ny, nx)), bc=(kind, 0), layer=L, gamma_max=gmax)
        g = O.init_state(m, E, B)
        e0 = O.diagnostics(m, g)[0]
        O.run(m, g, T)
        left.append(O.diagnostics(m, g)[0] / e0)
    assert abs(left[0] - 1) < 1e-2, left
    assert left[1] < 1e-5, left


@pytest.mark.parametrize("kind", [PEC, PMC])
def test_walls_with_a_dispersive_pole_and_anisotropy_equal_the_mirror_image(kind):
    """The method of images with the other readings switched on: a Drude-Lorentz pole per site (its J and P
    mirror with E, times the wall sign) and a uniform permeability tensor (the mirror keeps each axis)."""
    ny, nx, nsteps = 8, 10, 40
    rng = np.random.default_rng(31 + kind)
    eps = 1.5 + rng.random((ny, nx))
    aniso = (1.8, 1.1)
    r = np.sqrt(aniso[0] / aniso[1])
    w0 = 1 - (r + 1 / r) * 0.5 / (eps * np.sqrt(aniso[0] * aniso[1]))
    wp2, wr2, gam = 2.0 * w0 * rng.random((ny, nx)), 1.0 * w0 * rng.random((ny, nx)), 0.1 * rng.random((ny, nx))
    E = np.zeros((ny, nx, 3))
    B = np.zeros_like(E)
    E[..., 2] = rng.standard_normal((ny, nx))
    B[..., :2] = rng.standard_normal((ny, nx, 2))
    m = O.medium(2, eps, bc=(kind, 0), aniso=aniso, dispersion=dict(wp2=wp2, wr2=wr2, gamma=gam))
    g = O.init_state(m, E, B)
    pole = O.pole_state(m)
    O.run(m, g, nsteps, pole=pole)
    Ew, Bw = O.fields(m, g, pole)
    s = -1.0 if kind == PEC else 1.0
    mb = O.medium(2, _mirror(eps, 1), aniso=aniso,
                  dispersion=dict(wp2=_mirror(wp2, 1), wr2=_mirror(wr2, 1), gamma=_mirror(gam, 1)))
    gb = _mirror_g(O.init_state(m, E, B), 1, s)
    pb = O.pole_state(mb)
    O.run(mb, gb, nsteps, pole=pb)
    Eb, Bb = O.fields(mb, gb, pb)
    scale = max(np.abs(Ew).max(), np.abs(Bw).max())
    np.testing.assert_allclose(Eb[:, :nx], Ew, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(Bb[:, :nx], Bw, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(pb["P"][:, :nx], pole["P"], rtol=0, atol=1e-12 * scale)


def _mirror3(a, axis, s=1.0):
    return np.concatenate([a, s * np.flip(a, axis=axis)], axis=axis)


def _mirror_g3(g, ax, kind):
    """3D oracle state (nz, ny, nx, 7, 3, 3) doubled across the wall normal to lattice axis `ax` (0 = x, 1 = y,
    2 = z): directions +ax and -ax swap, component (b, c) takes (b == ax ? -1 : 1)(c == ax ? -1 : 1), the
    geometric mirror of the tensor, times +1 for PEC and -1 for PMC."""
    arr_axis = 2 - ax
    gm = np.flip(g, axis=arr_axis).copy()
    p, m = 1 + ax, 4 + ax
    gm[..., [p, m], :, :] = gm[..., [m, p], :, :]
    sign = np.ones((3, 3))
    sign[ax, :] *= -1
    sign[:, ax] *= -1
    gm *= sign * (1.0 if kind == PEC else -1.0)
    return np.concatenate([g, gm], axis=arr_axis)


@pytest.mark.parametrize("bc", [(PEC, 0, 0), (0, PMC, 0), (0, 0, PEC), (PMC, PEC, 0), (PEC, PEC, PMC)])
def test_3d_walls_equal_the_mirror_image_on_a_doubled_periodic_domain(bc):
    """3D: the tensor's geometric mirror (PEC) or its negative (PMC) per walled axis; currents mirror with an
    extra -1 (the source enters as eps_gab S_g, a pseudotensor): j' = (PEC: -1, PMC: +1) x R j."""
    nz, ny, nx, nsteps = 4, 5, 6, 16
    rng = np.random.default_rng(41 + bc[0] + 3 * bc[1] + 9 * bc[2])
    shape = (nz, ny, nx)
    eps = 1.5 + rng.random(shape)
    mur = 1.0 + 0.5 * rng.random(shape)
    E = rng.standard_normal(shape + (3,))
    B = rng.standard_normal(shape + (3,))
    site = np.array([0, nx - 1, nx * ny * nz - 1, 37])
    comp = np.array([0, 1, 2, 2])
    amp = rng.standard_normal((site.size, nsteps))
    m = O.medium(3, eps, mur, bc=bc)
    g = O.init_state(m, E, B)
    O.run(m, g, nsteps, sources=dict(site=site, comp=comp, amp=amp))
    Ew, Bw = O.fields(m, g)

    ebig, mbig, g0 = eps, mur, O.init_state(m, E, B)
    for ax in range(3):
        if bc[ax]:
            ebig = _mirror3(ebig, 2 - ax)
            mbig = _mirror3(mbig, 2 - ax)
            g0 = _mirror_g3(g0, ax, bc[ax])
    NZ, NY, NX = ebig.shape
    Z, rem = np.divmod(site, nx * ny)
    Y, X = np.divmod(rem, nx)
    bsite, bcomp, bamp = [], [], []
    for z, y, x, c, a in zip(Z, Y, X, comp, amp):
        for fz in ((0, 1) if bc[2] else (0,)):
            for fy in ((0, 1) if bc[1] else (0,)):
                for fx in ((0, 1) if bc[0] else (0,)):
                    sgn = 1.0
                    for ax, f in ((0, fx), (1, fy), (2, fz)):
                        if f:
                            sgn *= (-1.0 if bc[ax] == PEC else 1.0) * (-1.0 if c == ax else 1.0)
                    zz = 2 * nz - 1 - z if fz else z
                    yy = 2 * ny - 1 - y if fy else y
                    xx = 2 * nx - 1 - x if fx else x
                    bsite.append(xx + NX * (yy + NY * zz))
                    bcomp.append(c)
                    bamp.append(sgn * a)
    mb = O.medium(3, ebig, mbig)
    O.run(mb, g0, nsteps, sources=dict(site=np.array(bsite), comp=np.array(bcomp), amp=np.array(bamp)))
    Eb, Bb = O.fields(mb, g0)
    scale = max(np.abs(Ew).max(), np.abs(Bw).max())
    np.testing.assert_allclose(Eb[:nz, :ny, :nx], Ew, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(Bb[:nz, :ny, :nx], Bw, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(m.dlnmu, mb.dlnmu[:nz, :ny, :nx], rtol=0, atol=1e-15)


def test_3d_walls_keep_the_discrete_invariant_exactly():
    rng = np.random.default_rng(43)
    shape = (5, 6, 7)
    m = O.medium(3, np.full(shape, 1.7), bc=(PEC, PMC, PEC))
    g = O.init_state(m, rng.standard_normal(shape + (3,)), rng.standard_normal(shape + (3,)))
    inv0 = O.diagnostics(m, g)[1]
    O.run(m, g, 60)
    assert abs(O.diagnostics(m, g)[1] / inv0 - 1) < 1e-13


def test_3d_layer_damps_each_population_by_the_factor_of_the_site_it_leaves():
    """3D: one step with and without a layer; every population of the new state is the undamped one times the
    product of the three axes' factors at the site it left (its upwind neighbour, or itself after a wall)."""
    nz, ny, nx, L, gmax = 9, 8, 10, 3, 0.35
    rng = np.random.default_rng(47)
    eps = 1.5 + rng.random((nz, ny, nx))
    E, B = rng.standard_normal((nz, ny, nx, 3)), rng.standard_normal((nz, ny, nx, 3))
    bc = (PEC, PMC, PEC)
    m0 = O.medium(3, eps, bc=bc)
    m1 = O.medium(3, eps, bc=bc, layer=L, gamma_max=gmax)
    g0 = O.init_state(m0, E, B)
    g1 = g0.copy()
    O.run(m0, g0, 1)
    O.run(m1, g1, 1)
    c = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0), (0, -1, 0), (0, 0, -1)]
    n = (nx, ny, nz)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for i in range(7):
                    src = [x - c[i][0], y - c[i][1], z - c[i][2]]
                    if any(not 0 <= src[a] < n[a] for a in range(3)):
                        src = [x, y, z]  # reflected at a wall: it left this site
                    f = np.prod([_layer_factor(src[a], n[a], L, gmax) for a in range(3)])
                    np.testing.assert_allclose(g1[z, y, x, i], f * g0[z, y, x, i], rtol=1e-14, atol=1e-15)
