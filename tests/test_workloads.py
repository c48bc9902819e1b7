"""The seeded workload recipes (host-side input generation; no GPU)."""
import numpy as np


def test_mu_heterogeneous_workload_keeps_the_refractive_index():
    """The mu-heterogeneous recipe changes the impedance, not the wave speed: eps_r mu_r = n^2 of the eps-only
    recipe, mu_r in [1, 2]."""
    from paper_1108_2651_gb300 import workloads as W

    a = W.heterogeneous_2d(64, seed=5, nsteps=10, sigma=6.0)
    b = W.heterogeneous_2d_mu(64, seed=5, nsteps=10, sigma=6.0)
    np.testing.assert_allclose(b.eps_r * b.mu_r, a.eps_r, rtol=3e-7)
    assert np.all(b.eps_r * b.mu_r >= a.eps_r)  # never faster than the eps-only medium (w0 >= 0 where n = 1)
    assert np.array_equal(b.eps_r.astype(np.float32).astype(np.float64), b.eps_r)  # exact in FP32
    assert b.mu_r.min() >= 1.0 and b.mu_r.max() <= 2.0 and b.mu_r.max() - b.mu_r.min() > 0.5
    np.testing.assert_array_equal(a.src_amp, b.src_amp)


def test_heterogeneous_2d_recipe():
    """n = 1 + 2 s with s a periodic Gaussian-smoothed, min-max normalised field (so n spans exactly [1, 3]),
    eps_r = n^2, mu = 1; a unit Ricker current j_z at the centre peaking at 20 cells per local wavelength; 64
    receivers on a circle of radius min(256, n/4) at angles 2 pi k / 64."""
    from paper_1108_2651_gb300 import workloads as W

    n = 256
    p = W.heterogeneous_2d(n, seed=1, nsteps=400, sigma=20.0)
    nidx = np.sqrt(p.eps_r)
    assert abs(nidx.min() - 1.0) < 1e-12 and abs(nidx.max() - 3.0) < 1e-12 and p.mu_r is None
    # smooth (std 20 cells) and periodic: neighbouring cells, the wrap included, differ by little
    for ax in (0, 1):
        assert np.abs(np.diff(nidx, axis=ax, append=np.take(nidx, [0], axis=ax))).max() < 0.05
    c = n // 2
    assert p.src_site.tolist() == [c * n + c] and p.src_comp.tolist() == [2]
    f = np.sqrt(0.5) / nidx[c, c] / 20.0  # c_eff(x_s) / 20 cells per wavelength
    t0 = 1.5 / f
    amp = p.src_amp[0]
    assert abs(amp.max() - 1.0) < 1e-3 and abs(np.argmax(amp) - t0) <= 1
    ys, xs = np.divmod(p.rec_site, n)
    assert p.rec_site.size == 64 and np.unique(p.rec_site).size == 64
    r = np.hypot(ys - c, xs - c)
    assert np.all(np.abs(r - min(256, n // 4)) <= 0.75)
    ang = np.arctan2(ys - c, xs - c) % (2 * np.pi)
    assert np.all(np.abs((ang - 2 * np.pi * np.arange(64) / 64 + np.pi) % (2 * np.pi) - np.pi) < 0.02)


def test_batch_sizes_are_log_uniform_in_64_512():
    """256 square media with N_b = round(exp(U(ln 64, ln 512))) from PCG64(3): sizes in range, the mean of ln N
    near ln(64 * 512) / 2, and the total site count near 256 E[N^2] = 256 (512^2 - 64^2) / (2 ln 8) = 15.9 M."""
    from paper_1108_2651_gb300 import workloads as W

    s = np.array(W.batch_sizes())
    assert s.size == 256 and s.min() >= 64 and s.max() <= 512
    assert s.tolist() == W.batch_sizes()  # seeded
    assert abs(np.log(s).mean() - 0.5 * np.log(64 * 512)) < 0.15
    expect = 256 * (512 ** 2 - 64 ** 2) / (2 * np.log(8))
    assert abs((s.astype(np.float64) ** 2).sum() / expect - 1) < 0.15
    assert len(set(s.tolist())) > 100  # ragged: many distinct sizes, most not multiples of the tile width


def test_drude_aniso_and_walls_recipes_respect_their_bounds():
    """The Drude cylinder (radius n/8, n/4 from the source along x) keeps wp^2 <= 4 w0 with w0 = 1 - 1/eps_r;
    the uniaxial medium keeps the rest weight 1 - c_x^2 - c_y^2 >= 0; the walled box has its layer inside
    half the grid."""
    from paper_1108_2651_gb300 import workloads as W

    n = 128
    d = W.heterogeneous_2d_drude(n, seed=2, nsteps=10)
    y, x = np.mgrid[0:n, 0:n]
    disk = (x - (n // 2 + n // 4)) ** 2 + (y - n // 2) ** 2 <= (n / 8) ** 2
    assert np.all(d.wp2[disk] == 0.5) and np.all(d.wp2[~disk] == 0) and np.all(d.gamma[disk] == 0.01)
    assert np.all(d.wr2 == 0) and np.all(d.eps_r[disk] >= 2.25)
    w0 = 1 - 1 / np.asarray(d.eps_r, np.float32).astype(np.float64)
    assert np.all(d.wp2 + d.wr2 <= 4 * w0)
    base = W.heterogeneous_2d(n, seed=2, nsteps=10)
    np.testing.assert_array_equal(d.eps_r[~disk], base.eps_r[~disk])
    a = W.heterogeneous_2d_aniso(n, seed=2, nsteps=10)
    mxx, myy = a.aniso
    e = np.asarray(a.eps_r, np.float32).astype(np.float64)
    assert np.all(1 - 0.5 / (e * myy) - 0.5 / (e * mxx) >= -1e-12) and a.mu_r is None
    w = W.heterogeneous_2d_walls(n, seed=2, nsteps=10)
    assert w.bc == (1, 1, 0) and 0 < 2 * w.layer <= n and 0 <= w.gamma_max < 1


def test_heterogeneous_3d_recipe():
    """192^3 recipe at a small size: n in [1, 3], Ricker j_z at the centre, 8 x 16 receivers of E_z on the plane
    z = n/2 + 48 (clamped inside the grid)."""
    from paper_1108_2651_gb300 import workloads as W

    n = 64
    p = W.heterogeneous_3d(n, nsteps=20, sigma=6.0, plane_dz=16)
    nidx = np.sqrt(p.eps_r)
    assert abs(nidx.min() - 1) < 1e-12 and abs(nidx.max() - 3) < 1e-12
    c = n // 2
    assert p.src_site.tolist() == [(c * n + c) * n + c] and p.src_comp.tolist() == [2]
    z, rem = np.divmod(p.rec_site, n * n)
    assert p.rec_site.size == 128 and np.all(z == c + 16) and np.all(p.rec_comp == 2)
    assert np.unique(rem).size == 128
