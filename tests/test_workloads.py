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
