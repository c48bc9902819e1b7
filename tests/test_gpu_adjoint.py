"""Hand-written adjoint (reverse-time stream-collide, FP64 gradient accumulation) against the oracle's own
adjoint on small grids and against central finite differences of the GPU forward on smooth permittivity
perturbations, including the full 192^3 x 1000-step configuration with checkpoints every 100 steps."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import f32, rel
from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu


def _small(D, shape, seed, nsteps):
    eps, _ = W.random_medium(shape, seed)
    p = W.Problem("adj", D, shape, eps, None, nsteps)
    n = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    p.src_site = np.array([n // 2, n // 3], np.int64)
    p.src_comp = np.array([2, 0 if D == 3 else 2], np.int32)
    p.src_amp = np.stack([W.ricker(nsteps, 0.12), 0.5 * W.ricker(nsteps, 0.2)])
    p.rec_site = rng.choice(n, 6, replace=False).astype(np.int64)
    p.rec_comp = np.array([2, 2, 3, 4, 5 if D == 3 else 2, 0 if D == 3 else 2], np.int32)
    return p


@pytest.mark.parametrize("D,shape,every,variant", [(2, (20, 27), 7, 0), (2, (9, 130), 40, 0), (3, (7, 8, 9), 5, 0),
                                                   (3, (7, 8, 9), 5, 1), (3, (5, 6, 70), 11, 1),
                                                   (3, (5, 6, 70), 11, 2)])
def test_adjoint_matches_oracle_adjoint(lbem, D, shape, every, variant):
    import torch

    from paper_1108_2651_gb300.autograd import misfit, receiver_traces

    p = _small(D, shape, 3, 30)
    obs = 0.05 * np.random.default_rng(4).standard_normal((p.rec_site.size, p.nsteps))
    s = lbem.Solver(shape)
    lbem.lbem_set_variant(s.h, variant)  # 3D: 0 = four sites per lane, 1 = one site per thread, 2 = capped
    eps = torch.tensor(np.asarray(p.eps_r, np.float32), device="cuda", requires_grad=True)
    tr = receiver_traces(eps, s, p, checkpoint_every=every)
    L = misfit(tr, torch.tensor(obs, device="cuda"))
    L.backward()
    g = eps.grad.double().cpu().numpy()
    s.close()
    m = O.medium(D, f32(p.eps_r))
    src = dict(site=p.src_site, comp=p.src_comp, amp=f32(p.src_amp))
    mis, og = O.adjoint(m, np.zeros(shape + (2 * D + 1, D, D)), p.nsteps, src, p.receivers(), obs)
    assert abs(L.item() - mis) < 1e-5 * mis
    assert rel(g, og) < 1e-4, rel(g, og)


def _fd_check(p, obs, perts, every, h, tol, c_ref2):
    import torch

    from paper_1108_2651_gb300.autograd import misfit, receiver_traces

    s = lbem.Solver(p.shape, c_ref2=c_ref2)
    eps0 = torch.tensor(np.asarray(p.eps_r, np.float32), device="cuda")
    obs_t = torch.as_tensor(obs, device="cuda")
    eps = eps0.clone().requires_grad_(True)
    L = misfit(receiver_traces(eps, s, p, checkpoint_every=every), obs_t)
    L.backward()
    grad = eps.grad.double()
    out = []

    def central(dt, hh):
        with torch.no_grad():
            lp = misfit(receiver_traces(eps0 + hh * dt, s, p, checkpoint_every=every), obs_t).item()
            lm = misfit(receiver_traces(eps0 - hh * dt, s, p, checkpoint_every=every), obs_t).item()
        return (lp - lm) / (2 * hh)

    for d in perts:
        dt = torch.as_tensor(d, device="cuda", dtype=torch.float32)
        # Richardson extrapolation of two central differences cancels their O(h^2) error
        fd = (4 * central(dt, h / 2) - central(dt, h)) / 3
        an = (grad * dt.double()).sum().item()
        out.append((fd, an))
    s.close()
    # FP32 forward runs put rounding noise of a fixed absolute size on the misfit, so the bar is relative
    # to the typical (RMS) directional derivative rather than to each one, some of which nearly vanish
    rms = float(np.sqrt(np.mean([an ** 2 for _, an in out])))
    for fd, an in out:
        assert abs(fd - an) <= tol * rms, (out, rms)
    return out


def test_adjoint_matches_finite_differences_2d(lbem):
    p = W.heterogeneous_2d(160, seed=9, nsteps=400, sigma=10.0, nrec=16, rec_radius=40)
    import torch

    s = lbem.Solver(p.shape)
    p2 = W.heterogeneous_2d(160, seed=10, nsteps=400, sigma=10.0, nrec=16, rec_radius=40)
    s.set_problem(p2)
    s.step(400)
    obs = s.traces(16).cpu().double().numpy()
    s.close()
    perts = [W.smooth_perturbation(p.shape, 100 + k, 8.0, amp=1.0) for k in range(4)]
    res = _fd_check(p, obs, perts, every=50, h=4e-3, tol=2e-3, c_ref2=0.97 * 0.5)
    rms = np.sqrt(np.mean([a ** 2 for _, a in res]))
    print("2D FD vs adjoint (|fd-adj|/rms):", [f"{abs(f - a) / rms:.1e}" for f, a in res])


@pytest.mark.slow
def test_adjoint_192_cubed_1000_steps_finite_differences_16_perturbations(lbem):
    """The full 3D configuration: 192^3, n in [1, 3] (smoothed, seed 4), Ricker j_z at the centre, 128
    receivers, 1000 steps, checkpoints every 100 steps, misfit against traces from a second medium (seed 5),
    16 smooth perturbations (seeds 100..115).  c_ref^2 is 3 % below 1/6 so that eps - h d stays a valid
    medium where n = 1."""
    import torch

    c_ref2 = 0.97 / 6.0
    p = W.heterogeneous_3d(192, seed=4, nsteps=1000)
    q = W.heterogeneous_3d(192, seed=5, nsteps=1000)
    s = lbem.Solver(q.shape, c_ref2=c_ref2)
    s.set_problem(q)
    s.step(1000)
    obs = s.traces(q.rec_site.size).cpu().double().numpy()
    s.close()
    perts = [W.smooth_perturbation(p.shape, 100 + k, 12.0, amp=1.0) for k in range(16)]
    res = _fd_check(p, obs, perts, every=100, h=4e-3, tol=1e-2, c_ref2=c_ref2)
    rms = np.sqrt(np.mean([a ** 2 for _, a in res]))
    print("192^3 FD vs adjoint (|fd-adj|/rms):", [f"{abs(f - a) / rms:.1e}" for f, a in res])
