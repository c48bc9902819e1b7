"""Shared helpers of the GPU parity tests: run one problem on the GPU library and on the oracle."""
import numpy as np

import oracle as O
from paper_1108_2651_gb300 import lbem


def gpu_run(p, storage="f32", nsteps=None, variant=None, graphs=False, steps_per_pass=None):
    """Run workloads.Problem p on the GPU; returns (E, B, traces) as float64 numpy, E/B grid + (3,).
    A given single-step variant runs every step (steps_per_pass 1); steps_per_pass None keeps the library
    default (two steps per launch where that applies)."""
    import torch

    nsteps = p.nsteps if nsteps is None else nsteps
    stream = torch.cuda.Stream() if graphs else None  # graph capture needs a non-default stream
    s = lbem.Solver(p.shape, storage=storage, stream=stream.cuda_stream if stream else None)
    try:
        s.set_problem(p)
        if variant is not None:
            lbem.lbem_set_variant(s.h, variant)
            steps_per_pass = 1 if steps_per_pass is None else steps_per_pass
        if steps_per_pass is not None:
            lbem.lbem_set_temporal_blocking(s.h, steps_per_pass, -1)
        if graphs:
            lbem.lbem_set_graphs(s.h, True)
        s.step(nsteps)
        E, B = s.fields()
        tr = s.traces(p.rec_site.size)
        torch.cuda.synchronize()
        lbem.lbem_check_guards(s.h)  # no kernel wrote outside a handle-owned array
        E = np.moveaxis(E.cpu().double().numpy(), 0, -1)
        B = np.moveaxis(B.cpu().double().numpy(), 0, -1)
        return E, B, tr.cpu().double().numpy()
    finally:
        s.close()


def f32(a):
    """The float32 value the GPU receives, as float64 (both sides get identical inputs)."""
    return None if a is None else np.asarray(a, np.float32).astype(np.float64)


def oracle_run(p, nsteps=None):
    """The same problem on the FP64 oracle; returns (E, B, traces, medium, state)."""
    nsteps = p.nsteps if nsteps is None else nsteps
    disp = None
    if p.wp2 is not None:
        full = lambda a: f32(np.broadcast_to(0.0 if a is None else a, p.shape))
        disp = dict(wp2=full(p.wp2), wr2=full(p.wr2), gamma=full(p.gamma))
    m = O.medium(p.D, f32(p.eps_r), f32(p.mu_r), bc=p.bc, layer=p.layer, gamma_max=p.gamma_max, dispersion=disp,
                 aniso=p.aniso)
    g = O.init_state(m, f32(p.E0), f32(p.B0))
    pole = O.pole_state(m) if disp is not None else None
    src = p.sources()
    if src is not None:
        src = dict(src, amp=f32(src["amp"]))
    tr = O.run(m, g, nsteps, sources=src, receivers=p.receivers(), pole=pole)
    E, B = O.fields(m, g, pole)
    return E, B, tr, m, g


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
