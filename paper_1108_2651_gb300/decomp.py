"""Spatial domain decomposition: slabs along the slowest axis (y in 2D, z in 3D).

The scheme is local: per step a site reads its own collided populations and one population from each neighbour
(pull streaming, Eq. 18).  Cut the grid into slabs of whole rows (2D) or planes (3D) and give every slab one ghost
layer on either side.  The library steps each slab as its own periodic grid, which only ever disturbs the ghost
layers.  What a real layer reads across a cut is the population moving across it: 2D g_2 (moving +y) from the
layer below and g_4 (-y) from the layer above; 3D the three +z and the three -z components.  So after every
single step each slab sends those populations of its first and last real layers to its neighbours, which write
them into their ghost layers, and the slabs together evolve exactly as the whole grid (bit for bit: every site
update has the same inputs).

Communication is neighbour point-to-point (torch.distributed send / receive: NCCL between GPUs, gloo on the host)
or, for slabs held by one process, direct copies.  Each slab steps one step per launch (the halo is one layer
deep).  Any medium the library steps: a heterogeneous mu, a uniform anisotropic tensor, a dispersive pole (its
J and P are site-local, so nothing of it crosses a cut), walls and absorbing layers on the axes along the cuts
(x in 2D; x, y in 3D); the slab axis itself stays periodic.  Sources and receivers on real layers.
"""
from dataclasses import replace

import numpy as np

from . import lbem

# populations crossing a cut, in the library's plane numbering: moving up (towards larger y / z), moving down
CROSSING = {2: ((2,), (4,)), 3: ((9, 10, 11), (18, 19, 20))}


def slab_range(n, world, rank):
    """Layers [start, start + count) of rank `rank` when n layers are cut into `world` nearly equal slabs."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def local_problem(p, rank, world):
    """The slab of workloads.Problem p held by `rank`, with one ghost layer on either side (the neighbouring
    layers of the whole grid, periodic).  Returns (local problem, start, count, indices of the global receivers
    it holds)."""
    D = len(p.shape)
    assert not p.bc[D - 1], "the slab axis must be periodic (walls only on the axes along the cuts)"
    n = p.shape[0]
    start, count = slab_range(n, world, rank)
    assert count >= 1, "more ranks than layers"
    layers = np.arange(start - 1, start + count + 1) % n
    take = lambda a: None if a is None else np.take(a, layers, axis=0)
    site = lambda a: None if a is None else take(np.broadcast_to(a, p.shape))  # a per-site parameter or a scalar
    shape = (count + 2,) + tuple(p.shape[1:])
    per_layer = int(np.prod(p.shape[1:]))

    def localize(sites):
        layer = sites // per_layer
        keep = (layer >= start) & (layer < start + count)
        return keep, (layer - start + 1) * per_layer + sites % per_layer

    q = replace(p, shape=shape, eps_r=take(p.eps_r), mu_r=take(p.mu_r), E0=take(p.E0), B0=take(p.B0),
                wp2=site(p.wp2), wr2=site(p.wr2), gamma=site(p.gamma))
    keep, loc = localize(p.src_site)
    q.src_site, q.src_comp, q.src_amp = loc[keep].astype(np.int64), p.src_comp[keep], p.src_amp[keep]
    keep, loc = localize(p.rec_site)
    q.rec_site, q.rec_comp = loc[keep].astype(np.int64), p.rec_comp[keep]
    return q, start, count, np.nonzero(keep)[0]


class LbemSlab:
    """One slab on the current GPU, stepped by the library (one step per launch)."""

    def __init__(self, q, count, stream=None):
        import torch

        self.D = len(q.shape)
        self.count = count
        self.rows_per_layer = 1 if self.D == 2 else q.shape[1]
        self.nx = q.shape[-1]
        self.s = lbem.Solver(q.shape, stream=stream)
        self.s.set_problem(q)
        lbem.lbem_set_temporal_blocking(self.s.h, 1, -1)
        self.torch = torch

    def step(self):
        self.s.step(1)

    def _rows(self, planes, layer, buf, to_state):
        r = self.rows_per_layer
        for k, pl in enumerate(planes):
            lbem.lbem_rows(self.s.h, pl, layer * r, r, buf[k], to_state)

    def halo_out(self, up):
        """Populations this slab sends across its upper (up) or lower cut: the crossing planes of its last or
        first real layer."""
        planes = CROSSING[self.D][0 if up else 1]
        buf = self.torch.empty((len(planes), self.rows_per_layer * self.nx), dtype=self.torch.float32, device="cuda")
        self._rows(planes, self.count if up else 1, buf, False)
        return buf

    def halo_in(self, from_below, buf):
        """Write what the slab below (from_below) or above sent into the matching ghost layer."""
        planes = CROSSING[self.D][0 if from_below else 1]
        self._rows(planes, 0 if from_below else self.count + 1, buf.to(device="cuda", dtype=self.torch.float32),
                   True)

    def fields(self):
        """E, B of the real layers, each (3,) + slab shape without ghosts (torch, on the GPU)."""
        E, B = self.s.fields()
        return E[:, 1:self.count + 1], B[:, 1:self.count + 1]

    def traces(self, n):
        return self.s.traces(n)

    def close(self):
        self.s.close()


def exchange_local(slabs):
    """Halo exchange between slabs held by one process (periodic: the last slab's upper neighbour is the first)."""
    ups = [s.halo_out(True) for s in slabs]
    downs = [s.halo_out(False) for s in slabs]
    n = len(slabs)
    for r, s in enumerate(slabs):
        s.halo_in(True, ups[(r - 1) % n])
        s.halo_in(False, downs[(r + 1) % n])


def exchange_dist(slab, rank, world, host=False):
    """Halo exchange of this rank's slab with its neighbours over torch.distributed (periodic ring).  host=True
    stages the buffers through host memory (gloo)."""
    import torch.distributed as dist

    up, down = slab.halo_out(True), slab.halo_out(False)
    if host:
        up, down = up.cpu(), down.cpu()
    if world == 1:
        slab.halo_in(True, up)
        slab.halo_in(False, down)
        return
    from_below, from_above = up.clone(), down.clone()
    UP, DOWN = 1, 2  # message tags: with two ranks both neighbours are the same rank
    ops = [dist.P2POp(dist.isend, up, (rank + 1) % world, tag=UP),
           dist.P2POp(dist.isend, down, (rank - 1) % world, tag=DOWN),
           dist.P2POp(dist.irecv, from_below, (rank - 1) % world, tag=UP),
           dist.P2POp(dist.irecv, from_above, (rank + 1) % world, tag=DOWN)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    slab.halo_in(True, from_below)
    slab.halo_in(False, from_above)


def step_local(slabs, nsteps):
    """Advance slabs held by one process by nsteps steps."""
    for _ in range(nsteps):
        for s in slabs:
            s.step()
        exchange_local(slabs)


def step_dist(slab, rank, world, nsteps, host=False):
    """Advance this rank's slab by nsteps steps, exchanging halos after each."""
    for _ in range(nsteps):
        slab.step()
        exchange_dist(slab, rank, world, host)


def energy(E, B, eps_r, mu_r, c_ref2):
    """FP64 field energy sum_a (B_a^2 + E_a^2 / c_eff^2), c_eff^2 = c_ref2 / (eps_r mu_r), over one slab's real
    layers (E, B: (3,) + slab shape, torch or numpy; eps_r, mu_r: slab shape, mu_r None for 1).  Summed over the
    slabs (an FP64 all-reduce across ranks) it is the whole grid's energy."""
    e = np.asarray(E.double().cpu().numpy() if hasattr(E, "cpu") else E, np.float64)
    b = np.asarray(B.double().cpu().numpy() if hasattr(B, "cpu") else B, np.float64)
    em = np.asarray(eps_r, np.float32).astype(np.float64)
    if mu_r is not None:
        em = em * np.asarray(mu_r, np.float32).astype(np.float64)
    return float((b ** 2).sum() + ((e ** 2).sum(axis=0) * em / c_ref2).sum())
