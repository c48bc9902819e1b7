"""Spatial domain decomposition: slabs along the slowest axis (y in 2D, z in 3D).

The scheme is local: per step a site reads its own collided populations and one population from each neighbour
(pull streaming, Eq. 18).  Cut the grid into slabs of whole rows (2D) or planes (3D) and give every slab `halo`
ghost layers on either side.  The library steps each slab as its own periodic grid, which disturbs only the ghost
layers; after every `halo` steps each slab sends its neighbours what their ghost layers need, and the slabs together
evolve exactly as the whole grid (bit for bit: every site update has the same inputs).

* halo = 1 (2D and 3D, every medium): after each single step, the populations crossing a cut: 2D g_2 (moving +y)
  of the last real layer up and g_4 (-y) of the first real layer down; 3D the three +z and the three -z components.
* halo = 2 (2D; not with a dispersive pole, whose P would have to cross too): two steps per exchange, so the
  library advances each slab two steps per launch (temporal blocking).  The inner ghost layer's first-step
  collision now feeds a real layer, so it needs its own populations and sources: up go g_0..g_3 of the last real
  layer and g_2 of the one below it, down g_0, g_1, g_3, g_4 of the first real layer and g_4 of the one above it:
  5 rows of nx floats per cut and direction per two steps (against 2 for two single-step exchanges), in half the
  messages.

Communication is neighbour point-to-point (torch.distributed send / receive: NCCL between GPUs, gloo on the host)
or, for slabs held by one process, direct copies.  Any medium the library steps: a heterogeneous mu, a uniform
anisotropic tensor, a dispersive pole (halo 1: its J and P are site-local, so nothing of it crosses a cut), walls and
absorbing layers on the axes along the cuts (x in 2D; x, y in 3D); the slab axis itself stays periodic.  Receivers
on real layers; sources on real layers and, with halo = 2, on ghost layers as well.
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


def local_problem(p, rank, world, halo=1):
    """The slab of workloads.Problem p held by `rank`, with `halo` ghost layers on either side (the neighbouring
    layers of the whole grid, periodic).  Returns (local problem, start, count, indices of the global receivers it
    holds).  Receivers are kept on the real layers only; sources on the real layers and, for halo > 1, on the ghost
    layers too (the inner ghost layer's collisions then feed real layers)."""
    D = len(p.shape)
    assert not p.bc[D - 1], "the slab axis must be periodic (walls only on the axes along the cuts)"
    assert halo in (1, 2) and (halo == 1 or (D == 2 and p.wp2 is None)), \
        "a two-layer halo is for 2D media without a dispersive pole"
    n = p.shape[0]
    start, count = slab_range(n, world, rank)
    assert count >= halo, "each slab needs at least `halo` real layers"
    layers = np.arange(start - halo, start + count + halo) % n
    take = lambda a: None if a is None else np.take(a, layers, axis=0)
    site = lambda a: None if a is None else take(np.broadcast_to(a, p.shape))  # a per-site parameter or a scalar
    shape = (count + 2 * halo,) + tuple(p.shape[1:])
    per_layer = int(np.prod(p.shape[1:]))
    real = np.zeros(layers.size, bool)
    real[halo:halo + count] = True

    def localize(sites, ghosts):
        """(index of the global entry, local flat site) for every local layer position holding the entry's layer."""
        if sites.size == 0:
            return np.zeros(0, np.int64), np.zeros(0, np.int64)
        layer = sites // per_layer
        hit = (layer[:, None] == layers[None, :]) & (real | ghosts)[None, :]
        idx, pos = np.nonzero(hit)
        return idx, pos * per_layer + sites[idx] % per_layer

    q = replace(p, shape=shape, eps_r=take(p.eps_r), mu_r=take(p.mu_r), E0=take(p.E0), B0=take(p.B0),
                wp2=site(p.wp2), wr2=site(p.wr2), gamma=site(p.gamma))
    idx, loc = localize(p.src_site, halo > 1)
    q.src_site, q.src_comp, q.src_amp = loc.astype(np.int64), p.src_comp[idx], p.src_amp[idx]
    idx, loc = localize(p.rec_site, False)
    q.rec_site, q.rec_comp = loc.astype(np.int64), p.rec_comp[idx]
    return q, start, count, idx


class LbemSlab:
    """One slab on the current GPU, stepped by the library: one step per launch with halo = 1, two with halo = 2."""

    def __init__(self, q, count, stream=None, halo=1):
        import torch

        self.D = len(q.shape)
        self.count = count
        self.halo = halo
        self.rows_per_layer = 1 if self.D == 2 else q.shape[1]
        self.nx = q.shape[-1]
        self.s = lbem.Solver(q.shape, stream=stream)
        self.s.set_problem(q)
        lbem.lbem_set_temporal_blocking(self.s.h, halo, -1)
        self.torch = torch

    @property
    def steps_per_exchange(self):
        return self.halo

    def step(self, k=None):
        """Advance k steps (default: the steps between two exchanges)."""
        self.s.step(self.halo if k is None else k)

    def _rows(self, planes, layer, buf, to_state):
        r = self.rows_per_layer
        for k, pl in enumerate(planes):
            lbem.lbem_rows(self.s.h, pl, layer * r, r, buf[k], to_state)

    def halo_out(self, up):
        """What this slab sends across its upper (up) or lower cut, as one [rows][layer sites] tensor: in 2D the
        library's halo rows (lbem_halo_out: 1 row with halo 1, 5 with halo 2), in 3D the crossing planes."""
        if self.D == 2:
            buf = self.torch.empty((1 if self.halo == 1 else 5, self.nx), dtype=self.torch.float32, device="cuda")
            lbem.lbem_halo_out(self.s.h, self.halo, buf if up else None, None if up else buf)
            return buf
        planes = CROSSING[self.D][0 if up else 1]
        buf = self.torch.empty((len(planes), self.rows_per_layer * self.nx), dtype=self.torch.float32, device="cuda")
        self._rows(planes, self.count if up else 1, buf, False)
        return buf

    def halo_in(self, from_below, buf):
        """Write what the slab below (from_below) or above sent into the matching ghost layers."""
        buf = buf.to(device="cuda", dtype=self.torch.float32).contiguous()
        if self.D == 2:
            lbem.lbem_halo_in(self.s.h, self.halo, buf if from_below else None, None if from_below else buf)
            return
        planes = CROSSING[self.D][0 if from_below else 1]
        self._rows(planes, 0 if from_below else self.count + 1, buf, True)

    def fields(self):
        """E, B of the real layers, each (3,) + slab shape without ghosts (torch, on the GPU)."""
        E, B = self.s.fields()
        h = self.halo
        return E[:, h:self.count + h], B[:, h:self.count + h]

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


def _chunks(nsteps, every):
    """Steps between exchanges: `every` at a time, then the remainder."""
    out = [every] * (nsteps // every)
    if nsteps % every:
        out.append(nsteps % every)
    return out


def step_local(slabs, nsteps):
    """Advance slabs held by one process by nsteps steps, exchanging halos every slab.steps_per_exchange steps."""
    for k in _chunks(nsteps, getattr(slabs[0], "steps_per_exchange", 1)):
        for s in slabs:
            s.step(k)
        exchange_local(slabs)


def step_dist(slab, rank, world, nsteps, host=False):
    """Advance this rank's slab by nsteps steps, exchanging halos every slab.steps_per_exchange steps."""
    for k in _chunks(nsteps, getattr(slab, "steps_per_exchange", 1)):
        slab.step(k)
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
