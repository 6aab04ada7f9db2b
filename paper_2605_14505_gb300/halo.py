"""z-slab decomposition of one periodic lattice: the halo exchange schedule.

A lattice of nx * ny * NZ nodes is split along z into slabs, one per rank;
each slab is a library handle in slab mode (lbm_set_slab) with one ghost plane
below and above its own planes. The even AA step is local to a node; the odd
step reads and writes the neighbouring planes' slots with e_z = +-1, so the
ranks exchange two halo buffers each way around every odd step: phase 0
before it (the boundary planes' slots into the neighbours' ghost planes),
phase 1 after it (what the odd step wrote into the ghost planes, back to the
planes that own it). The C header (lbm_set_slab, lbm_halo_pack,
lbm_halo_unpack) states which slots and planes each buffer holds.

The schedule is the same whatever moves the buffers:
  - SlabExchange: one rank per process, torch.distributed point-to-point
    (NCCL between GPUs, gloo on CPU);
  - LocalSlabs: every slab in one process, buffers copied directly (one GPU
    standing in for several ranks, or several GPUs driven by one process).
A backend holds one slab and offers: halo_bytes, new_buffer(), pack(phase,
to_lower, to_upper), unpack(phase, from_lower, from_upper), step() (one AA
step), synchronize(). LibrarySlab is the backend of the CUDA library.
"""
from __future__ import annotations


class LibrarySlab:
    """One slab of the CUDA library: a Simulation (already initialised with its
    own planes and the two neighbouring ones) switched to slab mode. The AA
    parity is the handle's step count since its initialisation (natural layout
    after an even count), so a slab may be wrapped after it has stepped."""

    def __init__(self, sim):
        import torch

        from . import lbm

        self._lbm = lbm
        self._torch = torch
        self.sim = sim
        lbm.lbm_set_slab(sim.h, True)
        self.halo_bytes = lbm.lbm_halo_bytes(sim.h)
        self.odd = lbm.lbm_step_count(sim.h) & 1

    def new_buffer(self):
        return self._torch.empty(self.halo_bytes, dtype=self._torch.uint8, device="cuda")

    def pack(self, phase, to_lower, to_upper):
        self._lbm.lbm_halo_pack(self.sim.h, phase, to_lower.data_ptr(), to_upper.data_ptr())

    def unpack(self, phase, from_lower, from_upper):
        self._lbm.lbm_halo_unpack(self.sim.h, phase, from_lower.data_ptr(), from_upper.data_ptr())

    def step(self):
        self._lbm.lbm_step(self.sim.h, 1)
        self.odd ^= 1

    def synchronize(self):
        self._lbm.lbm_synchronize(self.sim.h)


def _copy(dst, src):
    if hasattr(dst, "copy_"):
        dst.copy_(src)
    else:
        dst[...] = src


class LocalSlabs:
    """All slabs of the lattice in one process: slab r's lower neighbour is
    slab r - 1, its upper neighbour slab r + 1 (periodic)."""

    def __init__(self, backends):
        self.b = list(backends)
        self.buf = [{k: b.new_buffer() for k in ("to_lower", "to_upper", "from_lower", "from_upper")}
                    for b in self.b]

    def _exchange(self, phase):
        n = len(self.b)
        for b, bf in zip(self.b, self.buf):
            b.pack(phase, bf["to_lower"], bf["to_upper"])
        for b in self.b:
            b.synchronize()
        for r in range(n):
            _copy(self.buf[r]["from_lower"], self.buf[(r - 1) % n]["to_upper"])
            _copy(self.buf[r]["from_upper"], self.buf[(r + 1) % n]["to_lower"])
        for b, bf in zip(self.b, self.buf):
            b.unpack(phase, bf["from_lower"], bf["from_upper"])

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            odd = self.b[0].odd
            if odd:
                self._exchange(0)
            for b in self.b:
                b.step()
            if odd:
                self._exchange(1)
        for b in self.b:
            b.synchronize()

    def refresh_ghosts(self):
        """After an odd step count the store keeps a node's populations at
        neighbour locations, so reading the boundary planes (diagnostics,
        fields, populations) needs the neighbours' current slots in the ghost
        planes: the phase-0 exchange (repeated harmlessly by the next step)."""
        if self.b[0].odd:
            self._exchange(0)
        for b in self.b:
            b.synchronize()


class SlabExchange:
    """One rank's slab; its neighbours are ranks rank - 1 and rank + 1 of the
    process group (periodic). With one rank the slab is its own neighbour.
    Messages travel with tags (0: towards lower ranks, 1: towards higher) and
    in a fixed order, so that two ranks that are each other's lower and upper
    neighbour still match them."""

    def __init__(self, backend, rank: int, world: int, group=None):
        self.b = backend
        self.rank, self.world, self.group = rank, world, group
        self.to_lower, self.to_upper = backend.new_buffer(), backend.new_buffer()
        self.from_lower, self.from_upper = backend.new_buffer(), backend.new_buffer()

    def _exchange(self, phase):
        self.b.pack(phase, self.to_lower, self.to_upper)
        self.b.synchronize()
        if self.world == 1:
            _copy(self.from_lower, self.to_upper)
            _copy(self.from_upper, self.to_lower)
        else:
            import torch.distributed as dist

            lower = (self.rank - 1) % self.world
            upper = (self.rank + 1) % self.world
            ops = [dist.P2POp(dist.isend, self.to_lower, lower, self.group, 0),
                   dist.P2POp(dist.isend, self.to_upper, upper, self.group, 1),
                   dist.P2POp(dist.irecv, self.from_upper, upper, self.group, 0),
                   dist.P2POp(dist.irecv, self.from_lower, lower, self.group, 1)]
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        self.b.unpack(phase, self.from_lower, self.from_upper)

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            odd = self.b.odd
            if odd:
                self._exchange(0)
            self.b.step()
            if odd:
                self._exchange(1)
        self.b.synchronize()

    def refresh_ghosts(self):
        """As LocalSlabs.refresh_ghosts: the phase-0 exchange when the step
        count is odd, before reading the boundary planes."""
        if self.b.odd:
            self._exchange(0)
        self.b.synchronize()
