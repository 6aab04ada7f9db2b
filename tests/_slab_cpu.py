"""A CPU stand-in for one lattice (or one z-slab of it) under the in-place AA
pattern, for testing the halo exchange schedule (paper_2605_14505_gb300.halo)
without a GPU: populations f[q][z][y][x] in FP64, the library's velocity set
and slot order, and a local nonlinear map in place of the collision (the
exchange only moves slots, so any node-local map tests it). Even step: node x
reads slot i at x and writes slot opp(i) at x. Odd step: reads slot opp(i) at
x - e_i, writes slot i at x + e_i. Periodic in x and y; in z periodic for a
whole lattice, through the ghost planes 0 and nz - 1 for a slab. The halo
buffers follow the contract of lbm_halo_pack / lbm_halo_unpack."""
import numpy as np
import torch

from paper_2605_14505_gb300 import lbm


def collide(vals, w):
    """Node-local nonlinear map of the q values of every node (q, ...):
    relaxation towards w_i times the node's sum plus a quadratic coupling of
    neighbouring slots."""
    total = vals.sum(axis=0)
    out = vals + 0.3 * (w.reshape((-1,) + (1,) * (vals.ndim - 1)) * total - vals)
    return out + 0.01 * vals * np.roll(vals, 1, axis=0)


class NumpyAA:
    def __init__(self, f, q=19, slab=False):
        self.e, self.w, _ = lbm.lbm_velocity_set(q)
        self.q = q
        self.opp = np.array([[tuple(-v) for v in self.e].index(tuple(v)) for v in self.e])
        self.f = np.array(f, dtype=np.float64)            # (q, nz, ny, nx)
        self.slab = slab
        self.odd = 0
        nz, ny, nx = self.f.shape[1:]
        self.plane = ny * nx
        self.up = [i for i in range(q) if self.e[i][2] == 1]
        self.dn = [i for i in range(q) if self.e[i][2] == -1]
        self.halo_bytes = len(self.up) * self.plane * 8

    # -- one AA step
    def _planes(self):
        nz = self.f.shape[1]
        return (1, nz - 1) if self.slab else (0, nz)

    def _src(self, z, dz):
        nz = self.f.shape[1]
        return z + dz if self.slab else (z + dz) % nz

    def step(self):
        z0, z1 = self._planes()
        zs = np.arange(z0, z1)
        f = self.f
        if not self.odd:
            vals = f[:, z0:z1]
            out = collide(vals, self.w)
            f[self.opp, z0:z1] = out
        else:
            vals = np.empty((self.q, z1 - z0) + f.shape[2:])
            for i in range(self.q):
                ex, ey, ez = self.e[i]
                j = self.opp[i]
                # slot opp(i) at x - e_i
                rolled = np.roll(f[j], shift=(ey, ex), axis=(1, 2))
                vals[i] = rolled[self._src(zs, -ez)]
            out = collide(vals, self.w)
            for i in range(self.q):
                ex, ey, ez = self.e[i]
                # slot i at x + e_i
                f[i, self._src(zs, ez)] = np.roll(out[i], shift=(ey, ex), axis=(1, 2))
        self.odd ^= 1

    # -- halo contract
    def new_buffer(self):
        return torch.zeros(self.halo_bytes, dtype=torch.uint8)

    def _copy(self, z, slots, buf, pack):
        b = buf.numpy().view(np.float64).reshape(len(slots), *self.f.shape[2:])
        if pack:
            b[...] = self.f[slots, z]
        else:
            self.f[slots, z] = b

    def pack(self, phase, to_lower, to_upper):
        top = self.f.shape[1] - 1
        if phase == 0:
            self._copy(1, self.up, to_lower, True)
            self._copy(top - 1, self.dn, to_upper, True)
        else:
            self._copy(0, self.dn, to_lower, True)
            self._copy(top, self.up, to_upper, True)

    def unpack(self, phase, from_lower, from_upper):
        top = self.f.shape[1] - 1
        if phase == 0:
            self._copy(0, self.dn, from_lower, False)
            self._copy(top, self.up, from_upper, False)
        else:
            self._copy(1, self.up, from_lower, False)
            self._copy(top - 1, self.dn, from_upper, False)

    def synchronize(self):
        pass


def slabs_of(f, nranks):
    """Split a whole lattice's populations (q, nz, ny, nx) into nranks slabs
    with their ghost planes (planes z_r - 1 .. z_r + nz_r, periodic)."""
    nz = f.shape[1]
    bounds = np.linspace(0, nz, nranks + 1).astype(int)
    out = []
    for r in range(nranks):
        zs = np.arange(bounds[r] - 1, bounds[r + 1] + 1) % nz
        out.append((bounds[r], bounds[r + 1], f[:, zs].copy()))
    return out
