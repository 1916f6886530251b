"""Differentiable cell volumes and centroidal energy (torch.autograd), and Lloyd/CVT steps.

The forward pass builds the Voronoi cells with ``vt_build`` and returns the cell
volumes V_i and energies E_i = integral over the cell of |y - x_i|^2
(``vt_cells``, ``vt_moments``); the backward pass is the hand-written adjoint
``vt_backward``:

    dL/dx_k = sum_j (A_kj/|r_kj|)(g_k - g_j)(c_kj - x_k) + gE * 2 V_k (x_k - z_k),

g = dL/dV, A and c the facet area and centroid, r the separation, z the cell
centroid.  The energy term needs a weight gE that is the same for every cell
(true for L = sum_i E_i); other weights raise.  The paper has no backward pass;
the volume derivative follows from the bisector planes moving with the
particles, the energy derivative is the classical centroidal Voronoi result
(the facet terms cancel).
"""
from __future__ import annotations

import torch

from . import binding as vt


class VoronoiCells(torch.autograd.Function):
    """(volume [N], energy [N]) = VoronoiCells.apply(pos, box_lo, box_hi, periodic, precision)."""

    @staticmethod
    def forward(ctx, pos, box_lo, box_hi, periodic=True, precision="filter32"):
        h = vt.vt_build(pos.detach(), None, box_lo, box_hi, periodic, precision)
        vol = torch.empty(pos.shape[0], dtype=pos.dtype, device=pos.device)
        vt.vt_cells(h, vol)
        energy = torch.empty_like(vol)
        vt.vt_moments(h, None, energy)
        ctx.h = h
        return vol, energy

    @staticmethod
    def backward(ctx, g_vol, g_energy):
        h = ctx.h
        gE = 0.0
        if g_energy is not None:
            gE = float(g_energy.reshape(-1)[0])
            if not bool(torch.all(g_energy == gE)):
                raise NotImplementedError("the energy adjoint needs the same weight for every cell")
        if g_vol is not None:
            g_vol = g_vol.contiguous()
        out = torch.empty(h.N, 3, dtype=h.dtype, device=h.device)
        vt.vt_backward(h, g_vol, gE, out)
        return out, None, None, None, None


def cells(pos, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), periodic=True, precision="filter32"):
    """Differentiable (volume, energy) of every particle's cell."""
    return VoronoiCells.apply(pos, box_lo, box_hi, periodic, precision)


def lloyd_step(pos, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), alpha=1.0, precision="filter32"):
    """One centroidal-Voronoi descent step x <- x - alpha * dE/dx / (2 V) (alpha = 1: Lloyd, x <- centroid),
    computed through autograd, wrapped into the periodic box.  Returns (new positions, total energy)."""
    x = pos.detach().clone().requires_grad_(True)
    vol, energy = cells(x, box_lo, box_hi, True, precision)
    E = energy.sum()
    (grad,) = torch.autograd.grad(E, x)
    with torch.no_grad():
        lo = torch.tensor(box_lo, dtype=pos.dtype, device=pos.device)
        hi = torch.tensor(box_hi, dtype=pos.dtype, device=pos.device)
        L = hi - lo
        step = alpha * grad / (2.0 * vol.detach()[:, None])
        y = torch.remainder(pos.detach() - step - lo, L) + lo
        y = torch.where(y >= hi, lo.expand_as(y), y)
    return y, float(E.detach())


class LloydRunner:
    """Repeated Lloyd steps on one handle: the tessellation of each new configuration goes through vt_rebuild
    (no allocation, no synchronisation), and with ``graph=True`` the whole step (rebuild, moments, position
    update) is captured once in a CUDA graph and replayed.  Positions stay on the device; ``step()`` returns
    the total centroidal energy of the configuration it started from (a device scalar; ``float()`` syncs)."""

    def __init__(self, pos, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), alpha=1.0, precision="filter32",
                 graph=False):
        self.stream = torch.cuda.Stream(device=pos.device)
        self.x = pos.detach().clone().contiguous()
        self.lo = torch.tensor(box_lo, dtype=pos.dtype, device=pos.device)
        self.hi = torch.tensor(box_hi, dtype=pos.dtype, device=pos.device)
        self.alpha = alpha
        n = self.x.shape[0]
        self.cen = torch.empty(n, 3, dtype=pos.dtype, device=pos.device)
        self.energy = torch.empty(n, dtype=pos.dtype, device=pos.device)
        self.E = torch.zeros((), dtype=torch.float64, device=pos.device)
        torch.cuda.synchronize(pos.device)
        with torch.cuda.stream(self.stream):
            self.h = vt.vt_build(self.x, None, box_lo, box_hi, True, precision, stream=self.stream)
            self._body()  # one untimed step outside any capture
        self.stream.synchronize()
        self.graph = None
        if graph:
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._body()

    def _body(self):
        # Lloyd: x <- centroid of its cell (alpha = 1); centroid = x + (z - x), wrapped into the box
        vt.vt_rebuild(self.h, self.x)
        vt.vt_moments(self.h, self.cen, self.energy)
        self.E.copy_(self.energy.sum(dtype=torch.float64))
        L = self.hi - self.lo
        d = torch.remainder(self.cen - self.x + 0.5 * L, L) - 0.5 * L  # minimum image of z - x
        y = torch.remainder(self.x + self.alpha * d - self.lo, L) + self.lo
        self.x.copy_(torch.where(y >= self.hi, self.lo.expand_as(y), y))

    def step(self):
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._body()
        torch.cuda.current_stream(self.x.device).wait_stream(self.stream)
        return self.E

    def status(self):
        return vt.vt_status(self.h)
