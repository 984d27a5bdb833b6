"""Differentiable runs of the charge-conserving PIC step.

A run loads one species from positions x0 and momenta w0 (float64, shape
(3, n)), advances `steps` full steps from zero fields, and returns the field
energy in a window of the final state,

    L = V/(8 pi) sum_{window} (|E^N|^2 + |B^N|^2),  B^N = B^{N-1/2} - (1/2) c curl_h E^N,

over the staggered points whose integer indices lie in the window.  Its gradient
with respect to x0 and w0 comes from libpic's discrete adjoint
(pic_adjoint_step): the forward run keeps a state snapshot every
`checkpoint_every` steps; the backward pass restores each checkpoint in reverse
order, recomputes that segment keeping one device snapshot per step
(pic_step_saving), and runs the adjoint steps back through it
(pic_adjoint_steps), with one host synchronization per segment.  Everything numerical runs in libpic; torch
only holds device buffers and the window mask, and chains the gradient to the
caller's parameters (e.g. a density-perturbation amplitude) through
torch.autograd.
"""
import math

import torch

from . import pic as P


class DifferentiableRun:
    def __init__(self, desc, q, m, weight, steps, window, checkpoint_every=20):
        self.grid = P.Grid(desc)
        self.q, self.m, self.weight = q, m, weight
        self.steps = int(steps)
        self.window = window            # ((x0, x1), (y0, y1)[, (z0, z1)]) in cell indices, half-open
        self.ce = int(checkpoint_every)
        self.dims = desc.dims
        self.dtype = torch.float64 if desc.precision == P.PIC_FP64 else torch.float32
        self.shape = self.grid.shape
        self.V = desc.dx * desc.dy * (desc.dz if desc.dims == 3 else 1.0)
        self.n = 0
        self.checkpoints = {}
        self.lamE = self.lamB = None
        mask = torch.zeros(self.shape, dtype=self.dtype, device="cuda")
        (x0, x1), (y0, y1) = window[0], window[1]
        if self.dims == 3:
            z0, z1 = window[2]
            mask[z0:z1, y0:y1, x0:x1] = 1
        else:
            mask[:, y0:y1, x0:x1] = 1
        self.mask = mask

    # ---- helpers -----------------------------------------------------------------
    def snapshot(self):
        buf = torch.empty(P.pic_state_bytes(self.grid.h), dtype=torch.uint8, device="cuda")
        P.pic_state_save(self.grid.h, buf)
        return buf

    def restore(self, buf):
        P.pic_state_restore(self.grid.h, buf)

    def fields(self):
        E = [torch.empty(self.shape, dtype=self.dtype, device="cuda") for _ in range(3)]
        B = [torch.empty(self.shape, dtype=self.dtype, device="cuda") for _ in range(3)]
        torch.cuda.synchronize()
        P.pic_get_fields(self.grid.h, E, B)
        torch.cuda.synchronize()
        return E, B

    def load(self, x0, w0):
        x0 = x0.detach().to(device="cuda", dtype=torch.float64).contiguous()
        w0 = w0.detach().to(device="cuda", dtype=torch.float64).contiguous()
        self.n = x0.shape[1]
        zero = [torch.zeros(self.shape, dtype=self.dtype, device="cuda") for _ in range(3)]
        torch.cuda.synchronize()
        P.pic_set_fields(self.grid.h, zero, [z.clone() for z in zero])
        P.pic_load_particles(self.grid.h, 0, self.q, self.m, self.weight, list(x0), list(w0))
        torch.cuda.synchronize()

    def loss_and_seeds(self):
        snap = self.snapshot()
        P.pic_yee_update(self.grid.h, P.PIC_B_HALF)
        E, Bn = self.fields()
        self.restore(snap)
        c8 = self.V / (8 * math.pi)
        L = c8 * sum(float((self.mask * (E[a] ** 2 + Bn[a] ** 2)).sum()) for a in range(3))
        lamE = [(2 * c8) * self.mask * E[a] for a in range(3)]
        lamB = [(2 * c8) * self.mask * Bn[a] for a in range(3)]
        torch.cuda.synchronize()
        P.pic_adjoint_yee_half_B(self.grid.h, lamB, lamE)
        torch.cuda.synchronize()
        return L, lamE, lamB

    # ---- forward and backward ---------------------------------------------------
    def forward(self, x0, w0):
        self.load(x0, w0)
        self.checkpoints = {}
        for s in range(0, self.steps, self.ce):   # one snapshot, then one call for the segment's steps
            self.checkpoints[s] = self.snapshot()
            P.pic_step(self.grid.h, min(self.ce, self.steps - s))
        P.pic_sync(self.grid.h)
        L, self.lamE, self.lamB = self.loss_and_seeds()
        return L

    def backward(self):
        lamE, lamB = self.lamE, self.lamB
        lamx = [torch.zeros(self.n, dtype=self.dtype, device="cuda") for _ in range(3)]
        lamw = [torch.zeros(self.n, dtype=self.dtype, device="cuda") for _ in range(3)]
        nbytes = P.pic_state_bytes(self.grid.h)
        bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(min(self.ce, self.steps))]
        torch.cuda.synchronize()
        for start in sorted(self.checkpoints, reverse=True):
            self.restore(self.checkpoints[start])
            states = bufs[:min(start + self.ce, self.steps) - start]
            # recompute the segment keeping the state of every level, then run
            # the adjoint back through it; both calls only enqueue work
            P.pic_step_saving(self.grid.h, states)
            P.pic_adjoint_steps(self.grid.h, states, lamE, lamB, lamx, lamw)
        P.pic_sync(self.grid.h)
        torch.cuda.synchronize()
        gx = torch.stack(lamx).to(torch.float64)
        if self.dims == 2:
            gx[2] = 0
        return gx, torch.stack(lamw).to(torch.float64)


class WindowEnergyLoss(torch.autograd.Function):
    """L(x0, w0) of a DifferentiableRun as a torch function with gradients."""

    @staticmethod
    def forward(ctx, x0, w0, run):
        ctx.run = run
        ctx.device = x0.device
        return torch.tensor(run.forward(x0, w0), dtype=torch.float64, device=x0.device)

    @staticmethod
    def backward(ctx, gL):
        gx, gw = ctx.run.backward()
        return (gL * gx).to(ctx.device), (gL * gw).to(ctx.device), None
