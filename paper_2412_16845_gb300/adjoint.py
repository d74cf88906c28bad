"""Gradient of the probe objective with respect to per-cell eps, by the hand-written adjoint of
the GKS step (C ABI: gks_set_objective, gks_adjoint_seed, gks_adjoint_step), with sqrt(N)-step
checkpointing and recomputation, and a ``torch.autograd.Function`` on top.

J(eps) = sum_{n=1}^{N} dt sum_{i in probe} |Omega_i| Ez_i^n(eps)^2 for a 2-D TM workload with a
design region.  The forward pass stores the state every K steps (device tensors in the
library's layout); the backward pass walks the segments in reverse: restore the checkpoint,
recompute the segment's states, then run the adjoint steps over them.  PyTorch provides the
device buffers and the stream; every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from .gks import (GKSSolver, gks_adjoint_seed, gks_adjoint_step, gks_copy_state,
                  gks_copy_state_box, gks_load_state, gks_objective, gks_reset_objective,
                  gks_set_materials_box, gks_set_objective, gks_state_layout, gks_step_window)


def design_box(design, nx):
    """Bounding box (x0, x1, y0, y1) of the design cells on an nx-wide grid, the position of each
    design cell in the box's row-major order, and the grid index of every box cell."""
    design = np.asarray(design, dtype=np.int64)
    dx, dy = design % nx, design // nx
    box = (int(dx.min()), int(dx.max()) + 1, int(dy.min()), int(dy.max()) + 1)
    index = (dy - box[2]) * (box[1] - box[0]) + (dx - box[0])
    ys, xs = np.mgrid[box[2]:box[3], box[0]:box[1]]
    return box, index, (ys * nx + xs).ravel()


class DesignProblem:
    def __init__(self, w, precision="fp32", nsteps=None, checkpoint_every=None, stream=None):
        import torch
        if w.dim != 2 or w.design is None or w.probe is None:
            raise ValueError("a 2-D workload with a probe and a design region is required")
        self.torch = torch
        self.w = w
        self.N = int(nsteps if nsteps is not None else w.steps)
        self.K = int(checkpoint_every or max(1, int(round(math.sqrt(self.N)))))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.base_eps = np.array(w.eps, dtype=np.float64)
        self.design = np.asarray(w.design, dtype=np.int64)
        mu = np.ones_like(self.base_eps) if w.mu is None else np.asarray(w.mu, dtype=np.float64)
        # J is differentiated at a fixed lattice speed c (the adjoint holds dt and C1..C5
        # constant): c is the workload's, else the fastest light speed of its eps and mu.
        self.c = float(getattr(w, "c_lattice", 0.0) or np.max(1.0 / np.sqrt(self.base_eps * mu)))
        self.mu_design = mu[self.design]
        self.solver = GKSSolver.from_workload(w, precision=precision,
                                              stream=self.stream.cuda_stream, c_lattice=self.c)
        self.ctx = self.solver.ctx
        gks_set_objective(self.ctx, w.probe, w.design)
        self.elems, _ = gks_state_layout(self.ctx)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        # V^0 stays on the device; each forward() restarts from it
        self.init = self._buf()
        gks_copy_state(self.ctx, self.init.data_ptr())
        # a design update rewrites eps only on the design's bounding box
        self.dbox, self.dbox_index, cells = design_box(self.design, w.n[0])
        self.dbox_eps = self.base_eps[cells]
        self.checkpoints = None
        self.final = None
        self.eps_design = None
        # the adjoint reads states only on the design cells and their two-cell stencil and on
        # the probe: that box (cbox) is what is stored of a recomputed state.  Step m of a
        # segment of k steps is recomputed on cbox widened by 2 (k - m) cells, its domain of
        # dependence, so the window shrinks by the stencil radius every step.
        nx, ny = w.n
        self.nx, self.ny = nx, ny
        self.per = (w.bc[0] == "periodic", w.bc[2] == "periodic")
        cells = np.concatenate([self.design, np.asarray(w.probe, dtype=np.int64)])
        xs, ys = cells % nx, cells // nx
        self.cbox = (max(0, int(xs.min()) - 2), min(nx, int(xs.max()) + 3),
                     max(0, int(ys.min()) - 2), min(ny, int(ys.max()) + 3))

    def _window(self, r):
        """cbox widened by r cells, clipped to the grid (a whole periodic axis once it wraps)."""
        x0, x1, y0, y1 = self.cbox
        x0, x1, y0, y1 = x0 - r, x1 + r, y0 - r, y1 + r
        if x0 < 0 or x1 > self.nx:
            x0, x1 = (0, self.nx) if self.per[0] else (max(0, x0), min(self.nx, x1))
        if y0 < 0 or y1 > self.ny:
            y0, y1 = (0, self.ny) if self.per[1] else (max(0, y0), min(self.ny, y1))
        return x0, x1, y0, y1

    def _buf(self):
        return self.torch.empty(self.elems, dtype=self.dtype, device="cuda")

    def set_design(self, eps_design):
        e = np.array(eps_design, dtype=np.float64).reshape(-1)
        if e.size != self.design.size:
            raise ValueError("eps_design needs one value per design cell")
        if not np.all(np.isfinite(e) & (e > 0)):
            raise ValueError("eps_design must be finite and > 0")
        if np.any(1.0 / np.sqrt(e * self.mu_design) > self.c * (1 + 1e-12)):
            raise ValueError(f"eps_design puts a light speed above the lattice speed c = {self.c}")
        box = self.dbox_eps.copy()
        box[self.dbox_index] = e
        gks_set_materials_box(self.ctx, *self.dbox, box)
        self.eps_design = e

    def forward(self, eps_design, keep_checkpoints=True):
        """J(eps_design); keeps the checkpoints for a following backward()."""
        self.set_design(eps_design)
        gks_load_state(self.ctx, self.init.data_ptr(), 0)
        gks_reset_objective(self.ctx)
        ck = []
        n = 0
        while n < self.N:
            if keep_checkpoints:
                b = self._buf()
                gks_copy_state(self.ctx, b.data_ptr())
                ck.append((n, b))
            k = min(self.K, self.N - n)
            self.solver.step(k)
            n += k
        J = gks_objective(self.ctx)
        if keep_checkpoints:
            self.final = self._buf()
            gks_copy_state(self.ctx, self.final.data_ptr())
            self.checkpoints = ck
        return J

    def backward(self):
        """dJ/d eps over the design cells (device float64 tensor), after forward()."""
        torch = self.torch
        if self.checkpoints is None:
            raise RuntimeError("forward() with keep_checkpoints=True must come first")
        lam = self._buf()
        lam2 = self._buf()
        grad = torch.zeros(self.design.size, dtype=torch.float64, device="cuda")
        gks_adjoint_seed(self.ctx, self.final.data_ptr(), lam.data_ptr())
        # the recomputed states of one segment live in K buffers reused by every segment
        # (addresses, windows and the box taken once, not per step)
        pool = [self._buf() for _ in range(self.K)]
        pool_ptr = [b.data_ptr() for b in pool]
        lam_ptr, lam2_ptr, grad_ptr = lam.data_ptr(), lam2.data_ptr(), grad.data_ptr()
        ctx, cbox = self.ctx, self.cbox
        for (s, ckb), e in zip(reversed(self.checkpoints),
                               reversed([c[0] for c in self.checkpoints[1:]] + [self.N])):
            k = e - s
            # recompute V^s .. V^e of this segment
            ck_ptr = ckb.data_ptr()
            gks_load_state(ctx, ck_ptr, s)
            ptrs = [ck_ptr] + pool_ptr[:k]
            for m in range(1, k + 1):
                gks_step_window(ctx, 1, *self._window(2 * (k - m)))
                gks_copy_state_box(ctx, ptrs[m], *cbox)
            for n in range(e - 1, s - 1, -1):
                gks_adjoint_step(ctx, ptrs[n - s], ptrs[n - s + 1], lam_ptr, lam2_ptr, grad_ptr,
                                 n >= 1)
                lam_ptr, lam2_ptr = lam2_ptr, lam_ptr
        del pool
        return grad

    def value_and_grad(self, eps_design):
        J = self.forward(eps_design)
        g = self.backward()
        return J, g.cpu().numpy()

    def close(self):
        self.solver.close()


def _autograd_class():
    import torch

    class GKSEnergyObjective(torch.autograd.Function):
        """J = GKSEnergyObjective.apply(eps_design, problem): the probe objective of a
        DesignProblem as a differentiable function of the design eps (float64 scalar)."""

        @staticmethod
        def forward(ctx, eps_design, problem):
            J = problem.forward(eps_design.detach().to("cpu", torch.float64).numpy())
            ctx.problem = problem
            ctx.dev = eps_design.device
            ctx.dt = eps_design.dtype
            return torch.tensor(J, dtype=torch.float64, device=eps_design.device)

        @staticmethod
        def backward(ctx, gJ):
            g = ctx.problem.backward()
            return (gJ * g).to(ctx.dev, ctx.dt), None

    return GKSEnergyObjective


_CLASS = None


def __getattr__(name):
    global _CLASS
    if name == "GKSEnergyObjective":
        if _CLASS is None:
            _CLASS = _autograd_class()
        return _CLASS
    raise AttributeError(name)
