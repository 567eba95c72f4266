"""Differentiable multiblob rollouts: torch.autograd over K ICM steps with checkpointing.

`rollout_particle_velocities(sim, q0, k_spring, ...)` runs K steps of one box from blob
positions q0 (fluid at rest) with spring stiffness k_spring and returns the particle velocities
U0 (Sec. 2: U0 = mean blob velocity) after the last step.  Its backward pass is the hand-written
adjoint of the step (mb_adjoint_step, mb_particle_velocity_adjoint): the state is checkpointed every
`checkpoint` steps in the forward pass, and each segment is recomputed from its checkpoint in
the backward pass, so memory holds at most `checkpoint` states at a time.

Gradients flow to q0 (every blob coordinate) and to k_spring.  Requires an FP64 context
(precision 1) with batch 1.  Marshalling only: all arithmetic runs in libmb.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Multiblob, adjoint_step, particle_velocity_adjoint, set_positions,
               set_velocity_field, step)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, q0, k_spring, sim, topo, K, checkpoint, ext, body):
        pid, bonds, rest, k_rep, r_cut = topo
        sim.set_particles(0, q0.detach(), pid, bonds, rest, float(k_spring), k_rep, r_cut)
        dev, dt = sim.device, sim.grid_dtype
        v0 = torch.zeros(sim.grid_shape(), dtype=dt, device=dev)
        set_velocity_field(sim.ctx, v0)
        chk = []
        for s in range(K):
            if s % checkpoint == 0:
                chk.append((sim.blob_positions().clone(), sim.velocity_field().clone()))
            step(sim.ctx, 1, ext, body)
        U, _ = sim.particle_velocities()
        fctx.sim, fctx.topo, fctx.K, fctx.checkpoint = sim, topo, K, checkpoint
        fctx.ext, fctx.body, fctx.chk = ext, body, chk
        fctx.qK = sim.blob_positions().clone()
        fctx.vK = sim.velocity_field().clone()
        return U.clone()

    @staticmethod
    def backward(fctx, gU):
        sim = fctx.sim
        gq = torch.zeros_like(fctx.qK)
        gv = torch.zeros_like(fctx.vK)
        particle_velocity_adjoint(sim.ctx, fctx.qK, fctx.vK,
                                  gU.to(dtype=torch.float64, device=sim.device).contiguous(),
                                  gq, gv)
        gk = np.zeros(1, dtype=np.float64)
        K, chk_every = fctx.K, fctx.checkpoint
        for seg in reversed(range(len(fctx.chk))):
            q_s, v_s = fctx.chk[seg]
            set_positions(sim.ctx, q_s)
            set_velocity_field(sim.ctx, v_s)
            n_seg = min(chk_every, K - seg * chk_every)
            states = []
            for _ in range(n_seg):
                states.append((sim.blob_positions().clone(), sim.velocity_field().clone()))
                step(sim.ctx, 1, fctx.ext, fctx.body)
            for qn, vn in reversed(states):
                adjoint_step(sim.ctx, qn, vn, fctx.ext, fctx.body, gq, gv, gk)
        gk_t = torch.tensor(gk[0], dtype=torch.float64, device=sim.device)
        return gq, gk_t, None, None, None, None, None, None


def rollout_particle_velocities(sim: Multiblob, q0: torch.Tensor, k_spring: torch.Tensor,
                                particle_id, bonds, rest_len, K: int, checkpoint: int = 10,
                                ext_blob_force=None, body_force=None, k_rep: float = 0.0,
                                r_cut: float = 0.0) -> torch.Tensor:
    """U0 [n_particles, 3] after K steps from positions q0 (FP64 CUDA tensor [n, 3])."""
    if sim.desc.precision != 1 or sim.desc.batch != 1:
        raise ValueError("differentiable rollouts need an FP64 context with batch 1")
    ext = None
    if ext_blob_force is not None:
        ext = torch.as_tensor(ext_blob_force, dtype=torch.float64, device=sim.device).contiguous()
    topo = (np.asarray(particle_id, dtype=np.int32), np.asarray(bonds, dtype=np.int32).reshape(-1, 2),
            np.asarray(rest_len, dtype=np.float64), float(k_rep), float(r_cut))
    return _Rollout.apply(q0, k_spring, sim, topo, int(K), int(checkpoint), ext, body_force)
