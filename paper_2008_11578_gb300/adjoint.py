"""Differentiable ORCA rollouts: ``torch.autograd.Function`` over liborca.

The forward pass is ``orca_rollout`` (n_steps ORCA steps that store the
state every ``ckpt_every`` steps); the backward pass is ``orca_adjoint``
(each segment is recomputed from its checkpoint with the LP active sets
recorded, then the hand-written adjoint kernel runs the steps in reverse).
Leaves: the preferred-velocity offsets ``vpref_delta`` [T, N, 2] and the
waypoint table [R, W, 2].  Outputs: positions after the last step [N, 2]
and the velocity after every step [T, N, 2].  torch supplies memory and
streams only; every step of the forward and reverse pass runs in liborca.
"""
from __future__ import annotations

from . import api


def _torch():
    import torch
    return torch


class Rollout:
    """A scene on the GPU plus the buffers of its differentiable rollouts.

    Every call starts from the scene's initial state (``scene.pos``,
    ``scene.vel``, ``scene.wp_idx``), so repeated calls are independent.
    """

    def __init__(self, scene, n_steps: int, ckpt_every: int = 8, device="cuda",
                 cell_size=None):
        torch = _torch()
        self.scene = scene
        self.ds = api.DeviceScene(scene, device, cell_size=cell_size)
        self.n_steps = int(n_steps)
        self.ckpt_every = int(ckpt_every)
        self.n = scene.n
        self._init = (self.ds.pos.clone(), self.ds.vel.clone(),
                      None if self.ds.wp_idx is None else self.ds.wp_idx.clone())
        self.ws_bytes = api.orca_adjoint_workspace_bytes(self.ds.handle, self.n_steps,
                                                         self.ckpt_every)
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.ds.device)
        self.vel_traj = torch.empty((self.n_steps, self.n, 2), dtype=torch.float32,
                                    device=self.ds.device)
        self.generation = 0

    def reset(self):
        pos, vel, wp = self._init
        self.ds.pos.copy_(pos)
        self.ds.vel.copy_(vel)
        if wp is not None:
            self.ds.wp_idx.copy_(wp)

    def forward_raw(self, vpref_delta):
        """The checkpointing forward alone (no autograd bookkeeping)."""
        self.reset()
        api.orca_rollout(self.ds.handle, self.n_steps, self.ckpt_every, vpref_delta, self.ws,
                         self.ws_bytes, self.vel_traj)
        self.generation += 1

    def backward_raw(self, vpref_delta, dl_dpos, dl_dvel_traj=None, want_waypoints=True,
                     want_state0=False):
        """Gradients after forward_raw with the same vpref_delta."""
        torch = _torch()
        dev = self.ds.device
        dvpd = torch.empty((self.n_steps, self.n, 2), dtype=torch.float32, device=dev)
        dwp = None
        if want_waypoints and self.ds.waypoints is not None:
            dwp = torch.empty_like(self.ds.waypoints)
        dp0 = dv0 = None
        if want_state0:
            dp0 = torch.empty((self.n, 2), dtype=torch.float32, device=dev)
            dv0 = torch.empty((self.n, 2), dtype=torch.float32, device=dev)
        api.orca_adjoint(self.ds.handle, self.n_steps, self.ckpt_every, vpref_delta, self.ws,
                         self.ws_bytes, dl_dpos.contiguous(),
                         None if dl_dvel_traj is None else dl_dvel_traj.contiguous(), dvpd,
                         dwp, dp0, dv0)
        return dvpd, dwp, dp0, dv0

    def __call__(self, vpref_delta, waypoints=None):
        return _RolloutFn.apply(vpref_delta, waypoints, self)

    def close(self):
        self.ds.close()


def _rollout_fn():
    torch = _torch()

    class RolloutFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vpref_delta, waypoints, roll):
            if waypoints is not None:
                if roll.ds.waypoints is None:
                    raise ValueError("this scene has no waypoint routes")
                roll.ds.waypoints.copy_(waypoints.detach().reshape(-1, 2))
            vpd = vpref_delta.detach().to(torch.float32).contiguous()
            roll.forward_raw(vpd)
            ctx.roll = roll
            ctx.vpd = vpd
            ctx.gen = roll.generation
            ctx.wp_shape = None if waypoints is None else waypoints.shape
            return roll.ds.pos.clone(), roll.vel_traj.clone()

        @staticmethod
        def backward(ctx, gpos, gvel):
            roll = ctx.roll
            if roll.generation != ctx.gen:
                raise RuntimeError("the rollout ran again since this forward pass; its "
                                   "checkpoints are gone (use one Rollout per graph)")
            if gpos is None:
                gpos = torch.zeros((roll.n, 2), dtype=torch.float32, device=roll.ds.device)
            dvpd, dwp, _, _ = roll.backward_raw(ctx.vpd, gpos, gvel,
                                                want_waypoints=ctx.wp_shape is not None)
            return dvpd, None if dwp is None else dwp.view(ctx.wp_shape), None

    return RolloutFn


class _Lazy:
    fn = None


def _apply(*args):
    if _Lazy.fn is None:
        _Lazy.fn = _rollout_fn()
    return _Lazy.fn.apply(*args)


class _RolloutFn:
    apply = staticmethod(_apply)


def workload_loss(pos_T, vel_traj, goal, is_vehicle, target_speed=5.0, weight=0.1):
    """Mean squared distance to the goal after the last step, plus ``weight``
    times the summed squared deviation of every vehicle's speed from
    ``target_speed`` over all steps (the adjoint benchmark's loss)."""
    torch = _torch()
    term = ((pos_T - goal) ** 2).sum(-1).mean()
    sp = torch.sqrt((vel_traj[:, is_vehicle] ** 2).sum(-1).clamp_min(1e-30))
    return term + weight * ((sp - target_speed) ** 2).sum()
