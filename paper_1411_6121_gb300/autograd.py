"""``torch.autograd.Function`` over a checkpointed DUGKS rollout.

The forward pass runs ``nsteps`` steps of a D2Q9 simulation through ``dugks_record``
(checkpoint every ``every`` steps) and returns the final moments; the backward pass calls
``dugks_adjoint``, the library's hand-written transposed step, for the gradients with
respect to the per-cell acceleration field, the wall velocities and the initial state.
Argument marshalling only: every step and every transposed step runs in the CUDA library.
"""
import torch

from . import dugks as _d


def _sync(dev):
    # the library works on the handle's own stream: order it after torch's producers
    torch.cuda.current_stream(dev).synchronize()


class DugksRollout(torch.autograd.Function):
    """``moments(T) = DugksRollout.apply(field, wall_u, sim, state0, nsteps, every, t0)``

    field   CUDA float32 [2][ncell]: acceleration field G(x) (added to the uniform g of sim)
    wall_u  float64 [6][3]: wall velocities per face (read for velocity walls only)
    sim     ``dugks.Sim`` (D2Q9, F32 or F64 storage) whose handle runs the rollout
    state0  CUDA [Q][ncell] initial deviation state of the storage dtype, or None to start
            from the handle's current state
    nsteps, every, t0   rollout length, checkpoint interval, start step (clock)
    Returns the final moments [3][ncell] float32 (p, u_x, u_y).
    """

    @staticmethod
    def forward(ctx, field, wall_u, sim, state0, nsteps, every, t0):
        dev = field.device
        _sync(dev)
        bcs = []
        for w in range(6):
            f = sim.bcs.face[w]
            bcs.append((int(f.type), tuple(float(x) for x in wall_u[w].tolist()), float(f.p)))
        sim.set_boundaries(bcs)
        sim.set_force_field(field.detach().contiguous())
        if state0 is not None:
            sim.set_state(state0.detach().contiguous())
        sim.set_clock(int(t0))
        sim.record(int(nsteps), int(every))
        out = torch.empty((sim.dim + 1, sim.ncell), dtype=torch.float32, device=dev)
        sim.moments(out)
        ctx.sim = sim
        ctx.wall_meta = (wall_u.dtype, wall_u.device)
        return out

    @staticmethod
    def backward(ctx, grad):
        need_f, need_w, _, need_s = ctx.needs_input_grad[:4]
        g = grad.detach().contiguous().float()
        _sync(g.device)
        dfield, dwall, dstate = ctx.sim.adjoint(g, field_grad=True, state_grad=bool(need_s))
        gw = torch.from_numpy(dwall).to(dtype=ctx.wall_meta[0], device=ctx.wall_meta[1]) if need_w else None
        return (dfield if need_f else None), gw, None, dstate, None, None, None


def rollout(sim, field, wall_u, nsteps, every=100, state0=None, t0=0):
    """Differentiable final moments of ``nsteps`` steps (see ``DugksRollout``)."""
    return DugksRollout.apply(field, wall_u, sim, state0, nsteps, every, t0)
