"""torch.autograd.Function over the library's time step and its adjoint.

``GaugeSeries.apply(h, eta0, u0, w0, tank, dt, nsteps, gauges, every)`` runs
``nsteps`` steps of ``tank`` (a 2D ``Tank``) from the state (eta0, u0, w0)
over bathymetry h and returns the surface elevation after every step at the
gauge node indices, shape (nsteps, len(gauges)).  Its backward pass gives
the gradients with respect to h and the initial state: the forward pass
keeps the state every ``every`` steps (checkpoints); the backward pass
recomputes each segment's step-start states from its checkpoint with
``wt_step`` and reverses the steps with ``wt_adjoint_step``, which
recomputes the step's stages and runs their adjoint (the transposed pressure
problem solved by the same p-multigrid).  Every step of the computation runs
in the CUDA library; this module only moves tensors between calls.

All tensors are float64 on the tank's CUDA device: h (Nx,), eta0 (Nx,),
u0 and w0 (Nz+1, Nx).
"""

import torch

from . import wt_get_state


def _state(tank):
    Nx, M1 = tank.Nx, tank.M1
    dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.empty((1, Nx), dtype=torch.float64, device=dev)
    u = torch.empty((M1, 1, Nx), dtype=torch.float64, device=dev)
    v = torch.empty_like(u)
    w = torch.empty_like(u)
    return e, u, v, w


def _read(tank, bufs):
    e, u, v, w = bufs
    st, _ = wt_get_state(tank.handle, e, u, v, w)
    if st != 0:
        from . import _check
        _check(st)
    return e.clone(), u.clone(), w.clone()


class GaugeSeries(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, eta0, u0, w0, tank, dt, nsteps, gauges, every):
        if tank.Ny != 1:
            raise ValueError("GaugeSeries needs a 2D tank")
        Nx, M1 = tank.Nx, tank.M1
        gauges = torch.as_tensor(gauges, dtype=torch.long, device=h.device)
        hh = h.detach().reshape(1, Nx).contiguous()
        tank.set_bathymetry(hh)
        e = eta0.detach().reshape(1, Nx).contiguous().clone()
        u = u0.detach().reshape(M1, 1, Nx).contiguous().clone()
        w = w0.detach().reshape(M1, 1, Nx).contiguous().clone()
        tank.set_state(e, u, torch.zeros_like(u), w)
        ckpts = [(e, u, w)]
        bufs = _state(tank)
        out = torch.empty((nsteps, len(gauges)), dtype=torch.float64, device=h.device)
        for n in range(nsteps):
            tank.step(dt, 1)
            s = _read(tank, bufs)
            out[n] = s[0][0, gauges]
            if (n + 1) % every == 0 and n + 1 < nsteps:
                ckpts.append(s)
        ctx.tank, ctx.dt, ctx.nsteps, ctx.every = tank, dt, nsteps, every
        ctx.gauges, ctx.ckpts, ctx.hh = gauges, ckpts, hh
        ctx.shapes = (h.shape, eta0.shape, u0.shape, w0.shape)
        return out

    @staticmethod
    def backward(ctx, gout):
        tank, dt, every = ctx.tank, ctx.dt, ctx.every
        Nx, M1 = tank.Nx, tank.M1
        dev = gout.device
        tank.set_bathymetry(ctx.hh)
        le = torch.zeros((1, Nx), dtype=torch.float64, device=dev)
        lu = torch.zeros((M1, 1, Nx), dtype=torch.float64, device=dev)
        lw = torch.zeros_like(lu)
        dh = torch.zeros((1, Nx), dtype=torch.float64, device=dev)
        bufs = _state(tank)
        g = gout.detach().contiguous()
        for s in reversed(range(len(ctx.ckpts))):
            n0 = s * every
            n1 = min(ctx.nsteps, n0 + every)
            states = [ctx.ckpts[s]]
            e, u, w = ctx.ckpts[s]
            tank.set_state(e, u, torch.zeros_like(u), w)
            for _ in range(n0, n1 - 1):
                tank.step(dt, 1)
                states.append(_read(tank, bufs))
            for n in reversed(range(n0, n1)):
                le[0, ctx.gauges] += g[n]
                e, u, w = states[n - n0]
                tank.adjoint_step(dt, e, u, w, le, lu, lw, dh)
        hs, es, us, ws = ctx.shapes
        return (dh.reshape(hs), le.reshape(es), lu.reshape(us), lw.reshape(ws),
                None, None, None, None, None)


def gauge_series(tank, h, eta0, u0, w0, dt, nsteps, gauges, every=20):
    """Differentiable gauge series (see GaugeSeries)."""
    return GaugeSeries.apply(h, eta0, u0, w0, tank, dt, nsteps, gauges, every)
