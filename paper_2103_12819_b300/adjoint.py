"""The discrete adjoint behind torch.autograd: the time-integrated Poynting
flux through a z plane as a differentiable function of the per-cell eps_r
(FluxLoss) or of eps_r and the bias H0 (FluxLossBias).

    loss = FluxLoss.apply(eps_r, make_solver, kp, nsteps)
    loss.backward()          # eps_r.grad = d loss / d eps_r (the adjoint)
    loss = FluxLossBias.apply(eps_r, h0, make_solver, kp, nsteps)
    loss.backward()          # eps_r.grad and h0.grad

`make_solver(eps_r_numpy)` builds a fresh solver at the initial state with
those permittivities (a callable the caller owns, so sources, boundaries and
precision are the caller's); the forward pass runs the steps and the adjoint
together (mmx_flux_gradient), the backward pass only scales the stored
gradient."""
import torch


class FluxLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r, make_solver, kp, nsteps, checkpoint_every=None):
        solver = make_solver(eps_r.detach().to("cpu", torch.float64).numpy())
        try:
            loss, grad = solver.flux_gradient(kp, nsteps, checkpoint_every)
        finally:
            solver.close()
        ctx.save_for_backward(torch.from_numpy(grad).to(device=eps_r.device, dtype=eps_r.dtype))
        return eps_r.new_tensor(loss)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None


class FluxLossBias(torch.autograd.Function):
    """As FluxLoss, with the uniform bias H0 (3 components, A/m) as a second
    differentiable input: `make_solver(eps_r_numpy, h0_numpy)` builds the
    solver with both applied."""

    @staticmethod
    def forward(ctx, eps_r, h0, make_solver, kp, nsteps, checkpoint_every=None):
        solver = make_solver(eps_r.detach().to("cpu", torch.float64).numpy(),
                             h0.detach().to("cpu", torch.float64).numpy())
        try:
            loss, grad, gh0 = solver.flux_gradient(kp, nsteps, checkpoint_every, with_h0=True)
        finally:
            solver.close()
        ctx.save_for_backward(torch.from_numpy(grad).to(device=eps_r.device, dtype=eps_r.dtype),
                              torch.from_numpy(gh0).to(device=h0.device, dtype=h0.dtype))
        return eps_r.new_tensor(loss)

    @staticmethod
    def backward(ctx, g):
        grad, gh0 = ctx.saved_tensors
        return g * grad, g * gh0, None, None, None, None
