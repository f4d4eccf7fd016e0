"""torch.autograd wrapper of the collision operator.

Q^(pq)(f_p, f_q) is bilinear in (f_p, f_q) (Eq. 7), so its adjoint is exact:
the backward pass calls dgfs_collide_backward, which recomputes the per-(rho,
sigma) translates instead of storing them and also returns dL/d omega_pq
through beta^(pq)(omega) and the radial weights rho^{gamma+2}, gamma = 2(1 - omega).

The backward runs on the forward's own plan by default: the tensor-core forms
have their own adjoint (the (rho, sigma) loop on the tensor cores in the
plan's operand format, the parts outside it in FP64).  backward="fp64" builds
a second, FP64 plan with the same parameters instead and promotes f and dQ to
double for it.  All arithmetic runs in the CUDA library; this module only
orchestrates calls.
"""
import torch

from . import binding as B


class CollisionOperator:
    """Owns a forward plan (any precision) and the plan that runs its adjoint:
    the same plan (backward="native") or an FP64 one (backward="fp64")."""

    def __init__(self, N, L, M, N_rho, masses, pairs, precision="fp64", max_points=1, device=0,
                 backward="native"):
        if backward not in ("native", "fp64"):
            raise ValueError("backward must be 'native' or 'fp64'")
        self.args = (N, L, M, N_rho, list(masses), [dict(p) for p in pairs])
        self.S = len(masses)
        self.fwd = B.Plan(N, L, M, N_rho, masses, pairs, precision, max_points, device)
        if precision == "fp64" or backward == "native":
            self.bwd = self.fwd
        else:
            self.bwd = B.Plan(N, L, M, N_rho, masses, pairs, "fp64", max_points, device)
        self.omega = torch.tensor([p["omega"] for p in pairs], dtype=torch.float64,
                                  device="cuda").view(self.S, self.S)

    def __call__(self, f, omega=None):
        """Q = collide(f); omega (an [S, S] tensor equal to the plan's values) may be
        passed with requires_grad to receive dL/d omega."""
        if omega is None:
            omega = self.omega
        elif tuple(omega.shape) != (self.S, self.S) or not torch.equal(
                omega.detach().to(self.omega.device, torch.float64), self.omega):
            # the plans' tables are built for fixed omega: a different value would
            # give Q at the plan's omega and a gradient that looks valid
            raise ValueError("omega must equal the plan's VHS/VSS exponents %s; build a new "
                             "CollisionOperator for other values" % self.omega.cpu().tolist())
        return _Collide.apply(f, omega, self)


class _Collide(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, omega, op):
        ctx.op = op
        ctx.save_for_backward(f)
        return op.fwd.collide(f.contiguous())

    @staticmethod
    def backward(ctx, dQ):
        (f,) = ctx.saved_tensors
        op = ctx.op
        dt = op.bwd.dtype
        df, dom = op.bwd.backward(f.contiguous().to(dt), dQ.contiguous().to(dt))
        return df.to(f.dtype), dom.view(op.S, op.S), None
