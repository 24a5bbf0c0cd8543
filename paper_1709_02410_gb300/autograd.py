"""torch.autograd.Function around the wall-RPY matvec (FP64).

forward:  U = M(r) F                      (rpbd_mobility_apply)
backward: dL/dr = d(G^T M(r) F)/dr        (rpbd_mobility_adjoint, G = dL/dU)
          dL/dF = M(r)^T G = M(r) G       (M is symmetric)
Both derivatives run in the CUDA library.
"""
import torch


class MobilityApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, F, handle):
        ctx.handle = handle
        ctx.save_for_backward(r, F)
        return handle.mobility_apply(r.contiguous(), F.contiguous())

    @staticmethod
    def backward(ctx, G):
        r, F = ctx.saved_tensors
        h = ctx.handle
        G = G.contiguous()
        gr = gF = None
        if ctx.needs_input_grad[0]:
            if F.dim() == 2:
                gr = h.mobility_adjoint(r, G, F)
            else:  # k right-hand sides: sum of the per-RHS adjoints
                gr = torch.zeros_like(r)
                for m in range(F.shape[0]):
                    gr += h.mobility_adjoint(r, G[m].contiguous(), F[m].contiguous())
        if ctx.needs_input_grad[1]:
            gF = h.mobility_apply(r, G)
        return gr, gF, None


def mobility_apply(handle, r, F):
    """Differentiable U = M(r) F (float64 tensors on the handle's device)."""
    return MobilityApply.apply(r, F, handle)
