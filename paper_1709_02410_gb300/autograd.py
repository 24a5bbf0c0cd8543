"""torch.autograd.Function around the wall-RPY matvec (FP64).

forward:  U = M(r) F                      (rpbd_mobility_apply)
backward: dL/dr = d(sum_m G_m^T M(r) F_m)/dr  (rpbd_mobility_adjoint_multi, G = dL/dU)
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
            # one library call: for k right-hand sides the sum over them of
            # d(G_m^T M F_m)/dr is formed on the device
            gr = h.mobility_adjoint(r, G, F)
        if ctx.needs_input_grad[1]:
            gF = h.mobility_apply(r, G)
        return gr, gF, None


def mobility_apply(handle, r, F):
    """Differentiable U = M(r) F (float64 tensors on the handle's device)."""
    return MobilityApply.apply(r, F, handle)
