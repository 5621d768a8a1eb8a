"""torch.autograd binding of the projected-Hamiltonian application (FP64, GPU).

`heff(qn, left, right, f0, f1, f2, L, R, x, W1, W2)` returns y = H_eff(L, W1, W2, R) x computed by
the library's matvec, and its backward is the library's hand-written backward
(`dmrg_heff_backward`): gradients to x, L, R (device tensors in the packed layouts) and to the
two MPO tensors W1, W2 (dense host tensors; entries that are zero in the MPO get no gradient).
The forward intermediates are recomputed in the backward, not stored.
"""
import numpy as np
import torch

from . import Bond, FP64, heff_apply, heff_backward


class _Heff(torch.autograd.Function):
    @staticmethod
    def forward(ctx, static, L, R, x, W1, W2):
        qn, left, right, f0, f1, f2 = static
        for t in (L, R, x):
            if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("L, R, x must be contiguous float64 CUDA tensors")
        bond = Bond(qn, left, right, W1.detach().cpu().numpy(), f0, f1, W2.detach().cpu().numpy(), f2)
        y = torch.empty_like(x)
        torch.cuda.current_stream().synchronize()
        heff_apply(bond, FP64, L.data_ptr(), R.data_ptr(), x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        ctx.static = static
        ctx.save_for_backward(L, R, x, W1, W2)
        return y

    @staticmethod
    def backward(ctx, ybar):
        L, R, x, W1, W2 = ctx.saved_tensors
        qn, left, right, f0, f1, f2 = ctx.static
        bond = Bond(qn, left, right, W1.detach().cpu().numpy(), f0, f1, W2.detach().cpu().numpy(), f2)
        ybar = ybar.contiguous()
        xbar, Lbar, Rbar = torch.empty_like(x), torch.empty_like(L), torch.empty_like(R)
        torch.cuda.current_stream().synchronize()
        want_w = ctx.needs_input_grad[4] or ctx.needs_input_grad[5]
        W1b, W2b = heff_backward(bond, L.data_ptr(), R.data_ptr(), x.data_ptr(), ybar.data_ptr(), xbar.data_ptr(),
                                 Lbar.data_ptr(), Rbar.data_ptr(), want_w=want_w)
        gW1 = torch.from_numpy(np.ascontiguousarray(W1b)).to(W1.device) if want_w else None
        gW2 = torch.from_numpy(np.ascontiguousarray(W2b)).to(W2.device) if want_w else None
        return None, Lbar, Rbar, xbar, gW1, gW2


def heff(qn, left, right, f0, f1, f2, L, R, x, W1, W2):
    """y = H_eff x with autograd support (see the module docstring)."""
    static = (list(qn), dict(left), dict(right), np.asarray(f0), np.asarray(f1), np.asarray(f2))
    return _Heff.apply(static, L, R, x, W1, W2)
