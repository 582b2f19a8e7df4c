"""torch.autograd.Function for the LUCJ ansatz (§4.3, §4.5.1).

Forward and backward both run in libfsgpu.so: the backward calls the
library's VJP, which recovers the input state by uncomputation (reverse
sweeps) instead of storing intermediate states.  Only the output state is
kept between the two passes, as the starting point of the reverse sweeps.

Gradient conventions (PyTorch's for complex tensors): for a real loss L and
complex z, z.grad = dL/dRe z + i dL/dIm z.  K (n_reps, N, N) complex128 and
J_aa, J_ab (n_reps, N, N) float64 may live on any device; their gradients
treat every entry as independent (project onto the anti-Hermitian or
symmetric parameterisation in the caller if needed).
"""

import numpy as np
import torch

from . import fsgpu


class LUCJFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vec, K, J_aa, J_ab, norb, nelec, from_hf):
        Kn = K.detach().cpu().numpy()
        Ja = J_aa.detach().cpu().numpy()
        Jb = J_ab.detach().cpu().numpy()
        out = vec.detach().clone().contiguous()
        fsgpu.lucj_forward_(out, Kn, Ja, Jb, norb, nelec, from_hf=from_hf)
        ctx.save_for_backward(out)
        ctx.params = (Kn, Ja, Jb, norb, nelec, from_hf)
        ctx.devs = (K.device, K.dtype, J_aa.device, J_aa.dtype, J_ab.device, J_ab.dtype)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (out,) = ctx.saved_tensors
        Kn, Ja, Jb, norb, nelec, from_hf = ctx.params
        psi = out.clone()
        cot = grad_out.detach().to(out.dtype).contiguous().clone()
        dK, dJa, dJb = fsgpu.lucj_vjp_(psi, cot, Kn, Ja, Jb, norb, nelec, from_hf=from_hf)
        kd, kt, ad, at, bd, bt = ctx.devs
        gvec = None if from_hf else cot
        return (gvec, torch.from_numpy(dK).to(kd, kt), torch.from_numpy(dJa).to(ad, at),
                torch.from_numpy(dJb).to(bd, bt), None, None, None)


def lucj(vec, K, J_aa, J_ab, norb, nelec, from_hf=False):
    """LUCJ state: vec (CUDA complex tensor; its values are ignored when
    from_hf) -> new tensor.  Differentiable with respect to vec, K, J_aa, J_ab."""
    return LUCJFunction.apply(vec, K, J_aa, J_ab, norb, tuple(nelec), bool(from_hf))
