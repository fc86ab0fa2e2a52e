"""Differentiation form: the Elfpie cost of Eq. 8 as a torch.autograd.Function.

forward(psi, pupil) returns L = L_fid + alpha L_A + beta L_Phi (Eq. 8) for the
handle's measurements, reduced and weighted in FP64 on the GPU by the library
(elf_cost_grad returns the total beside its three terms); the same call
(elf_cost_grad) produces the closed-form Wirtinger gradients dL/d(conj Psi)
(Eq. 15 = Eq. 9 + alpha Eq. 13 + beta Eq. 14) and dL/d(conj P) (Eq. 18) in the
same pass, and backward returns them scaled.  PyTorch's convention for a real
function of a complex tensor is grad = 2 dL/d(conj z) (the gradient of |z|^2 at
z is 2z), so backward returns 2 * grad_output * dL/d(conj z).

Inputs are complex64 CUDA tensors (the kernels compute in FP32); there is no
double backward.
"""
from __future__ import annotations

import torch

from . import elfpie as E


class ElfCostFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, pupil, elf: E.Elf):
        if psi.dtype != torch.complex64 or pupil.dtype != torch.complex64:
            raise TypeError("psi and pupil must be complex64 (the kernels compute in FP32)")
        if not (psi.is_cuda and pupil.is_cuda):
            raise ValueError("psi and pupil must be CUDA tensors")
        psi_c = psi.detach().contiguous()
        pup_c = pupil.detach().contiguous()
        g_psi = torch.empty_like(psi_c)
        g_pup = torch.empty_like(pup_c)
        costs, _, _ = elf.cost_grad(psi_c, pup_c, g_psi, g_pup)
        ctx.save_for_backward(g_psi, g_pup)
        ctx.costs = costs
        return torch.tensor(costs[3], dtype=torch.float64, device=psi.device)  # Eq. 8's total, from the library

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, grad_out):
        g_psi, g_pup = ctx.saved_tensors
        scale = 2.0 * grad_out.to(torch.float32)
        d_psi = g_psi * scale if ctx.needs_input_grad[0] else None
        d_pup = g_pup * scale if ctx.needs_input_grad[1] else None
        return d_psi, d_pup, None


def elf_cost(psi: torch.Tensor, pupil: torch.Tensor, elf: E.Elf) -> torch.Tensor:
    """Eq. 8 at (psi, pupil) as a differentiable scalar (float64)."""
    return ElfCostFunction.apply(psi, pupil, elf)


class ElfCost(torch.nn.Module):
    """Module form holding the problem handle (measurements, geometry, alpha, beta)."""

    def __init__(self, elf: E.Elf):
        super().__init__()
        self.elf = elf

    def forward(self, psi: torch.Tensor, pupil: torch.Tensor) -> torch.Tensor:
        return ElfCostFunction.apply(psi, pupil, self.elf)
