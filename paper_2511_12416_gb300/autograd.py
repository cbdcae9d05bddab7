"""torch.autograd.Function over the library's Exact probabilities.

Forward: ef_circuit_set_angles + ef_prob_exact_dev on the caller's stream.
Backward: ef_prob_grad_dev (the adjoint kernels) with grad_output as dL/dp.
Argument marshalling only; both directions run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import ef_circuit_num_angles, ef_circuit_set_angles, ef_prob_exact_dev, ef_prob_grad_dev


class BornProbabilities(torch.autograd.Function):
    """p = BornProbabilities.apply(angles, circuit, bits): probabilities of the
    bitstrings ``bits`` (int64 CUDA tensor of shape (nb, 2), the uint64 words
    reinterpreted) for the circuit ``circuit`` (a handle from
    ef_circuit_create) with its angle vector replaced by ``angles`` (float64)."""

    @staticmethod
    def forward(ctx, angles, circuit, bits):
        ef_circuit_set_angles(circuit, angles.detach().to("cpu", torch.float64).numpy())
        nb = bits.shape[0]
        out = torch.empty(nb, dtype=torch.float64, device=bits.device)
        stream = torch.cuda.current_stream(bits.device).cuda_stream
        ef_prob_exact_dev(circuit, bits.data_ptr(), nb, out.data_ptr(), 0, stream)
        ctx.circuit = circuit
        ctx.angles_device = angles.device
        ctx.save_for_backward(bits)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (bits,) = ctx.saved_tensors
        nb = bits.shape[0]
        g = grad_out.detach().to(bits.device, torch.float64).contiguous()
        grad = torch.empty(ef_circuit_num_angles(ctx.circuit), dtype=torch.float64, device=bits.device)
        stream = torch.cuda.current_stream(bits.device).cuda_stream
        ef_prob_grad_dev(ctx.circuit, bits.data_ptr(), nb, g.data_ptr(), 0, grad.data_ptr(), stream)
        return grad.to(ctx.angles_device), None, None
