"""Trainable per-iteration phases: a torch.autograd.Function over the C ABI.

forward(phi, psi) runs K = len(phi) iterations of the generalised Grover gate
G_k = D(psi_k) O(phi_k) on the handle's MPS (checkpointing every few
iterations) and returns P_marked; backward calls grover_mps_backward, the
hand-written adjoint (costate MPS swept backwards, the segment between two
checkpoints recomputed).  PyTorch supplies only the tensors; every step runs
in libgrover_mps.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


class GroverPhases(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi: torch.Tensor, psi: torch.Tensor, handle: "binding.GroverMPS"):
        ph = phi.detach().to("cpu", torch.float64).numpy()
        ps = psi.detach().to("cpu", torch.float64).numpy()
        handle.reset()
        handle.iterate(len(ph), ph, ps)
        p = handle.prob_marked()
        ctx.handle = handle
        ctx.meta = (phi.dtype, phi.device, psi.dtype, psi.device)
        return torch.tensor(p, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_p):
        gphi, gpsi = ctx.handle.backward(float(grad_p))
        d1, v1, d2, v2 = ctx.meta
        return (torch.from_numpy(np.ascontiguousarray(gphi)).to(v1, d1),
                torch.from_numpy(np.ascontiguousarray(gpsi)).to(v2, d2), None)


def differentiable_handle(n, marked, K, dtype="c128", apply="fused", chi_max=None, checkpoint_every=8,
                          stream=None):
    """A handle able to record K iterations for GroverPhases."""
    return binding.GroverMPS(n, marked, dtype=dtype, apply=apply,
                             chi_max=chi_max if chi_max else len(marked) + 1,
                             differentiable=True, checkpoint_every=checkpoint_every, max_iters=K,
                             stream=stream)


def loss_and_grad_batch(n, marked, phis, psis, dtype="c128", apply="fused", chi_max=None, checkpoint_every=8,
                        stream=None):
    """L = 1 - P_marked and its gradients for B independent phase vectors
    (rows of phis, psis: B x K), all at once through
    grover_mps_diff_batch_run: the forward segments, checkpoint copies,
    projection, segment recomputes and costate sweeps of the B vectors each
    run as one launch (one thread block per vector).  Returns (L[B],
    dL/dphi[B, K], dL/dpsi[B, K])."""
    phis = np.ascontiguousarray(phis, dtype=np.float64)
    psis = np.ascontiguousarray(psis, dtype=np.float64)
    nb, K = phis.shape
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    db = binding.DiffBatch(n, marked, nb, K, dtype=dtype, apply=apply, chi_max=chi_max,
                           checkpoint_every=checkpoint_every, stream=stream)
    try:
        return db.run(phis, psis)
    finally:
        db.close()
