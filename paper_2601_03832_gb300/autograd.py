"""Trainable per-iteration phases: a torch.autograd.Function over the C ABI.

forward(phi, psi) runs K = len(phi) iterations of the generalised Grover gate
G_k = D(psi_k) O(phi_k) on the handle's MPS (checkpointing every few
iterations) and returns P_marked; backward calls grover_mps_backward, the
hand-written adjoint (costate MPS swept backwards, the segment between two
checkpoints recomputed).  PyTorch supplies only the tensors; every step runs
in libgrover_mps.so.
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

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


def loss_and_grad_batch(n, marked, phis, psis, dtype="c128", apply="fused", chi_max=None, checkpoint_every=8):
    """L = 1 - P_marked and its gradients for B independent phase vectors
    (rows of phis, psis: B x K), all at once.  Each vector gets its own
    handle and CUDA stream and is driven from its own host thread (the C
    calls release the GIL), so the single-block launches of the B vectors
    run side by side on different SMs.  Returns (L[B], dL/dphi[B, K],
    dL/dpsi[B, K])."""
    phis = np.ascontiguousarray(phis, dtype=np.float64)
    psis = np.ascontiguousarray(psis, dtype=np.float64)
    nb, K = phis.shape
    binding.load()
    streams = [torch.cuda.Stream() for _ in range(nb)]
    # handles are created up front: device allocations from many threads at
    # once contend (measured slower than creating them in turn)
    handles = [differentiable_handle(n, marked, K, dtype=dtype, apply=apply, chi_max=chi_max,
                                     checkpoint_every=checkpoint_every, stream=s.cuda_stream) for s in streams]

    def run(i):
        h = handles[i]
        h.iterate(K, phis[i], psis[i])
        p = h.prob_marked()
        gphi, gpsi = h.backward(-1.0)
        return 1.0 - p, gphi, gpsi

    try:
        # more concurrent single-block launches than SMs buy nothing
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        with ThreadPoolExecutor(max_workers=max(1, min(nb, sms))) as ex:
            out = list(ex.map(run, range(nb)))
    finally:
        for h in handles:
            h.close()
    return (np.array([o[0] for o in out]), np.stack([o[1] for o in out]), np.stack([o[2] for o in out]))
