"""Adjoint (reverse-mode phase gradient) of the CUDA path against the CPU
oracle: the statevector adjoint, the invariant-plane model's own reverse
mode (any n) and central finite differences (h = 1e-4, FP64)."""
import numpy as np
import pytest

from oracle import reduced
from oracle import statevector as sv
from paper_2601_03832_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_G = 1e-9      # FP64 gradient entries (|dP/dtheta| <= ~2)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_03832_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("apply", ["split", "fused", "mpo"])
@pytest.mark.parametrize("n,M,K,every", [(6, 2, 10, 3), (9, 3, 7, 8), (4, 1, 5, 1), (10, 1, 12, 5)])
def test_adjoint_vs_statevector(B, apply, n, M, K, every):
    marked = inputs.marked_strings(n, M, seed=300 + n * M + K)
    rng = np.random.default_rng(n + 10 * K)
    phis, psis = rng.normal(np.pi, 0.4, K), rng.normal(np.pi, 0.4, K)
    g = B.GroverMPS(n, marked, apply=apply, chi_max=M + 1, differentiable=True, checkpoint_every=every,
                    max_iters=K)
    g.iterate(K, phis, psis)
    L, rphi, rpsi = sv.adjoint(n, marked, phis, psis)
    assert abs((1 - g.prob_marked()) - L) < 1e-12
    gphi, gpsi = g.backward(-1.0)          # dL/dtheta for L = 1 - P
    assert np.abs(gphi - rphi).max() < TOL_G
    assert np.abs(gpsi - rpsi).max() < TOL_G
    # a second backward from the same forward gives the same result
    gphi2, gpsi2 = g.backward(-1.0)
    assert np.array_equal(gphi, gphi2) and np.array_equal(gpsi, gpsi2)


def test_adjoint_vs_finite_differences(B):
    n, marked, K = 7, [5, 99], 6
    rng = np.random.default_rng(2)
    phis, psis = rng.normal(np.pi, 0.3, K), rng.normal(np.pi, 0.3, K)
    g = B.GroverMPS(n, marked, apply="split", chi_max=3, differentiable=True, checkpoint_every=4, max_iters=K)
    g.iterate(K, phis, psis)
    gphi, gpsi = g.backward(1.0)           # dP/dtheta

    def P(ph, ps):
        return sv.prob_marked(sv.grover(n, marked, K, ph, ps), marked)
    h = 1e-4
    for j in range(K):
        e = np.zeros(K); e[j] = h
        fphi = (P(phis + e, psis) - P(phis - e, psis)) / (2 * h)
        fpsi = (P(phis, psis + e) - P(phis, psis - e)) / (2 * h)
        assert abs(gphi[j] - fphi) < 1e-7 and abs(gpsi[j] - fpsi) < 1e-7


def test_differentiable_config_against_reduced_model(B):
    """n = 20, M = 4, K = 64, phases N(pi, 0.1) in float32: two of the 64
    phase vectors, checked against the invariant-plane reverse mode."""
    inst, phi, psi = inputs.config_differentiable(B=2)
    for b in range(2):
        g = B.GroverMPS(inst.n, inst.marked, apply="split", chi_max=inst.M + 1, differentiable=True,
                        checkpoint_every=8, max_iters=inst.k)
        g.iterate(inst.k, phi[b], psi[b])
        L, rphi, rpsi = reduced.loss_and_grad(inst.n, inst.M, phi[b], psi[b])
        assert abs((1 - g.prob_marked()) - L) < 1e-10
        gphi, gpsi = g.backward(-1.0)
        assert np.abs(gphi - rphi).max() < TOL_G
        assert np.abs(gpsi - rpsi).max() < TOL_G
        g.close()


def test_autograd_function(B):
    import torch
    from paper_2601_03832_gb300.autograd import GroverPhases, differentiable_handle
    n, marked, K = 8, [3, 200], 9
    rng = np.random.default_rng(9)
    phi = torch.tensor(rng.normal(np.pi, 0.2, K), dtype=torch.float32, requires_grad=True)
    psi = torch.tensor(rng.normal(np.pi, 0.2, K), dtype=torch.float32, requires_grad=True)
    h = differentiable_handle(n, marked, K, checkpoint_every=4)
    loss = 1.0 - GroverPhases.apply(phi, psi, h)
    loss.backward()
    L, rphi, rpsi = sv.adjoint(n, marked, phi.detach().double().numpy(), psi.detach().double().numpy())
    assert abs(loss.item() - L) < 1e-10
    assert phi.grad.dtype == torch.float32
    assert np.abs(phi.grad.double().numpy() - rphi).max() < 1e-6
    assert np.abs(psi.grad.double().numpy() - rpsi).max() < 1e-6


def test_backward_requires_differentiable_handle(B):
    g = B.GroverMPS(5, [3], chi_max=2)
    g.iterate(2)
    with pytest.raises(B.GMPSError) as e:
        g.backward(-1.0)
    assert e.value.status == 7


@pytest.mark.parametrize("apply,every", [("fused", 8), ("split", 5), ("mpo", 16)])
def test_batched_launch_matches_one_by_one(B, apply, every):
    """grover_mps_diff_batch_run runs the phase vectors as batched launches;
    every vector's loss and gradients equal those of a differentiable handle
    run alone (same kernels, same arithmetic), and the reduced model's."""
    import torch
    from paper_2601_03832_gb300 import autograd as AG
    n, M, K = 12, 3, 16
    marked = inputs.marked_strings(n, M, seed=91)
    rng = np.random.default_rng(5)
    phis, psis = rng.normal(np.pi, 0.3, (6, K)), rng.normal(np.pi, 0.3, (6, K))
    L, gphi, gpsi = AG.loss_and_grad_batch(n, marked, phis, psis, apply=apply, checkpoint_every=every)
    torch.cuda.synchronize()
    for b in range(len(phis)):
        h = AG.differentiable_handle(n, marked, K, apply=apply, checkpoint_every=every)
        h.iterate(K, phis[b], psis[b])
        l1 = 1.0 - h.prob_marked()
        g1, g2 = h.backward(-1.0)
        h.close()
        assert abs(L[b] - l1) < 1e-14
        assert np.abs(gphi[b] - g1).max() < 1e-14 and np.abs(gpsi[b] - g2).max() < 1e-14
        Lr, rphi, rpsi = reduced.loss_and_grad(n, M, phis[b], psis[b])
        assert abs(L[b] - Lr) < 1e-10
        assert np.abs(gphi[b] - rphi).max() < TOL_G and np.abs(gpsi[b] - rpsi).max() < TOL_G


def test_differentiable_batch_of_64_against_reduced_model(B):
    """The differentiable workload (n = 20, M = 4, K = 64, 64 phase vectors
    N(pi, 0.1) in float32, checkpoint every 8) in one batched run: every loss
    and gradient entry against the invariant-plane reverse mode."""
    from paper_2601_03832_gb300 import autograd as AG
    inst, phi, psi = inputs.config_differentiable(B=64)
    L, gphi, gpsi = AG.loss_and_grad_batch(inst.n, inst.marked, phi, psi)
    for b in range(64):
        Lr, rphi, rpsi = reduced.loss_and_grad(inst.n, inst.M, phi[b], psi[b])
        assert abs(L[b] - Lr) < 1e-10
        assert np.abs(gphi[b] - rphi).max() < TOL_G and np.abs(gpsi[b] - rpsi).max() < TOL_G
