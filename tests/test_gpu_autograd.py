"""The differentiable ST-AGM loss (torch.autograd.Function over the CUDA adjoint)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2011_00162_gb300 as od
from paper_2011_00162_gb300 import build as odbuild
from paper_2011_00162_gb300 import synth
from paper_2011_00162_gb300.autograd import stagm_loss

from _cases import rel_l2

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    odbuild.build()


def _case(m=16, n=64, step=4, seed=2):
    p = synth.Problem("ag", n, m, step, 1, 1, 1, 0, 1e4, 1, seed=seed)
    offs = p.offsets()
    u_true, w = p.truth(), p.probe()
    f = synth.poissonize(np.abs(oracle.forward(u_true, w, offs)) ** 2, p.peak, 3)
    rng = np.random.default_rng(seed)
    u0 = (u_true * (1 + 0.2 * (rng.standard_normal(u_true.shape) + 1j * rng.standard_normal(u_true.shape)))).astype(np.complex64)
    w0 = (w * (1 + 0.1 * rng.standard_normal(w.shape))).astype(np.complex64)
    plan = od.ptycho_plan(od.Geometry(n, n, m, offs, eps=0.5), torch.from_numpy(f).to(DEV))
    return plan, u0, w0, offs, f


def test_autograd_equals_c_abi_gradients_and_oracle():
    plan, u0, w0, offs, f = _case()
    u = torch.from_numpy(u0).to(DEV).requires_grad_(True)
    w = torch.from_numpy(w0).to(DEV).requires_grad_(True)
    L = stagm_loss(u, w, plan)
    L.backward()
    loss, gu, gw = od.stagm_loss_grad(plan, u.detach(), w.detach())
    assert torch.equal(L.detach().reshape(1), loss)
    assert torch.equal(u.grad, gu) and torch.equal(w.grad, gw)
    Lo, gu_o, gw_o = oracle.loss_grad(u0, w0, offs, f.astype(np.float64), 0.5)
    assert rel_l2(u.grad.cpu().numpy(), gu_o) < 1e-5 and rel_l2(w.grad.cpu().numpy(), gw_o) < 1e-5
    # the chain rule through a scalar multiple of the loss
    u.grad = None
    (3.0 * stagm_loss(u, w, plan)).backward()
    assert torch.allclose(u.grad, 3.0 * gu, rtol=1e-6, atol=0)


def test_autograd_central_differences_fp32():
    plan, u0, w0, offs, f = _case()
    u = torch.from_numpy(u0).to(DEV).requires_grad_(True)
    w = torch.from_numpy(w0).to(DEV).requires_grad_(True)
    stagm_loss(u, w, plan).backward()
    rng = np.random.default_rng(0)
    h = 3e-2
    for _ in range(8):
        i, k = (int(v) for v in rng.integers(8, 56, 2))
        for unit, part in ((1.0, torch.real), (1j, torch.imag)):
            up, um = u.detach().clone(), u.detach().clone()
            up[i, k] += h * unit
            um[i, k] -= h * unit
            fd = (stagm_loss(up, w.detach(), plan) - stagm_loss(um, w.detach(), plan)).item() / (2 * h)
            g = part(u.grad[i, k]).item()
            assert abs(fd - g) <= 2e-2 * abs(g) + 2e-3, (i, k, fd, g)
        i, k = (int(v) for v in rng.integers(3, 13, 2))
        wp, wm = w.detach().clone(), w.detach().clone()
        wp[i, k] += h
        wm[i, k] -= h
        fd = (stagm_loss(u.detach(), wp, plan) - stagm_loss(u.detach(), wm, plan)).item() / (2 * h)
        g = torch.real(w.grad[i, k]).item()
        assert abs(fd - g) <= 2e-2 * abs(g) + 2e-3, (i, k, fd, g)


def test_gradient_descent_on_object_and_probe_lowers_the_loss():
    plan, u0, w0, offs, f = _case(m=64, n=256, step=16, seed=5)
    u = torch.from_numpy(u0).to(DEV).requires_grad_(True)
    w = torch.from_numpy(w0).to(DEV).requires_grad_(True)
    opt = torch.optim.Adam([u, w], lr=2e-3)
    L0 = None
    for _ in range(25):
        opt.zero_grad()
        L = stagm_loss(u, w, plan)
        L.backward()
        opt.step()
        L0 = L.item() if L0 is None else L0
    assert stagm_loss(u.detach(), w.detach(), plan).item() < 0.7 * L0


@pytest.mark.parametrize("m,n,step", [(16, 64, 4), (128, 384, 48), (256, 512, 96), (48, 144, 12)])
def test_stored_gradient_frames_equal_recomputed(m, n, step):
    """recompute = 0 keeps the gradient frames, recompute = 2 gathers from them:
    the same loss and gradients bit for bit as recomputing; a store made for
    other u / w pointers, or none at all, is refused."""
    plan, u0, w0, offs, f = _case(m=m, n=n, step=step, seed=m)
    u = torch.from_numpy(u0).to(DEV)
    w = torch.from_numpy(w0).to(DEV)
    with pytest.raises(od.PtychoError) as e:
        od.stagm_loss_grad(plan, u, w, recompute=od.FROM_STORE)
    assert e.value.code == 6
    L1, gu1, gw1 = od.stagm_loss_grad(plan, u, w, recompute=od.RECOMPUTE)
    Ls, _, _ = od.stagm_loss_grad(plan, u, w, grad_u=False, grad_w=False, recompute=od.STORE)
    # other frame work on the plan (here a recomputed loss elsewhere) leaves the store alone
    od.stagm_loss_grad(plan, u * 0.5, w, recompute=od.RECOMPUTE)
    L2, gu2, gw2 = od.stagm_loss_grad(plan, u, w, recompute=od.FROM_STORE)
    assert torch.equal(L1, Ls) and torch.equal(L1, L2)
    assert torch.equal(gu1, gu2) and torch.equal(gw1, gw2)
    with pytest.raises(od.PtychoError) as e:
        od.stagm_loss_grad(plan, u.clone(), w, recompute=od.FROM_STORE)
    assert e.value.code == 6


def test_autograd_store_and_recompute_agree():
    from paper_2011_00162_gb300 import autograd
    plan, u0, w0, offs, f = _case()
    grads = []
    for budget in (8 << 30, 0):  # frames kept for the backward; recomputed
        autograd.STORE_BUDGET_BYTES = budget
        u = torch.from_numpy(u0).to(DEV).requires_grad_(True)
        w = torch.from_numpy(w0).to(DEV).requires_grad_(True)
        stagm_loss(u, w, plan).backward()
        grads.append((u.grad.clone(), w.grad.clone()))
    autograd.STORE_BUDGET_BYTES = 8 << 30
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])
    # two graphs on one plan: the first backward finds the store replaced and recomputes
    u1 = torch.from_numpy(u0).to(DEV).requires_grad_(True)
    u2 = torch.from_numpy(u0 * 0.9).to(DEV).requires_grad_(True)
    w = torch.from_numpy(w0).to(DEV)
    L1, L2 = stagm_loss(u1, w, plan), stagm_loss(u2, w, plan)
    L1.backward()
    assert torch.equal(u1.grad, grads[0][0])
    L2.backward()
    _, gu2, _ = od.stagm_loss_grad(plan, u2.detach(), w)
    assert torch.equal(u2.grad, gu2)
