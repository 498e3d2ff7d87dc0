"""Differentiation through the transforms (torch.autograd with the library's
adjoint kernels as backward passes).

Workload: B=96, batch 16, FP64; f = inverse(c0) + 0.01 complex-normal noise on
the grid; loss = sum |forward(f) - c_target|^2 (c_target an independent draw
with the same 1/n scaling).  The loss is quadratic, so central differences
with h = 1e-6 are exact up to rounding: for a direction v the derivative
Re<grad, v> (PyTorch's conjugate-Wirtinger gradient) must match
(L(f + h v) - L(f - h v)) / 2h within 1e-8 relative (the difference is taken
per coefficient before summing; its rounding is ~1e-16 |F f| / h relative to
each term's derivative, about 1e-10).  The gradient is also
compared with 2 F^H (F f - c) from the FP64 oracle's adjoint.  Real-function
plans (B=8, FP64) and TF32x3 plans (B=16, twice the split gate: a forward
and an adjoint in a row) are checked against the
oracle's adjoints the same way.
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs
from tolerances import SPLIT_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B, NB = 96, 16


@pytest.fixture(scope="module")
def setup():
    from paper_1604_05140_gb300 import Plan
    plan = Plan(B, NB, "fp64")
    c0 = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 5, decay=True)
    ct = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 6, decay=True)
    noise = 0.01 * inputs.random_samples(B, NB, seed=inputs.BASE_SEED + 7)
    c0_t = torch.from_numpy(c0).cuda()
    f = plan.inverse(c0_t) + torch.from_numpy(noise).cuda()
    return plan, f.contiguous(), torch.from_numpy(ct).cuda()


def _loss_difference(plan, f, v, h, ct):
    """L(f + h v) - L(f - h v) for L(x) = sum |forward(x) - ct|^2, with the
    difference of the two losses taken per coefficient before the sum, so
    that the rounding of two large totals does not swamp it."""
    rp = (plan.forward(f + h * v) - ct).abs() ** 2
    rm = (plan.forward(f - h * v) - ct).abs() ** 2
    return float((rp - rm).sum().item())


def test_autograd_gradient_matches_finite_differences(setup):
    from paper_1604_05140_gb300 import sgl_forward_autograd
    plan, f, ct = setup
    x = f.clone().requires_grad_(True)
    out = sgl_forward_autograd(x, plan)
    loss = ((out - ct).abs() ** 2).sum()
    loss.backward()
    g = x.grad.detach()
    rng = np.random.default_rng(123)
    h = 1e-6
    worst = 0.0
    for k in range(16):
        v = rng.standard_normal(f.shape)
        v = torch.from_numpy(v if k < 8 else 1j * v).to(torch.complex128).cuda()
        fd = _loss_difference(plan, f, v, h, ct) / (2 * h)
        an = float(torch.real(torch.vdot(g.reshape(-1), v.reshape(-1))).item())
        rel = abs(fd - an) / abs(an)
        worst = max(worst, rel)
    assert worst < 1e-8, worst


def test_autograd_gradient_matches_oracle_adjoint(setup):
    from paper_1604_05140_gb300 import sgl_forward_autograd
    plan, f, ct = setup
    x = f.clone().requires_grad_(True)
    loss = ((sgl_forward_autograd(x, plan) - ct).abs() ** 2).sum()
    loss.backward()
    g = x.grad.detach().cpu().numpy()
    fn = f.cpu().numpy()
    ctn = ct.cpu().numpy()
    for k in (0, NB - 1):   # two functions of the batch through the oracle
        resid = O.forward(fn[k], B) - ctn[k][None]
        ref = 2 * O.adjoint_forward(resid, B)[0]
        err = np.abs(g[k] - ref).max() / np.abs(ref).max()
        assert err < 1e-12, (k, err)


def test_inverse_autograd_matches_oracle_adjoint(setup):
    from paper_1604_05140_gb300 import sgl_inverse_autograd
    plan, f, _ = setup
    c = torch.from_numpy(inputs.random_coeffs(B, NB, seed=11, decay=True)).cuda().requires_grad_(True)
    w = f.detach()
    # L = Re <w, inverse(c)> -> grad_c = F_inv^H w (conjugate-Wirtinger, times 1)
    s = sgl_inverse_autograd(c, plan)
    loss = torch.real(torch.vdot(w.reshape(-1), s.reshape(-1)))
    loss.backward()
    g = c.grad.detach().cpu().numpy()
    wn = w.cpu().numpy()
    ref = O.adjoint_inverse(wn[:1], B)[0]
    err = np.abs(g[0] - ref).max() / np.abs(ref).max()
    assert err < 1e-12, err


def test_real_plan_autograd_matches_oracle_adjoints():
    # real samples: the forward's gradient is the real part of the complex
    # adjoint, the inverse's (samples = Re of the complex inverse) is the
    # complex adjoint of the real sample gradient
    from paper_1604_05140_gb300 import Plan, sgl_forward_autograd, sgl_inverse_autograd
    Bs, nb = 8, 3
    p = Plan(Bs, nb, "fp64", samples="real")
    rng = np.random.default_rng(321)
    g = rng.standard_normal(p.sample_shape)
    ct = inputs.random_coeffs(Bs, nb, seed=322)
    x = torch.from_numpy(g).cuda().requires_grad_(True)
    loss = ((sgl_forward_autograd(x, p) - torch.from_numpy(ct).cuda()).abs() ** 2).sum()
    loss.backward()
    assert x.grad.dtype == torch.float64
    resid = O.forward(g, Bs) - ct
    ref = 2 * O.adjoint_forward(resid, Bs).real
    gx = x.grad.cpu().numpy()
    assert np.abs(gx - ref).max() / np.abs(ref).max() < 1e-12

    c = torch.from_numpy(inputs.random_coeffs(Bs, nb, seed=323)).cuda().requires_grad_(True)
    w = rng.standard_normal(p.sample_shape)
    s = sgl_inverse_autograd(c, p)
    assert s.dtype == torch.float64
    (s * torch.from_numpy(w).cuda()).sum().backward()
    ref = O.adjoint_inverse(w + 0j, Bs)
    gc = c.grad.cpu().numpy()
    assert np.abs(gc - ref).max() / np.abs(ref).max() < 1e-12


def test_tf32x3_autograd_matches_oracle_adjoint():
    # the tensor-core adjoint kernels as backward passes, split-precision gate
    from paper_1604_05140_gb300 import Plan, sgl_forward_autograd
    Bs, nb = 16, 2
    p = Plan(Bs, nb, "tf32x3")
    c0 = inputs.random_coeffs(Bs, nb, seed=324, decay=True)
    f = O.inverse(c0, Bs).astype(np.complex64)
    ct = inputs.random_coeffs(Bs, nb, seed=325, decay=True).astype(np.complex64)
    x = torch.from_numpy(f).cuda().requires_grad_(True)
    loss = ((sgl_forward_autograd(x, p) - torch.from_numpy(ct).cuda()).abs() ** 2).sum()
    loss.backward()
    resid = O.forward(f.astype(np.complex128), Bs) - ct.astype(np.complex128)
    ref = 2 * O.adjoint_forward(resid, Bs)
    gx = x.grad.cpu().numpy()
    for k in range(nb):
        # two split-precision transforms in a row (forward, then its adjoint)
        assert np.abs(gx[k] - ref[k]).max() / np.abs(ref[k]).max() < 2 * SPLIT_TOL, k
