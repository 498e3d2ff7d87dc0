"""Reduced-precision variants of the tensor-core path: SGL_TF32 (hi*hi only)
and SGL_BF16X3 (BF16 hi/lo pairs, three products).

Every input and table entry is rounded to TF32 (unit round-off u = 2^-11) and
multiplied once, so each stage carries a relative error of up to 2u ~ 1e-3 of
its terms; four chained stages (inverse then forward) give the bound
TF32_TOL = 4 * 2u = 3.9e-3 on the normwise error, doubled for the forward of
arbitrary samples, whose sums cancel more.  The test also checks that the
variant is indeed coarser than SGL_TF32X3 (the products really are dropped).

SGL_BF16X3 represents every input and table entry as hi + lo with 8 + 8
significant bits (representation error <= 2^-17 relative, the dropped lo*lo
product <= 2^-18), so each stage carries up to ~2^-16 of its terms; four
stages and a factor 2 for cancellation give BF16X3_TOL = 8 * 2^-16 = 1.2e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs
from tolerances import SPLIT_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -11
TF32_TOL = 4 * 2 * U
BF16X3_TOL = 8 * 2.0 ** -16


def _err(gpu, ref):
    g = np.asarray(gpu).reshape(np.asarray(gpu).shape[0], -1)
    r = np.asarray(ref).reshape(np.asarray(ref).shape[0], -1)
    return (np.abs(g - r).max(axis=1) / np.abs(r).max(axis=1)).max()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()


@pytest.mark.parametrize("B", [8, 32, 64])
def test_tf32_vs_oracle(B):
    from paper_1604_05140_gb300 import Plan
    p = Plan(B, 2, "tf32")
    c = inputs.random_coeffs(B, 2, seed=7300 + B)
    s_gpu = p.inverse(_dev(c)).cpu().numpy()
    e_inv = _err(s_gpu, O.inverse(c, B))
    assert e_inv < TF32_TOL
    g = inputs.random_samples(B, 2, seed=7400 + B)
    e_fwd = _err(p.forward(_dev(g)).cpu().numpy(), O.forward(g.astype(np.complex64), B))
    assert e_fwd < 2 * TF32_TOL
    e_rt = _err(p.forward(_dev(O.inverse(c, B))).cpu().numpy(), c)
    assert e_rt < TF32_TOL
    # the three-product plan on the same input is far more accurate
    p3 = Plan(B, 2, "tf32x3")
    e3 = _err(p3.forward(_dev(O.inverse(c, B))).cpu().numpy(), c)
    assert e3 < SPLIT_TOL and e_rt > 10 * e3
    p.check()


def test_tf32_full_size_round_trip():
    from paper_1604_05140_gb300 import Plan
    B, NB = 128, 64
    p = Plan(B, NB, "tf32")
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 3, decay=True)
    s = p.inverse(_dev(c))
    f = p.forward(s).cpu().numpy()
    assert _err(f, c) < TF32_TOL
    sk = s[0].cpu().numpy()
    assert _err(sk[None], O.inverse(c[0], B)) < TF32_TOL
    p.check()


@pytest.mark.parametrize("B", [8, 32, 64])
def test_bf16x3_vs_oracle(B):
    from paper_1604_05140_gb300 import Plan
    p = Plan(B, 2, "bf16x3")
    c = inputs.random_coeffs(B, 2, seed=7500 + B)
    s_gpu = p.inverse(_dev(c)).cpu().numpy()
    assert _err(s_gpu, O.inverse(c, B)) < BF16X3_TOL
    g = inputs.random_samples(B, 2, seed=7600 + B)
    assert _err(p.forward(_dev(g)).cpu().numpy(), O.forward(g.astype(np.complex64), B)) < 2 * BF16X3_TOL
    e_rt = _err(p.forward(_dev(O.inverse(c, B))).cpu().numpy(), c)
    assert e_rt < BF16X3_TOL
    p.check()


def test_bf16x3_adjoint_and_uneven():
    from paper_1604_05140_gb300 import Plan
    B = 16
    p = Plan(B, 2, "bf16x3")
    y = inputs.random_coeffs(B, 2, seed=9300)
    a1 = p.adjoint(_dev(y), of_inverse=False).cpu().numpy()
    assert _err(a1, O.adjoint_forward(y, B)) < BF16X3_TOL
    Bs = [16, 40, 8, 64]
    q = Plan.many(Bs, precision="bf16x3")
    cs = [inputs.random_coeffs(b, 1, seed=960 + k)[0] for k, b in enumerate(Bs)]
    f = q.forward(q.inverse(_dev(np.concatenate(cs)))).cpu().numpy()
    for k, b in enumerate(Bs):
        co = q.coeff_offset(k)
        assert _err(f[co:co + O.coeff_count(b)][None], cs[k][None]) < BF16X3_TOL, (k, b)
    q.check()


def test_bf16x3_full_size_round_trip():
    from paper_1604_05140_gb300 import Plan
    B, NB = 128, 64
    p = Plan(B, NB, "bf16x3")
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 3, decay=True)
    s = p.inverse(_dev(c))
    f = p.forward(s).cpu().numpy()
    assert _err(f, c) < BF16X3_TOL
    sk = s[NB - 1].cpu().numpy()
    assert _err(sk[None], O.inverse(c[NB - 1], B)) < BF16X3_TOL
    p.check()
