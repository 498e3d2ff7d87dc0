"""SGL_FP16X3: the Legendre sums (Eq. DLT) and radial sums (Eq. DRT_matrix) as
three products of FP16 hi/lo pairs on the tensor cores, against the FP64
oracle.

FP16 pairs carry 11 + 11 significant bits, as TF32 pairs do, so the path is
held to the split-precision gate (tests/tolerances.py: 1e-6 normwise per
function).  FP16's exponent range (normal values 6e-5 .. 65504) is handled by
power-of-two scales, per table block on the host and per function and stage
on the device (from the measured largest magnitude of the function's
phi-spectra or coefficients); the tests therefore also run functions whose
magnitudes differ by 27 orders in one batch, and a function that is zero.
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs
from tolerances import SPLIT_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _err(gpu, ref):
    g = np.asarray(gpu).reshape(np.asarray(gpu).shape[0], -1)
    r = np.asarray(ref).reshape(np.asarray(ref).shape[0], -1)
    return (np.abs(g - r).max(axis=1) / np.abs(r).max(axis=1)).max()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()


def _plan(B, batch, **kw):
    from paper_1604_05140_gb300 import Plan
    return Plan(B, batch, "fp16x3", **kw)


@pytest.mark.parametrize("B,batch", [(8, 3), (32, 2), (64, 2), (128, 2)])
def test_fp16x3_vs_oracle(B, batch):
    p = _plan(B, batch)
    c = inputs.random_coeffs(B, batch, seed=7900 + B, decay=True)
    s_gpu = p.inverse(_dev(c)).cpu().numpy()
    assert _err(s_gpu, O.inverse(c, B)) < SPLIT_TOL
    g = inputs.random_samples(B, batch, seed=8100 + B)
    assert _err(p.forward(_dev(g)).cpu().numpy(), O.forward(g.astype(np.complex64), B)) < SPLIT_TOL
    back = p.forward(_dev(O.inverse(c, B))).cpu().numpy()
    assert _err(back, c) < SPLIT_TOL
    p.check()


def test_fp16x3_functions_of_very_different_magnitude():
    # one batch, magnitudes from 1e-12 to 1e15 (FP16 alone holds 6e-8 .. 6.5e4):
    # each function gets its own scale, so each keeps the split-precision bound
    B = 32
    scales = np.array([1e-12, 1e-6, 1.0, 1e6, 1e15])
    p = _plan(B, len(scales))
    c = inputs.random_coeffs(B, len(scales), seed=8300, decay=True) * scales[:, None]
    s = p.inverse(_dev(c))
    ref = O.inverse(c, B)
    assert _err(s.cpu().numpy(), ref) < SPLIT_TOL
    assert _err(p.forward(s).cpu().numpy(), c) < SPLIT_TOL
    g = inputs.random_samples(B, len(scales), seed=8400) * scales[:, None, None, None]
    assert _err(p.forward(_dev(g)).cpu().numpy(), O.forward(g.astype(np.complex64), B)) < SPLIT_TOL
    p.check()


def test_fp16x3_zero_function_in_a_batch():
    # a function that is zero has no magnitude to scale by: its coefficients
    # and samples come out exactly zero, and its neighbours are unaffected
    B = 16
    p = _plan(B, 3)
    c = inputs.random_coeffs(B, 3, seed=8500)
    c[1] = 0
    s = p.inverse(_dev(c))
    f = p.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    assert not s[1].any() and not f[1].any()
    keep = [0, 2]
    assert _err(f[keep], c[keep]) < SPLIT_TOL
    assert _err(s[keep], O.inverse(c[keep], B)) < SPLIT_TOL
    p.check()


def test_fp16x3_adjoints_vs_oracle():
    B = 16
    p = _plan(B, 2)
    y = inputs.random_coeffs(B, 2, seed=8600)
    x = inputs.random_samples(B, 2, seed=8700)
    a1 = p.adjoint(_dev(y), of_inverse=False).cpu().numpy()
    assert _err(a1, O.adjoint_forward(y, B)) < SPLIT_TOL
    a2 = p.adjoint(_dev(x), of_inverse=True).cpu().numpy()
    assert _err(a2, O.adjoint_inverse(x.astype(np.complex64), B)) < SPLIT_TOL
    p.check()


def test_fp16x3_uneven_bandlimits_and_real_functions():
    from paper_1604_05140_gb300 import Plan
    Bs = [16, 40, 8, 128, 24, 64]
    q = Plan.many(Bs, precision="fp16x3")
    cs = [inputs.random_coeffs(b, 1, seed=8800 + k, decay=True)[0] for k, b in enumerate(Bs)]
    s = q.inverse(_dev(np.concatenate(cs)))
    f = q.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    for k, b in enumerate(Bs):
        co, so = q.coeff_offset(k), q.sample_offset(k)
        assert _err(f[co:co + O.coeff_count(b)][None], cs[k][None]) < SPLIT_TOL, (k, b)
        if b <= 64:
            sk = s[so:so + 4 * b ** 3].reshape(1, b, 2 * b, 2 * b)
            assert _err(sk, O.inverse(cs[k], b)) < SPLIT_TOL, (k, b)
    q.check()
    # real functions: two per complex transform, separated by the symmetry
    B, n = 16, 3
    r = _plan(B, n, samples="real")
    g = np.real(inputs.random_samples(B, n, seed=8900)).astype(np.float32)
    fr = r.forward(torch.from_numpy(g).cuda()).cpu().numpy()
    assert _err(fr, O.forward(g.astype(np.complex128), B)) < SPLIT_TOL
    r.check()


def test_fp16x3_full_size_round_trip():
    B, NB = 128, 64
    p = _plan(B, NB)
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 3, decay=True)
    s = p.inverse(_dev(c))
    f = p.forward(s).cpu().numpy()
    assert _err(f, c) < SPLIT_TOL
    sk = s[NB - 1].cpu().numpy()
    assert _err(sk[None], O.inverse(c[NB - 1], B)) < SPLIT_TOL
    p.check()
