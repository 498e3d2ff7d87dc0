"""GPU parity of the seminaive forward Legendre stage (sgl_set_dlt).

The oracle's seminaive sums (Eq. DCT, Eq. dct_trick over all 2B rings) are
pinned against its direct sums and the DCT truncation property in
test_oracle_pins; the GPU folds the rings (DCT-II of E, DCT-IV of O, each of
length B through an FFT of length 2B) and truncates each degree's inner
product.  Its forward results must equal the oracle's forward transform:
FP64 1e-12, FP32 2e-5 (normwise per function).
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plan(*a, seminaive=True, **k):
    from paper_1604_05140_gb300 import Plan
    p = Plan(*a, **k)
    p.set_dlt(seminaive)
    return p


def _err(gpu, ref):
    g = np.asarray(gpu).reshape(np.shape(gpu)[0], -1)
    r = np.asarray(ref).reshape(np.shape(ref)[0], -1)
    return (np.abs(g - r).max(axis=1) / np.abs(r).max(axis=1)).max()


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


@pytest.mark.parametrize("B", [1, 2, 3, 5, 8, 16, 24, 64])
def test_seminaive_forward_fp64_vs_oracle(B):
    p = _plan(B, 2, "fp64")
    g = inputs.random_samples(B, 2, seed=3000 + B)
    f = p.forward(_dev(g, torch.complex128)).cpu().numpy()
    assert _err(f, O.forward(g, B)) < 1e-12
    # without the weights: the adjoint of the inverse takes the forward pipeline
    a = p.adjoint(_dev(g, torch.complex128), of_inverse=True).cpu().numpy()
    assert _err(a, O.adjoint_inverse(g, B)) < 1e-12
    # and the round trip through the (direct) inverse
    c = inputs.random_coeffs(B, 2, seed=3100 + B)
    back = p.forward(p.inverse(_dev(c, torch.complex128))).cpu().numpy()
    assert _err(back, c) < 1e-12
    p.check()


def test_seminaive_forward_fp32():
    B = 16
    p = _plan(B, 3, "fp32")
    g = inputs.random_samples(B, 3, seed=3200)
    f = p.forward(_dev(g, torch.complex64)).cpu().numpy()
    assert _err(f, O.forward(g.astype(np.complex64), B)) < 2e-5


def test_seminaive_b128_matches_direct():
    B = 128
    p = _plan(B, 2, "fp64")
    c = inputs.random_coeffs(B, 2, seed=3300, decay=True)
    s = p.inverse(_dev(c, torch.complex128))
    semi = p.forward(s).cpu().numpy()
    p.set_dlt(False)
    direct = p.forward(s).cpu().numpy()
    assert _err(semi, direct) < 1e-12 and _err(semi, c) < 1e-12
    p.check()


def test_seminaive_with_real_functions_and_paper_grid():
    B = 8
    p = _plan(B, 3, "fp64", samples="real")
    g = np.random.default_rng(3400).standard_normal((3, B, 2 * B, 2 * B))
    assert _err(p.forward(_dev(g, torch.float64)).cpu().numpy(), O.forward(g, B)) < 1e-12
    p = _plan(B, 2, "fp64", grid="hermite")
    g = np.random.default_rng(3401).standard_normal((2, 2 * B, 2 * B, 2 * B)) + 0j
    assert _err(p.forward(_dev(g, torch.complex128)).cpu().numpy(), O.forward(g, B, rule="hermite")) < 1e-12


def test_seminaive_host_buffers_in_sub_batches():
    B, batch = 8, 17
    p = _plan(B, batch, "fp32")
    g = inputs.random_samples(B, batch, seed=3500).astype(np.complex64)
    dev = p.forward(_dev(g, torch.complex64)).cpu()
    host = p.forward(torch.from_numpy(g))
    assert torch.equal(dev, host)


def test_seminaive_unsupported_on_tensor_cores():
    from paper_1604_05140_gb300 import Plan, sgl
    p = Plan(8, 1, "tf32x3")
    assert p.lib.sgl_set_dlt(p.handle, 1) == sgl.SGL_ERR_UNSUPPORTED
    assert p.lib.sgl_set_dlt(p.handle, 0) == sgl.SGL_ERR_UNSUPPORTED


def test_seminaive_uneven_bandlimits():
    # one DCT launch per bandlimit segment
    from paper_1604_05140_gb300 import Plan
    Bs = [8, 5, 16, 8, 12]
    p = Plan.many(Bs, precision="fp64")
    p.set_dlt(True)
    gs = [inputs.random_samples(B, 1, seed=3600 + k)[0] for k, B in enumerate(Bs)]
    f = p.forward(_dev(np.concatenate([g.reshape(-1) for g in gs]), torch.complex128)).cpu().numpy()
    for k, B in enumerate(Bs):
        co = p.coeff_offset(k)
        assert _err(f[co:co + O.coeff_count(B)][None], O.forward(gs[k], B)) < 1e-12, (k, B)
    p.check()
