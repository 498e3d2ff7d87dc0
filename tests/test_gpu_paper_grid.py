"""GPU parity on the paper's own grid: 2B half-range Gauss-Hermite radii
(SGL_GRID_HALF_RANGE_HERMITE; Thm 3.3, Thm 3.4 / Eq. zwischenstufe_2).

The oracle computes that rule in high precision (Chebyshev's algorithm from
the moments) and is pinned by moment exactness and the closed forms in
test_oracle_pins; the library builds it independently (discretized Stieltjes
procedure in long double).  Checked here through the C ABI: the grid itself,
forward / inverse / adjoints against the oracle at FP64 (1e-12) and FP32
(2e-5), closed-form coefficients from physical samples at the library's
nodes, real-function plans, chunked host buffers, and B = 128 (256 radii).
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}
CTYPE = {"fp64": torch.complex128, "fp32": torch.complex64}


def _plan(B, batch, prec, samples="weighted"):
    from paper_1604_05140_gb300 import Plan
    return Plan(B, batch, prec, samples=samples, grid="hermite")


def _err(gpu, ref):
    g = np.asarray(gpu).reshape(np.shape(gpu)[0], -1)
    r = np.asarray(ref).reshape(np.shape(ref)[0], -1)
    return (np.abs(g - r).max(axis=1) / np.abs(r).max(axis=1)).max()


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


@pytest.mark.parametrize("B", [1, 4, 16, 64, 128])
def test_grid_matches_oracle(B):
    p = _plan(B, 1, "fp64")
    assert p.radii == 2 * B and p.sample_shape == (1, 2 * B, 2 * B, 2 * B)
    r, th, ph, wr, wt = p.grid()
    ro, tho, pho, wro, wto = O.grid(B, "hermite")
    assert r.shape == (2 * B,)
    np.testing.assert_allclose(r, ro, rtol=1e-14, atol=0)
    np.testing.assert_allclose(wr, wro, rtol=1e-12, atol=0)
    np.testing.assert_allclose(th, tho, rtol=1e-15)
    np.testing.assert_allclose(wt, wto, rtol=1e-13)


@pytest.mark.parametrize("prec,B,batch", [("fp64", 1, 1), ("fp64", 2, 2), ("fp64", 5, 3), ("fp64", 8, 2),
                                          ("fp64", 16, 2), ("fp64", 24, 1), ("fp32", 8, 3), ("fp32", 24, 2)])
def test_paper_grid_vs_oracle(prec, B, batch):
    p = _plan(B, batch, prec)
    c = inputs.random_coeffs(B, batch, seed=2000 + B)
    s = p.inverse(_dev(c, CTYPE[prec])).cpu().numpy()
    assert s.shape == (batch, 2 * B, 2 * B, 2 * B)
    assert _err(s, O.inverse(c, B, rule="hermite")) < TOL[prec]
    rng = np.random.default_rng(2100 + B)
    shape = (batch, 2 * B, 2 * B, 2 * B)
    g = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)  # noise on all 2B radii
    ref_in = g.astype(np.complex64).astype(np.complex128) if prec == "fp32" else g
    f = p.forward(_dev(g, CTYPE[prec])).cpu().numpy()
    assert _err(f, O.forward(ref_in, B, rule="hermite")) < TOL[prec]
    back = p.forward(_dev(O.inverse(c, B, rule="hermite"), CTYPE[prec])).cpu().numpy()
    assert _err(back, c) < TOL[prec]
    p.check()


def test_paper_grid_adjoints():
    B = 6
    p = _plan(B, 2, "fp64")
    y = inputs.random_coeffs(B, 2, seed=2200)
    x = np.random.default_rng(2201).standard_normal((2, 2 * B, 2 * B, 2 * B)) + 0j
    a1 = p.adjoint(_dev(y, torch.complex128), of_inverse=False).cpu().numpy()
    assert _err(a1, O.adjoint_forward(y, B, rule="hermite")) < TOL["fp64"]
    a2 = p.adjoint(_dev(x, torch.complex128), of_inverse=True).cpu().numpy()
    assert _err(a2, O.adjoint_inverse(x, B, rule="hermite")) < TOL["fp64"]


def test_paper_grid_physical_closed_forms():
    # 1, x, y, z, r^2 sampled at the library's own nodes (physical samples):
    # their coefficients are closed forms of Def 1.2 / Def 2.1
    import os
    B = 4
    from paper_1604_05140_gb300 import Plan
    p = Plan(B, 1, "fp64", samples="physical", grid="hermite")
    r, th, ph, _, _ = p.grid()
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    x, y, z = R * np.sin(TH) * np.cos(PH), R * np.sin(TH) * np.sin(PH), R * np.cos(TH)
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, n, l, m, re_, im_ = line.split()
            rows.append((name, int(n), int(l), int(m), complex(float(re_), float(im_))))
    for name, f in {"one": np.ones_like(x), "x": x, "y": y, "z": z, "r2": R ** 2}.items():
        fh_ = p.forward(_dev(f[None] + 0j, torch.complex128)).cpu().numpy()[0]
        expect = np.zeros_like(fh_)
        for (nm, n, l, m, v) in rows:
            if nm == name:
                expect[O.omega(n, l, m)] = v
        np.testing.assert_allclose(fh_, expect, atol=1e-12, rtol=0, err_msg=name)


def test_paper_grid_real_functions():
    B, batch = 8, 3
    p = _plan(B, batch, "fp64", samples="real")
    g = np.random.default_rng(2300).standard_normal((batch, 2 * B, 2 * B, 2 * B))
    f = p.forward(_dev(g, torch.float64)).cpu().numpy()
    assert _err(f, O.forward(g, B, rule="hermite")) < TOL["fp64"]
    c = inputs.random_coeffs(B, batch, seed=2301)
    s = p.inverse(_dev(c, torch.complex128)).cpu().numpy()
    assert _err(s, O.inverse(c, B, rule="hermite").real) < TOL["fp64"]


def test_paper_grid_host_buffers_in_sub_batches():
    # 17 functions: host-buffer calls run in chunks (per-function sizes follow
    # the 2B radii); the result equals the device-buffer call bit for bit
    B, batch = 8, 17
    p = _plan(B, batch, "fp32")
    c = inputs.random_coeffs(B, batch, seed=2400).astype(np.complex64)
    dev = p.inverse(_dev(c, torch.complex64)).cpu()
    host = p.inverse(torch.from_numpy(c))
    assert torch.equal(dev, host)
    fd = p.forward(dev.cuda()).cpu()
    fh = p.forward(dev)
    assert torch.equal(fd, fh)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_paper_grid_b128(prec):
    # B = 128 on 256 radii (the register FFT with 256 shells per function):
    # one function against the oracle, the round trip of two
    B = 128
    p = _plan(B, 2, prec)
    c = inputs.random_coeffs(B, 2, seed=2500, decay=True)
    s = p.inverse(_dev(c, CTYPE[prec]))
    f = p.forward(s).cpu().numpy()
    assert _err(f, c) < TOL[prec]
    s0 = s[0].cpu().numpy()
    assert _err(s0[None], O.inverse(c[0], B, rule="hermite")) < TOL[prec]
    p.check()


# tensor-core precisions on the paper's grid: each function's 2B radii run as
# two functions of B radii (the first and second half of the radial rule),
# whose radial partial sums (Eq. DRT_matrix) are added; the split-precision
# gate of tests/tolerances.py applies
SPLIT_PRECS = ["tf32x3", "fp16x3"]


@pytest.mark.parametrize("prec", SPLIT_PRECS)
@pytest.mark.parametrize("B,batch", [(8, 3), (32, 2), (64, 2)])
def test_paper_grid_split_precision_vs_oracle(prec, B, batch):
    from tolerances import SPLIT_TOL
    p = _plan(B, batch, prec)
    assert p.radii == 2 * B and p.sample_shape == (batch, 2 * B, 2 * B, 2 * B)
    assert p.coeff_shape == (batch, O.coeff_count(B)) and p.lib.sgl_num_functions(p.handle) == batch
    c = inputs.random_coeffs(B, batch, seed=2600 + B, decay=True)
    s = p.inverse(_dev(c, torch.complex64)).cpu().numpy()
    assert _err(s, O.inverse(c, B, rule="hermite")) < SPLIT_TOL
    rng = np.random.default_rng(2700 + B)
    shape = (batch, 2 * B, 2 * B, 2 * B)
    g = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    f = p.forward(_dev(g, torch.complex64)).cpu().numpy()
    assert _err(f, O.forward(g.astype(np.complex128), B, rule="hermite")) < SPLIT_TOL
    back = p.forward(_dev(O.inverse(c, B, rule="hermite"), torch.complex64)).cpu().numpy()
    assert _err(back, c) < SPLIT_TOL
    p.check()


@pytest.mark.parametrize("prec", SPLIT_PRECS)
def test_paper_grid_split_precision_adjoints_and_host_buffers(prec):
    from tolerances import SPLIT_TOL
    B, batch = 16, 2
    p = _plan(B, batch, prec)
    y = inputs.random_coeffs(B, batch, seed=2800)
    x = (np.random.default_rng(2801).standard_normal((batch, 2 * B, 2 * B, 2 * B)) + 0j).astype(np.complex64)
    a1 = p.adjoint(_dev(y, torch.complex64), of_inverse=False).cpu().numpy()
    assert _err(a1, O.adjoint_forward(y, B, rule="hermite")) < SPLIT_TOL
    a2 = p.adjoint(_dev(x, torch.complex64), of_inverse=True).cpu().numpy()
    assert _err(a2, O.adjoint_inverse(x.astype(np.complex128), B, rule="hermite")) < SPLIT_TOL
    # host buffers (whole-batch staging) give the device-buffer result bit for bit
    c = inputs.random_coeffs(B, batch, seed=2802).astype(np.complex64)
    dev = p.inverse(_dev(c, torch.complex64)).cpu()
    assert torch.equal(dev, p.inverse(torch.from_numpy(c)))
    assert torch.equal(p.forward(dev.cuda()).cpu(), p.forward(dev))
    p.check()


@pytest.mark.parametrize("prec", SPLIT_PRECS + ["bf16x3"])
@pytest.mark.parametrize("B,batch", [(8, 3), (32, 4), (64, 3)])
def test_paper_grid_split_precision_real_functions(prec, B, batch):
    # real functions on the paper's grid with a tensor-core precision: paired
    # into complex functions, each pair run as its two radial halves; odd
    # batches leave the last pair's second function empty
    from tolerances import SPLIT_TOL
    # BF16x3: 8 + 8 significant bits per pair, the gate of test_gpu_variants
    tol = 8 * 2.0 ** -16 if prec == "bf16x3" else SPLIT_TOL
    p = _plan(B, batch, prec, samples="real")
    assert p.sample_shape == (batch, 2 * B, 2 * B, 2 * B) and p.coeff_shape == (batch, O.coeff_count(B))
    g = np.random.default_rng(3000 + B).standard_normal((batch, 2 * B, 2 * B, 2 * B)).astype(np.float32)
    f = p.forward(_dev(g, torch.float32)).cpu().numpy()
    assert _err(f, O.forward(g.astype(np.float64), B, rule="hermite")) < tol
    c = inputs.random_coeffs(B, batch, seed=3100 + B, decay=True)
    s = p.inverse(_dev(c, torch.complex64)).cpu().numpy()
    assert s.dtype == np.float32
    assert _err(s, O.inverse(c, B, rule="hermite").real) < tol
    # adjoints: the real part of the complex adjoint of the forward, and the
    # complex adjoint of the inverse on real samples
    a1 = p.adjoint(_dev(c, torch.complex64), of_inverse=False).cpu().numpy().astype(np.float64)
    assert _err(a1, O.adjoint_forward(c, B, rule="hermite").real) < tol
    a2 = p.adjoint(_dev(g, torch.float32), of_inverse=True).cpu().numpy()
    assert _err(a2, O.adjoint_inverse(g.astype(np.complex128), B, rule="hermite")) < tol
    # host buffers give the device-buffer result bit for bit
    assert torch.equal(p.forward(torch.from_numpy(g)), torch.from_numpy(f))
    p.check()


def test_paper_grid_split_precision_real_b128():
    # B = 128 on 256 radii, TF32x3, three real functions (the last one
    # unpaired): its inverse against the oracle's real part, the forward of the
    # first function's samples against the oracle's forward
    from tolerances import SPLIT_TOL
    B = 128
    p = _plan(B, 3, "tf32x3", samples="real")
    c = inputs.random_coeffs(B, 3, seed=3200, decay=True).astype(np.complex64)
    s = p.inverse(torch.from_numpy(c).cuda())
    f = p.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    assert _err(s[2:], O.inverse(c[2].astype(np.complex128), B, rule="hermite").real) < SPLIT_TOL
    assert _err(f[:1], O.forward(s[0].astype(np.float64), B, rule="hermite")) < SPLIT_TOL
    p.check()


def test_paper_grid_split_precision_b128():
    # B = 128 on 256 radii, TF32x3: one function against the oracle, the round
    # trip of four, and bit-identical repeated calls
    from tolerances import SPLIT_TOL
    B = 128
    p = _plan(B, 4, "tf32x3")
    c = inputs.random_coeffs(B, 4, seed=2900, decay=True).astype(np.complex64)
    cd = torch.from_numpy(c).cuda()
    s = p.inverse(cd)
    f = p.forward(s)
    assert _err(f.cpu().numpy(), c) < SPLIT_TOL
    assert torch.equal(p.inverse(cd), s) and torch.equal(p.forward(s), f)
    s0 = s[0].cpu().numpy()
    assert _err(s0[None], O.inverse(c[0].astype(np.complex128), B, rule="hermite")) < SPLIT_TOL
    p.check()
