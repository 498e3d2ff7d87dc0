"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Error measure: per function, max |gpu - oracle| / max |oracle| over all of the
function's outputs (normwise).  Tolerances:
  FP64 plans  1e-12 (the FP64 target; round-off of the same sums in another
              order is ~1e-15 * sqrt(terms))
  FP32 plans  2e-5  (FP32 unit round-off 6e-8 times the ~sqrt(2B)*log2(2B)
              growth of three chained sums of up to 2B terms, with margin)
  TF32x3      1e-6  (the split-precision bound itself)
(tests/tolerances.py derives each.)
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs
from tolerances import FP32_TOL, FP64_TOL, SPLIT_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plan(*a, **k):
    from paper_1604_05140_gb300 import Plan
    return Plan(*a, **k)


def _err(gpu, ref, axis_batch=True):
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    if axis_batch:
        g = gpu.reshape(gpu.shape[0], -1)
        r = ref.reshape(ref.shape[0], -1)
        return (np.abs(g - r).max(axis=1) / np.abs(r).max(axis=1)).max()
    return np.abs(gpu - ref).max() / np.abs(ref).max()


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


BS = [1, 2, 3, 4, 5, 7, 8, 12, 16, 24, 32]


@pytest.mark.parametrize("B", BS)
@pytest.mark.parametrize("batch", [1, 3])
def test_fp64_inverse_and_forward_vs_oracle(B, batch):
    p = _plan(B, batch, "fp64")
    c = inputs.random_coeffs(B, batch, seed=1000 + B)
    s_ref = O.inverse(c, B)
    s_gpu = p.inverse(_dev(c, torch.complex128)).cpu().numpy()
    assert _err(s_gpu, s_ref) < FP64_TOL
    # forward of arbitrary (non-bandlimited) samples: the quadrature itself
    g = inputs.random_samples(B, batch, seed=2000 + B)
    f_ref = O.forward(g, B)
    f_gpu = p.forward(_dev(g, torch.complex128)).cpu().numpy()
    assert _err(f_gpu, f_ref) < FP64_TOL
    # round trip (sampling theorem)
    back = p.forward(_dev(s_ref, torch.complex128)).cpu().numpy()
    assert _err(back, c) < FP64_TOL


def test_fp64_b8_vs_direct_quadrature():
    # B=8, one function, c ~ complex normal: inverse, then forward, against
    # the direct O(B^7) sums of Algorithms 1/2
    B = 8
    c = inputs.random_coeffs(B, 1, seed=inputs.BASE_SEED + 1)
    p = _plan(B, 1, "fp64")
    s_gpu = p.inverse(_dev(c, torch.complex128))
    assert _err(s_gpu.cpu().numpy(), O.inverse_direct(c, B)) < FP64_TOL
    f_gpu = p.forward(s_gpu).cpu().numpy()
    assert _err(f_gpu, O.forward_direct(s_gpu.cpu().numpy(), B)) < FP64_TOL
    assert _err(f_gpu, c) < FP64_TOL


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_b64_decaying_spectrum(prec, tol):
    # B=64, one function, c/n decay: round trip and forward of synthesized data
    B = 64
    c = inputs.random_coeffs(B, 1, seed=inputs.BASE_SEED + 2, decay=True)
    p = _plan(B, 1, prec)
    dt = p.dtype
    s_ref = O.inverse(c, B)
    s_gpu = p.inverse(_dev(c, dt)).cpu().numpy()
    assert _err(s_gpu, s_ref) < tol
    f_gpu = p.forward(_dev(s_ref, dt)).cpu().numpy()
    assert _err(f_gpu, c) < tol
    assert _err(f_gpu, O.forward(s_ref.astype(np.complex64 if prec == "fp32" else np.complex128), B)) < tol


@pytest.mark.parametrize("B", [3, 8, 16, 24])
def test_fp32_vs_oracle(B):
    p = _plan(B, 2, "fp32")
    c = inputs.random_coeffs(B, 2, seed=3000 + B)
    s_gpu = p.inverse(_dev(c, torch.complex64)).cpu().numpy()
    assert _err(s_gpu, O.inverse(c, B)) < FP32_TOL
    g = inputs.random_samples(B, 2, seed=4000 + B)
    f_gpu = p.forward(_dev(g, torch.complex64)).cpu().numpy()
    assert _err(f_gpu, O.forward(g.astype(np.complex64), B)) < FP32_TOL


@pytest.mark.parametrize("B", list(range(16, 129, 8)))
def test_fp32_register_fft_every_size(B):
    # 2B = 16 N2 with N2 = 2 .. 16: every size of the register phi-FFT (radix
    # 2 for powers of two, mixed radix otherwise), both directions, against
    # the oracle
    p = _plan(B, 1, "fp32")
    c = inputs.random_coeffs(B, 1, seed=7700 + B)
    assert _err(p.inverse(_dev(c, torch.complex64)).cpu().numpy(), O.inverse(c, B)) < FP32_TOL
    g = inputs.random_samples(B, 1, seed=7800 + B)
    assert _err(p.forward(_dev(g, torch.complex64)).cpu().numpy(), O.forward(g.astype(np.complex64), B)) < FP32_TOL
    p.check()


@pytest.mark.parametrize("B", [5, 12])
def test_fp64_adjoints_vs_oracle(B):
    p = _plan(B, 2, "fp64")
    y = inputs.random_coeffs(B, 2, seed=5000 + B)
    x = inputs.random_samples(B, 2, seed=6000 + B)
    a1 = p.adjoint(_dev(y, torch.complex128), of_inverse=False).cpu().numpy()
    assert _err(a1, O.adjoint_forward(y, B)) < FP64_TOL
    a2 = p.adjoint(_dev(x, torch.complex128), of_inverse=True).cpu().numpy()
    assert _err(a2, O.adjoint_inverse(x, B)) < FP64_TOL
    # dot tests of the GPU maps against each other
    fx = p.forward(_dev(x, torch.complex128)).cpu().numpy()
    lhs = np.vdot(y, fx)
    rhs = np.vdot(a1, x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_fp64_physical_samples_closed_forms():
    # plain f samples (SGL_SAMPLES_PHYSICAL): f = 1 and f = x against the
    # closed forms of Def 1.2 / Def 2.1
    B = 6
    p = _plan(B, 2, "fp64", samples="physical")
    r, th, ph, _, _ = p.grid(0)
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    one = np.ones_like(R) + 0j
    x = R * np.sin(TH) * np.cos(PH) + 0j
    f = p.forward(_dev(np.stack([one, x]), torch.complex128)).cpu().numpy()
    e = np.zeros_like(f)
    e[0, O.omega(1, 0, 0)] = np.pi ** 0.75
    e[1, O.omega(2, 1, -1)] = np.pi ** 0.75 / 2
    e[1, O.omega(2, 1, 1)] = -np.pi ** 0.75 / 2
    assert np.abs(f - e).max() < 1e-12
    # inverse returns plain values
    back = p.inverse(_dev(f, torch.complex128)).cpu().numpy()
    assert np.abs(back[1] - x).max() < 1e-11 * np.abs(x).max()


def test_grid_matches_oracle():
    B = 16
    p = _plan(B, 1, "fp64")
    r, th, ph, wr, wt = p.grid(0)
    r0, th0, ph0, wr0, wt0 = O.grid(B)
    for a, b in [(r, r0), (th, th0), (ph, ph0), (wr, wr0), (wt, wt0)]:
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-300)


def test_host_buffers_match_device_buffers():
    B = 12
    p = _plan(B, 2, "fp64")
    c = inputs.random_coeffs(B, 2, seed=77)
    ch = torch.from_numpy(c.copy())            # pageable host
    cp = torch.from_numpy(c.copy()).pin_memory()  # pinned host
    s_dev = p.inverse(_dev(c, torch.complex128)).cpu()
    s_host = p.inverse(ch)
    assert not s_host.is_cuda
    s_pin = p.inverse(cp)
    assert torch.equal(s_host, s_dev)
    assert torch.equal(s_pin, s_dev)
    f_host = p.forward(s_host)
    f_dev = p.forward(s_dev.cuda()).cpu()
    assert torch.equal(f_host, f_dev)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_host_buffers_in_sub_batches_match_device_buffers(prec):
    # 17 functions: host-buffer calls run in chunks of 3 functions and a last
    # chunk of 2, the copies of one chunk overlapping the kernels of the
    # previous one; every function's arithmetic is the same as in the
    # whole-batch launch
    B, NB = 16, 17
    p = _plan(B, NB, prec)
    dt = p.dtype
    c = inputs.random_coeffs(B, NB, seed=78)
    s_dev = p.inverse(_dev(c, dt))
    s_pin = p.inverse(torch.from_numpy(c).to(dt).pin_memory())
    assert not s_pin.is_cuda and torch.equal(s_pin, s_dev.cpu())
    f_dev = p.forward(s_dev)
    f_host = p.forward(s_pin)                       # host in, host out
    f_mixed = p.forward(s_dev, out=torch.empty(p.coeff_shape, dtype=dt).pin_memory())  # device in, host out
    assert torch.equal(f_host, f_dev.cpu()) and torch.equal(f_mixed, f_dev.cpu())
    a_dev = p.adjoint(f_dev, of_inverse=False)
    a_host = p.adjoint(f_dev.cpu().pin_memory(), of_inverse=False)
    assert torch.equal(a_host, a_dev.cpu())
    p.check()


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32", FP32_TOL)])
def test_uneven_bandlimits_plan(prec, tol):
    from paper_1604_05140_gb300 import Plan
    Bs = [8, 16, 3, 12, 16, 24, 8]
    p = Plan.many(Bs, precision=prec)
    cs = [inputs.random_coeffs(B, 1, seed=900 + k)[0] for k, B in enumerate(Bs)]
    flat = np.concatenate(cs)
    s = p.inverse(_dev(flat, p.dtype))
    f = p.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    for k, B in enumerate(Bs):
        so, co = p.sample_offset(k), p.coeff_offset(k)
        sk = s[so:so + 4 * B ** 3].reshape(1, B, 2 * B, 2 * B)
        assert _err(sk, O.inverse(cs[k], B)) < tol, (k, B)
        fk = f[co:co + O.coeff_count(B)]
        assert _err(fk[None], cs[k][None]) < tol, (k, B)


def test_full_size_b128_sampled_functions_fp64():
    # B=128, batch 64 in the benchmark's launch configuration; the oracle
    # checks two of the 64 functions completely
    B, NB = 128, 64
    p = _plan(B, NB, "fp64")
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 3, decay=True)
    s = p.inverse(_dev(c, torch.complex128))
    f = p.forward(s).cpu().numpy()
    assert _err(f, c) < FP64_TOL
    for k in (0, NB - 1):
        sk = s[k].cpu().numpy()
        assert _err(sk[None], O.inverse(c[k], B)) < FP64_TOL
        assert _err(f[k][None], O.forward(sk, B)) < FP64_TOL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("B", [40, 104])
def test_simt_tile_shapes_vs_oracle(prec, B):
    # every SIMT tile shape (64, 48, 32 and 16 columns) in every stage: at
    # B = 104 the radial stages and the Legendre synthesis cover 104 columns
    # with a 64-column block and a 48-column tile, the forward Legendre groups
    # have up to 52 columns; at B = 40 the synthesis and the inverse radial
    # stage take one 48-column tile.  Coefficients without decay, so that the
    # high degrees weigh as much as the low ones.
    NB = 2
    p = _plan(B, NB, prec)
    ctype = torch.complex128 if prec == "fp64" else torch.complex64
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    c = inputs.random_coeffs(B, NB, seed=7000 + B)
    if prec == "fp32":
        c = c.astype(np.complex64).astype(np.complex128)
    s = p.inverse(_dev(c, ctype))
    s_ref = O.inverse(c[0], B)
    assert _err(s[0].cpu().numpy()[None], s_ref) < tol
    g = O.inverse(c[1], B)
    if prec == "fp32":
        g = g.astype(np.complex64).astype(np.complex128)
    f = p.forward(_dev(np.concatenate([s_ref, g]), ctype)).cpu().numpy()
    assert _err(f[1:], O.forward(g, B)) < tol
    assert _err(f, c) < tol
    assert _err(p.forward(s).cpu().numpy(), c) < tol


def test_inputs_not_modified():
    B = 8
    p = _plan(B, 1, "fp64")
    c = _dev(inputs.random_coeffs(B, 1, seed=5), torch.complex128)
    c0 = c.clone()
    s = p.inverse(c)
    s0 = s.clone()
    p.forward(s)
    assert torch.equal(c, c0) and torch.equal(s, s0)


@pytest.mark.parametrize("prec,ctype", [("fp64", torch.complex128), ("tf32x3", torch.complex64)])
def test_misaligned_device_pointers_are_rejected(prec, ctype):
    # the kernels move whole complex values: a device pointer off the complex
    # element's alignment is an argument error, found before any launch, and
    # the plan keeps working
    from paper_1604_05140_gb300 import sgl
    B = 8
    p = _plan(B, 1, prec)
    c = _dev(inputs.random_coeffs(B, 1, seed=6), ctype)
    s = p.inverse(c)
    raw = torch.empty(2 * s.numel() + 8, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    shift = raw.element_size()  # one real past the complex alignment
    st = p.lib.sgl_forward(p.handle, raw.data_ptr() + shift, c.data_ptr(), None)
    assert st == sgl.SGL_ERR_ARG
    st = p.lib.sgl_inverse(p.handle, c.data_ptr(), raw.data_ptr() + shift, None)
    assert st == sgl.SGL_ERR_ARG
    torch.cuda.synchronize()
    back = p.forward(s)
    tol = FP64_TOL if prec == "fp64" else SPLIT_TOL
    assert _err(back.cpu().numpy(), c.cpu().numpy()) < tol


# ---------------------------------------------------------------------------
# split precision: TF32x3 tensor-core stages
# ---------------------------------------------------------------------------
TF32X3_TOL = SPLIT_TOL  # three TF32 products (2^-22 per dropped term), FP32 accumulation and FFT


@pytest.mark.parametrize("B", [4, 8, 16, 24, 32, 64])
def test_tf32x3_vs_oracle(B):
    p = _plan(B, 3, "tf32x3")
    c = inputs.random_coeffs(B, 3, seed=7000 + B)
    s_gpu = p.inverse(_dev(c, torch.complex64)).cpu().numpy()
    assert _err(s_gpu, O.inverse(c, B)) < TF32X3_TOL
    g = inputs.random_samples(B, 3, seed=8000 + B)
    f_gpu = p.forward(_dev(g, torch.complex64)).cpu().numpy()
    assert _err(f_gpu, O.forward(g.astype(np.complex64), B)) < TF32X3_TOL
    back = p.forward(_dev(O.inverse(c, B), torch.complex64)).cpu().numpy()
    assert _err(back, c) < TF32X3_TOL
    p.check()


def test_tf32x3_adjoints_vs_oracle():
    B = 16
    p = _plan(B, 2, "tf32x3")
    y = inputs.random_coeffs(B, 2, seed=9100)
    x = inputs.random_samples(B, 2, seed=9200)
    a1 = p.adjoint(_dev(y, torch.complex64), of_inverse=False).cpu().numpy()
    assert _err(a1, O.adjoint_forward(y, B)) < TF32X3_TOL
    a2 = p.adjoint(_dev(x, torch.complex64), of_inverse=True).cpu().numpy()
    assert _err(a2, O.adjoint_inverse(x.astype(np.complex64), B)) < TF32X3_TOL


def test_tf32x3_uneven_bandlimits():
    from paper_1604_05140_gb300 import Plan
    Bs = [16, 40, 8, 24, 40, 64, 16, 128]
    p = Plan.many(Bs, precision="tf32x3")
    cs = [inputs.random_coeffs(B, 1, seed=950 + k)[0] for k, B in enumerate(Bs)]
    s = p.inverse(_dev(np.concatenate(cs), torch.complex64))
    f = p.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    for k, B in enumerate(Bs):
        so, co = p.sample_offset(k), p.coeff_offset(k)
        sk = s[so:so + 4 * B ** 3].reshape(1, B, 2 * B, 2 * B)
        assert _err(sk, O.inverse(cs[k], B)) < TF32X3_TOL, (k, B)
        assert _err(f[co:co + O.coeff_count(B)][None], cs[k][None]) < TF32X3_TOL, (k, B)
    p.check()


def test_tf32x3_full_size_b128_sampled_functions():
    # B=128, batch 64, the benchmark configuration; two functions checked
    # completely against the oracle, all 64 through the round trip
    B, NB = 128, 64
    p = _plan(B, NB, "tf32x3")
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 3, decay=True)
    s = p.inverse(_dev(c, torch.complex64))
    f = p.forward(s).cpu().numpy()
    assert _err(f, c) < TF32X3_TOL
    for k in (0, NB - 1):
        sk = s[k].cpu().numpy()
        assert _err(sk[None], O.inverse(c[k], B)) < TF32X3_TOL
        assert _err(f[k][None], O.forward(sk, B)) < TF32X3_TOL
    p.check()


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
def test_repeated_calls_are_bit_identical(prec):
    # B=128, 128 functions: every tile's arithmetic is fixed, whichever CTA
    # takes it from the work queue and whenever, so repeated calls on the same
    # input give the same bits; a race between the pipeline roles (a ring
    # slot refilled before its reader is done with it) shows up here as
    # differing rows of a few tiles
    B, NB = 128, 128
    p = _plan(B, NB, prec)
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 12, decay=True).astype(np.complex64)
    cd = torch.from_numpy(c).cuda()
    s = p.inverse(cd)
    f = p.forward(s)
    for _ in range(3):
        assert torch.equal(p.inverse(cd), s)
        assert torch.equal(p.forward(s), f)
    p.check()
    del s, f, cd
    torch.cuda.empty_cache()


def test_tf32x3_b128_batch256_offsets_beyond_2_31():
    # B=128, 256 functions: the phi-FFT spectra alone hold 4.3e9 floats
    # (beyond 2^31), so every offset of the path must be 64-bit.  Round trip
    # of all 256 functions; the first and the last also against a plan of one
    # function on the same coefficients (same arithmetic per function).
    B, NB = 128, 256
    p = _plan(B, NB, "tf32x3")
    c = inputs.random_coeffs(B, NB, seed=inputs.BASE_SEED + 11, decay=True).astype(np.complex64)
    cd = torch.from_numpy(c).cuda()
    s = p.inverse(cd)
    f = p.forward(s)
    p.check()
    assert _err(f.cpu().numpy(), c) < TF32X3_TOL
    one = _plan(B, 1, "tf32x3")
    for k in (0, NB - 1):
        s1 = one.inverse(cd[k:k + 1])
        assert _err(s[k:k + 1].cpu().numpy(), s1.cpu().numpy()) < 1e-6, k
    del s, f, cd
    torch.cuda.empty_cache()

