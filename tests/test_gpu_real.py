"""GPU parity of real-function plans (SGL_SAMPLES_REAL) against the FP64 oracle.

A real f has fhat_{n,l,-m} = (-1)^m conj(fhat_{n,l,m}) (Def 2.1; pinned on
the oracle in test_oracle_pins.test_real_function_symmetry).  The plans carry
two real functions as one complex function and separate the two coefficient
sets with that symmetry.  Checked here through the C ABI:
  forward   = the oracle's forward of the real samples (odd and even batches,
              so the last pair may have no second function);
  inverse   = the real part of the oracle's inverse, for any coefficients;
  adjoints  = the adjoint identities for the real inner product on samples
              and Re <u, v> on coefficients;
and the same numbers through host buffers.  Tolerances as for complex plans:
FP64 1e-12, FP32 2e-5, TF32x3 1e-6 (normwise per function; tests/tolerances.py).
"""
import numpy as np
import pytest

import oracle as O
from paper_1604_05140_gb300 import inputs
from tolerances import FP32_TOL, FP64_TOL, SPLIT_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": FP64_TOL, "fp32": FP32_TOL, "tf32x3": SPLIT_TOL}
RTYPE = {"fp64": torch.float64, "fp32": torch.float32, "tf32x3": torch.float32}
CTYPE = {"fp64": torch.complex128, "fp32": torch.complex64, "tf32x3": torch.complex64}


def _plan(B, batch, prec):
    from paper_1604_05140_gb300 import Plan
    return Plan(B, batch, prec, samples="real")


def _err(gpu, ref):
    g = np.asarray(gpu).reshape(np.shape(gpu)[0], -1)
    r = np.asarray(ref).reshape(np.shape(ref)[0], -1)
    return (np.abs(g - r).max(axis=1) / np.abs(r).max(axis=1)).max()


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


CASES = [("fp64", 5, 1), ("fp64", 8, 3), ("fp64", 16, 4), ("fp32", 8, 3), ("fp32", 24, 2),
         ("tf32x3", 8, 3), ("tf32x3", 16, 4), ("tf32x3", 64, 3)]


@pytest.mark.parametrize("prec,B,batch", CASES)
def test_real_forward_vs_oracle(prec, B, batch):
    p = _plan(B, batch, prec)
    assert p.n_samples == batch * 4 * B ** 3 and p.n_coeffs == batch * O.coeff_count(B)
    g = inputs.random_real((batch, B, 2 * B, 2 * B), seed=1200 + 10 * B + batch)
    f = p.forward(_dev(g, RTYPE[prec])).cpu().numpy()
    ref_in = g.astype(np.float32).astype(np.float64) if prec != "fp64" else g
    assert _err(f, O.forward(ref_in, B)) < TOL[prec]
    p.check()


@pytest.mark.parametrize("prec,B,batch", CASES)
def test_real_inverse_is_real_part(prec, B, batch):
    # any coefficients: the real part of the inverse transform
    p = _plan(B, batch, prec)
    c = inputs.random_coeffs(B, batch, seed=1300 + 10 * B + batch)
    s = p.inverse(_dev(c, CTYPE[prec])).cpu().numpy()
    assert s.dtype == (np.float64 if prec == "fp64" else np.float32)
    assert _err(s, O.inverse(c, B).real) < TOL[prec]
    p.check()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_real_round_trip(prec):
    # coefficients of real functions: forward(inverse(c)) = c
    B, batch = 16, 5
    p = _plan(B, batch, prec)
    g = inputs.random_real((batch, B, 2 * B, 2 * B), seed=1400)
    c = O.forward(g, B)                       # symmetric: coefficients of real functions
    s = p.inverse(_dev(c, CTYPE[prec]))
    assert _err(s.cpu().numpy(), O.inverse(c, B).real) < TOL[prec]
    back = p.forward(s).cpu().numpy()
    assert _err(back, c) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_real_adjoints(prec):
    # <F x, c> = x . F^H c  and  Re <c, I^H x> = x . I c  for real x
    B, batch = 12, 3
    p = _plan(B, batch, prec)
    x = inputs.random_real((batch, B, 2 * B, 2 * B), seed=1500)
    c = inputs.random_coeffs(B, batch, seed=1501)
    xd, cd = _dev(x, RTYPE[prec]), _dev(c, CTYPE[prec])
    fx = p.forward(xd).cpu().numpy().astype(np.complex128)
    fhc = p.adjoint(cd, of_inverse=False).cpu().numpy().astype(np.float64)
    bound = 10 * TOL[prec] * (np.abs(fx).max() * np.abs(c).sum() + np.abs(fhc).max() * np.abs(x).sum())
    lhs, rhs = np.real(np.vdot(fx, c)), np.sum(x * fhc)
    assert abs(lhs - rhs) < bound
    # against the oracle: the real part of the complex adjoint
    assert _err(fhc, O.adjoint_forward(c, B).real) < TOL[prec]
    ic = p.inverse(cd).cpu().numpy().astype(np.float64)
    ihx = p.adjoint(xd, of_inverse=True).cpu().numpy().astype(np.complex128)
    bound = 10 * TOL[prec] * (np.abs(ic).max() * np.abs(x).sum() + np.abs(ihx).max() * np.abs(c).sum())
    lhs, rhs = np.sum(x * ic), np.real(np.vdot(ihx, c))
    assert abs(lhs - rhs) < bound
    assert _err(ihx, O.adjoint_inverse(x.astype(np.complex128), B)) < TOL[prec]
    p.check()


def test_real_host_buffers_match_device_buffers():
    B, batch = 16, 3
    p = _plan(B, batch, "tf32x3")
    g = inputs.random_real((batch, B, 2 * B, 2 * B), seed=1600).astype(np.float32)
    dev = p.forward(_dev(g, torch.float32)).cpu()
    host = p.forward(torch.from_numpy(g))
    assert torch.equal(dev, host)
    s_dev = p.inverse(dev.cuda()).cpu()
    s_host = p.inverse(dev)
    assert torch.equal(s_dev, s_host)


def test_real_full_size_b128():
    # B=128, 65 real functions (an unpaired last one), decaying spectra: the
    # first and the last with coefficients of real functions (symmetrised)
    # checked against the oracle, all of them through the round trip, which
    # returns the symmetric part of arbitrary coefficients
    B, NB = 128, 65
    p = _plan(B, NB, "tf32x3")
    c = inputs.random_coeffs(B, NB, seed=1700, decay=True)
    sym = 0.5 * (c + _mirror(c, B))
    c[0], c[-1] = sym[0], sym[-1]
    s = p.inverse(_dev(c, torch.complex64))
    f = p.forward(s).cpu().numpy()
    s = s.cpu().numpy()
    assert _err(f, sym) < TOL["tf32x3"]
    for k in (0, NB - 1):
        ref = O.inverse(sym[k], B)
        assert np.abs(ref.imag).max() < 1e-12 * np.abs(ref).max()
        assert _err(s[k][None], ref.real) < TOL["tf32x3"], k
    p.check()


def _mirror(c, B):
    """S(c)_{n,l,m} = (-1)^m conj(c_{n,l,-m})."""
    out = np.empty_like(c)
    for n in range(1, B + 1):
        for l in range(n):
            ms = np.arange(-l, l + 1)
            base = O.omega(n, l, 0)
            out[:, base + ms] = ((-1.0) ** np.abs(ms)) * np.conj(c[:, base - ms])
    return out


def test_real_misaligned_pointers_are_rejected():
    from paper_1604_05140_gb300 import sgl
    B = 8
    p = _plan(B, 2, "tf32x3")
    raw = torch.zeros(p.n_samples + 4, dtype=torch.float32, device="cuda")
    c = torch.zeros(p.n_coeffs + 2, dtype=torch.complex64, device="cuda")
    # samples need only the real type's alignment; coefficients the complex one
    assert p.lib.sgl_forward(p.handle, raw.data_ptr() + 4, c.data_ptr(), None) == sgl.SGL_OK
    assert p.lib.sgl_forward(p.handle, raw.data_ptr() + 2, c.data_ptr(), None) == sgl.SGL_ERR_ARG
    assert p.lib.sgl_forward(p.handle, raw.data_ptr(), c.data_ptr() + 4, None) == sgl.SGL_ERR_ARG
    torch.cuda.synchronize()
    p.check()
