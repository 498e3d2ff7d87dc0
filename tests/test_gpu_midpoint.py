"""GPU parity of the Cartesian midpoint rule (sgl_midpoint) against the oracle.

sgl_midpoint is the practice the paper's Discussion describes (midpoint
quadrature of the inner product Eq. inner_product on a Cartesian grid), built
to compare accuracy and cost with the SGL transform.  The oracle sums the same
rule with the closed-form basis (pinned against the closed-form coefficients
in test_oracle_pins); the kernel builds the basis by the recurrences.  FP64
gate 1e-12 (relative to the largest coefficient), FP32 1e-5; the kernel
accumulates with atomic adds, so only the last bits may differ between runs.
"""
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f(M, L, seed):
    # a smooth complex test function: a polynomial of degree 3 (its SGL
    # expansion is finite) plus a shifted Gaussian (not band-limited)
    x, y, z, _ = O.cartesian_midpoints(M, L)
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    return (a[0] + a[1] * x + a[2] * y * z + a[3] * z ** 3
            + a[4] * np.exp(-((x - 0.5) ** 2 + y ** 2 + (z + 0.3) ** 2)) + a[5] * (x * x + y * y))


@pytest.mark.parametrize("B,M,batch", [(1, 6, 1), (2, 8, 2), (4, 10, 2), (6, 12, 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_midpoint_vs_oracle(B, M, batch, prec):
    from paper_1604_05140_gb300 import midpoint
    L = 5.0
    f = np.stack([_f(M, L, 10 * B + k) for k in range(batch)])
    ref = O.midpoint(f, B, M, L)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    got = midpoint(torch.from_numpy(f).to(dt).cuda(), B, L).cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < tol * np.abs(ref).max()


def test_midpoint_converges_to_closed_forms():
    # on [-6, 6]^3 with M = 40 the rule reproduces the closed-form coefficients
    # of 1, x, y, z, r^2 (fast convergence for Gaussian-weighted polynomials)
    from paper_1604_05140_gb300 import midpoint
    B, M, L = 3, 40, 6.0
    x, y, z, _ = O.cartesian_midpoints(M, L)
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, n, l, m, re_, im_ = line.split()
            rows.append((name, int(n), int(l), int(m), complex(float(re_), float(im_))))
    funcs = {"one": np.ones_like(x), "x": x, "y": y, "z": z, "r2": x * x + y * y + z * z}
    f = np.stack([funcs[k] for k in funcs]) + 0j
    got = midpoint(torch.from_numpy(f).cuda(), B, L).cpu().numpy()
    for k, name in enumerate(funcs):
        expect = np.zeros(O.coeff_count(B), dtype=np.complex128)
        for (nm, n, l, m, v) in rows:
            if nm == name:
                expect[O.omega(n, l, m)] = v
        assert np.abs(got[k] - expect).max() < 1e-11, name


def test_midpoint_rejects_host_and_misaligned_pointers():
    from paper_1604_05140_gb300 import sgl
    lib = sgl.load_library()
    f = torch.zeros((1, 4, 4, 4), dtype=torch.complex128, device="cuda")
    c = torch.zeros((1, 5 + 1), dtype=torch.complex128, device="cuda")
    host = torch.zeros((1, 4, 4, 4), dtype=torch.complex128)
    assert lib.sgl_midpoint(2, 4, 3.0, 1, sgl.SGL_FP64, host.data_ptr(), c.data_ptr(), None) == sgl.SGL_ERR_ARG
    assert lib.sgl_midpoint(2, 4, 3.0, 1, sgl.SGL_FP64, f.data_ptr() + 8, c.data_ptr(), None) == sgl.SGL_ERR_ARG
    assert lib.sgl_midpoint(2, 4, 3.0, 1, sgl.SGL_FP64, f.data_ptr(), c.data_ptr(), None) == sgl.SGL_OK
    torch.cuda.synchronize()
