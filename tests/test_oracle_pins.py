"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
coefficients (Def 1.2, Def 2.1), the B = 1 rule, the weight identities of
Thm 3.1 / Lemma 3.2, the explicit Laguerre sum (Eq. associated_laguerre_explicit)
and the Rodrigues form of Def 2.1, discrete orthonormality (Thm 3.1, the
radial Gram identity of Sect. 3.3.2), brute force (Algorithms 1/2), the sampling
theorem (Thm 3.4), an independent Cartesian Gauss-Hermite quadrature of the
inner product Eq. (inner_product), library routines (SciPy) where present, and
the adjoint identities of Sect. 3.4.  The last tests plant mistakes in the
oracle and check that a pin catches each of them.
"""
import os
from math import gamma, lgamma, pi, sqrt

import numpy as np
import pytest

import oracle as O
from oracle import sgl_oracle as OM
from paper_1604_05140_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cartesian(B, rule="laguerre"):
    r, th, ph, _, _ = O.grid(B, rule)
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    return R * np.sin(TH) * np.cos(PH), R * np.sin(TH) * np.sin(PH), R * np.cos(TH), R


def _closed_forms():
    rows = []
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, n, l, m, re, im = line.split()
            rows.append((name, int(n), int(l), int(m), complex(float(re), float(im))))
    return rows


@pytest.mark.parametrize("B", [2, 3, 5])
def test_closed_form_coefficients(B):
    x, y, z, R = _cartesian(B)
    funcs = {"one": np.ones_like(x), "z": z, "x": x, "y": y, "r2": R ** 2}
    table = _closed_forms()
    for name, f in funcs.items():
        fh = O.forward(O.physical_to_weighted(f + 0j, B), B)[0]
        expect = np.zeros_like(fh)
        for (nm, n, l, m, v) in table:
            if nm == name:
                expect[O.omega(n, l, m)] = v
        np.testing.assert_allclose(fh, expect, atol=1e-13, rtol=0, err_msg=name)


@pytest.mark.parametrize("B", [3, 5])
def test_closed_form_coefficients_paper_grid(B):
    # the same closed forms from samples on the paper's own grid: 2B
    # half-range Gauss-Hermite radii (Thm 3.3, Eq. zwischenstufe_2)
    x, y, z, R = _cartesian(B, "hermite")
    assert x.shape == (2 * B, 2 * B, 2 * B)
    funcs = {"one": np.ones_like(x), "z": z, "x": x, "y": y, "r2": R ** 2}
    table = _closed_forms()
    for name, f in funcs.items():
        fh = O.forward(O.physical_to_weighted(f + 0j, B, "hermite"), B, rule="hermite")[0]
        expect = np.zeros_like(fh)
        for (nm, n, l, m, v) in table:
            if nm == name:
                expect[O.omega(n, l, m)] = v
        np.testing.assert_allclose(fh, expect, atol=1e-13, rtol=0, err_msg=name)


@pytest.mark.parametrize("N", [1, 2, 7, 32, 128, 256])
def test_half_range_hermite_rule(N):
    # Thm 3.3: the N-point Gauss rule for e^{-r^2} on [0, inf) has simple
    # positive nodes, positive weights, and integrates r^k exactly for
    # k <= 2N - 1: int_0^inf r^k e^{-r^2} dr = Gamma((k+1)/2) / 2.  Such a rule
    # is unique, so these moments pin it.  Sums in logarithms (the weights
    # reach e^{-650} at N = 256).
    r, loga = O.half_range_hermite_rule(N)
    assert r[0] > 0 and np.all(np.diff(r) > 0) and np.all(np.isfinite(loga))
    for k in range(2 * N):
        terms = loga + k * np.log(r)
        mx = terms.max()
        lhs = mx + np.log(np.exp(terms - mx).sum())
        rhs = lgamma((k + 1) / 2) - np.log(2.0)
        assert abs(lhs - rhs) < 2e-15 * max(1.0, abs(rhs)), (k, lhs, rhs)
    if N == 1:  # one node: r_0 = mu_1 / mu_0 = 1/sqrt(pi), a_0 = mu_0 = sqrt(pi)/2
        assert abs(r[0] - 1 / sqrt(pi)) < 1e-15 and abs(np.exp(loga[0]) - sqrt(pi) / 2) < 1e-15


@pytest.mark.parametrize("B", [2, 3, 4])
def test_paper_grid_direct_equals_separated(B):
    # Algorithms 1/2 (brute force over the 8B^3 grid) against the separated
    # stages on the paper's grid
    c = inputs.random_coeffs(B, 2, seed=210 + B)
    s = O.inverse(c, B, rule="hermite")
    assert s.shape == (2, 2 * B, 2 * B, 2 * B)
    np.testing.assert_allclose(O.inverse_direct(c, B, rule="hermite"), s, atol=1e-13 * np.abs(s).max())
    g = np.random.default_rng(230 + B).standard_normal((2, 2 * B, 2 * B, 2 * B)) + 0j
    f = O.forward(g, B, rule="hermite")
    np.testing.assert_allclose(O.forward_direct(g, B, rule="hermite"), f, atol=1e-13 * np.abs(f).max())


@pytest.mark.parametrize("B", [2, 4, 8, 16, 32])
def test_sampling_theorem_round_trip_paper_grid(B):
    # Thm 3.4 on the paper's own grid, at the error scale of its Table 1
    # (which was measured on that grid)
    c = inputs.random_coeffs(B, 3, seed=300 + B, dist="uniform")
    back = O.forward(O.inverse(c, B, rule="hermite"), B, rule="hermite")
    err = np.abs(back - c).max(axis=1)
    am, asd, _, _ = _paper_table1()[B]
    assert err.mean() < 10 * (am + 3 * asd), (err, am)


@pytest.mark.parametrize("name", ["one", "x", "y", "z", "r2"])
def test_midpoint_rule_converges_to_closed_forms(name):
    # the midpoint rule of the Discussion, applied to the inner product Eq.
    # (inner_product) on [-6, 6]^3: for these Gaussian-weighted polynomials it
    # converges (fast) to the closed-form coefficients; a wrong weight, volume
    # element or conjugation would not
    B = 3
    table = [r for r in _closed_forms() if r[0] == name]
    errs = []
    for M in (12, 40):
        x, y, z, _ = O.cartesian_midpoints(M, 6.0)
        f = {"one": np.ones_like(x), "x": x, "y": y, "z": z, "r2": x * x + y * y + z * z}[name]
        c = O.midpoint(f[None] + 0j, B, M, 6.0)[0]
        expect = np.zeros_like(c)
        for (_, n, l, m, v) in table:
            expect[O.omega(n, l, m)] = v
        errs.append(np.abs(c - expect).max())
    assert errs[1] < 1e-11 and errs[0] > 1e3 * errs[1], errs


@pytest.mark.parametrize("B", [3, 6, 16])
def test_dct_truncation_property(B):
    # Eq. (DCT): C_2B is orthogonal, and the DCT of a cosine polynomial of
    # degree d on the 2B rings vanishes beyond index d.  Lambda_lm / w_m is one
    # of degree l (even m) or l - 1 (odd m, w_m = sin theta): this pins the
    # Legendre table's theta dependence and the odd-m reading of the
    # seminaive algorithm.
    C = O.dct_matrix(2 * B)
    np.testing.assert_allclose(C @ C.T, np.eye(2 * B), atol=1e-14)
    Q = O.legendre_cosine_coeffs(B)
    for m in range(B):
        for l in range(m, B):
            deg = l if m % 2 == 0 else l - 1
            assert np.abs(Q[m, l, deg + 1:]).max(initial=0.0) < 1e-13 * np.abs(Q[m, l]).max(), (m, l)
            # the degree is reached (the top coefficient of sin^m is about 2^(1-m))
            assert abs(Q[m, l, deg]) > 1e-9 * np.abs(Q[m, l]).max(), (m, l)


@pytest.mark.parametrize("B", [2, 5, 12])
def test_seminaive_equals_direct(B):
    # the seminaive Legendre sums (Eq. dct_trick) give the forward transform of
    # the direct sums (Eq. DLT), with and without the quadrature weights
    g = inputs.random_samples(B, 2, seed=400 + B)
    for w in (True, False):
        a = O.forward(g, B, weights=w)
        b = O.forward_seminaive(g, B, weights=w)
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max(), w


def test_single_node_rule():
    t, logw = O.laguerre_rule(1)
    assert abs(t[0] - 1.5) < 1e-15
    assert abs(np.exp(logw[0]) - sqrt(pi) / 2) < 1e-15


@pytest.mark.parametrize("B", [1, 2, 3, 8, 64, 128])
def test_sphere_weights(B):
    _, _, beta = O.sphere_rule(B)
    b = beta * B / pi
    assert abs(b.sum() - 2.0) < 1e-12          # Thm 3.1 as printed
    assert abs(2 * B * beta.sum() - 4 * pi) < 1e-12  # sum over (j, k) is the area
    assert np.all(beta > 0)                      # Lemma 3.2


@pytest.mark.parametrize("B", [2, 5, 16, 64, 128])
def test_laguerre_rule_moments(B):
    # sum_i w_i t_i^p = Gamma(p + 3/2) for p <= 2B-1 (Gauss exactness), done in
    # logs for large p; and zeros of L_B^(1/2) by the explicit sum at small B.
    t, logw = O.laguerre_rule(B)
    for p in [0, 1, 2, B, 2 * B - 1]:
        e = logw + p * np.log(t)
        log_lhs = e.max() + np.log(np.exp(e - e.max()).sum())
        assert abs(log_lhs - lgamma(p + 1.5)) < 1e-11 * max(1.0, lgamma(p + 1.5)), p
    if B <= 16:
        # zeros of L_B^(1/2): the explicit sum vanishes up to the round-off of
        # its terms (scale = sum of |terms| at each node)
        val = O.laguerre_explicit(B, 0.5, t)
        scale = sum(np.exp(lgamma(B + 1.5) - lgamma(B - j + 1) - lgamma(j + 1.5) - lgamma(j + 1)) * t ** j
                    for j in range(B + 1))
        assert np.all(np.abs(val) < 1e-13 * scale)


def test_laguerre_rule_vs_scipy():
    sp = pytest.importorskip("scipy.special")
    for B in [4, 17, 64]:
        x, w = sp.roots_genlaguerre(B, 0.5)
        t, logw = O.laguerre_rule(B)
        np.testing.assert_allclose(t, x, rtol=1e-12)
        np.testing.assert_allclose(np.exp(logw), w, rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("B", [3, 8, 12])
def test_laguerre_orthogonality(B):
    # Thm 2.3 (Eq. laguerre_ortho) under the B-node rule, alpha = 1/2
    t, logw = O.laguerre_rule(B)
    w = np.exp(logw)
    L = np.array([O.laguerre_explicit(k, 0.5, t) for k in range(B)])
    G = (L * w[None, :]) @ L.T
    expect = np.diag([gamma(k + 1.5) / gamma(k + 1) for k in range(B)])
    np.testing.assert_allclose(G, expect, atol=1e-10 * expect.max())


@pytest.mark.parametrize("B", [4, 9])
def test_radial_table_vs_explicit_sum(B):
    # Lemma 3.7 (normalized reading) against N_nl L_{n-l-1}^{(l+1/2)}(r^2) r^l
    r, t, _ = O.radial_weights(B)
    T = O.radial_table(B)
    for l in range(B):
        for n in range(l + 1, B + 1):
            k = n - l - 1
            norm = sqrt(2 * gamma(k + 1) / gamma(n + 0.5))
            ref = norm * O.laguerre_explicit(k, l + 0.5, t) * r ** l * np.exp(-t / 2)
            np.testing.assert_allclose(T[l, n - 1], ref, atol=1e-11 * max(1, np.abs(ref).max()))


@pytest.mark.parametrize("B", [4, 11])
def test_legendre_table_vs_rodrigues(B):
    theta, _, _ = O.sphere_rule(B)
    lam = O.legendre_table(B)
    from math import factorial
    for m in range(B):
        for l in range(m, B):
            c = sqrt((2 * l + 1) / (4 * pi) * factorial(l - m) / factorial(l + m))
            ref = c * O.legendre_rodrigues(l, m, np.cos(theta))
            np.testing.assert_allclose(lam[m, l], ref, atol=1e-11)


def test_legendre_table_vs_scipy():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    B = 20
    theta, _, _ = O.sphere_rule(B)
    lam = O.legendre_table(B)
    for m in range(B):
        for l in range(m, B):
            ref = sp.sph_harm_y(l, m, theta, 0.0).real
            np.testing.assert_allclose(lam[m, l], ref, atol=1e-12)


@pytest.mark.parametrize("B", [8, 64, 128])
def test_radial_gram_identity(B):
    # R_l diag(a r^2) R_l^T = I  (Sect. 3.3.2), in the weighted form
    _, _, what = O.radial_weights(B)
    T = O.radial_table(B)
    for l in [0, 1, B // 3, B - 2, B - 1]:
        Tl = T[l, l:, :]
        G = (Tl * what[None, :]) @ Tl.T
        np.testing.assert_allclose(G, np.eye(B - l), atol=1e-14 * B)


@pytest.mark.parametrize("B", [8, 64])
def test_angular_gram_identity(B):
    # discrete orthonormality of Y_lm, l < B, under the sphere rule (Thm 3.1);
    # the phi sum makes orders orthogonal, so check each m separately
    _, _, beta = O.sphere_rule(B)
    lam = O.legendre_table(B)
    for m in [0, 1, B // 2, B - 1]:
        A = lam[m, m:, :]
        G = 2 * B * (A * beta[None, :]) @ A.T
        np.testing.assert_allclose(G, np.eye(B - m), atol=1e-13)


@pytest.mark.parametrize("B", [1, 2, 3, 4, 6, 8])
def test_direct_equals_separated(B):
    c = inputs.random_coeffs(B, 2, seed=11 + B)
    s_dir = O.inverse_direct(c, B)
    s_sep = O.inverse(c, B)
    np.testing.assert_allclose(s_sep, s_dir, atol=1e-13 * np.abs(s_dir).max())
    g = inputs.random_samples(B, 2, seed=17 + B)
    np.testing.assert_allclose(O.forward(g, B), O.forward_direct(g, B), atol=1e-12)


def _paper_table1():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_table1.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            B, am, asd, rm, rsd = line.split()
            rows[int(B)] = (float(am), float(asd), float(rm), float(rsd))
    return rows


@pytest.mark.parametrize("B", [2, 4, 8, 16, 32])
def test_sampling_theorem_round_trip(B):
    # Thm 3.4: forward(inverse(c)) = c for bandlimited data; the error is FP64
    # round-off of the size the paper reports in Table 1 (U[-1,1] coefficients)
    c = inputs.random_coeffs(B, 3, seed=100 + B, dist="uniform")
    back = O.forward(O.inverse(c, B), B)
    err = np.abs(back - c).max(axis=1)
    am, asd, _, _ = _paper_table1()[B]
    assert err.mean() < 10 * (am + 3 * asd), (err, am)


@pytest.mark.parametrize("B", [2, 3, 4, 5])
def test_cartesian_gauss_hermite(B):
    # <f, H_nlm>_H for a random complex polynomial of degree B-1 computed by a
    # tensor Gauss-Hermite rule in x, y, z (NumPy's hermgauss) with H_nlm from
    # the closed forms; the polynomial is bandlimited, so the SGL quadrature
    # must agree, and the inverse must reproduce its samples.
    from numpy.polynomial.hermite import hermgauss
    rng = np.random.default_rng(5 + B)
    D = B - 1
    mons = [(a, b, c) for a in range(D + 1) for b in range(D + 1) for c in range(D + 1) if a + b + c <= D]
    cf = rng.standard_normal(len(mons)) + 1j * rng.standard_normal(len(mons))

    def f(x, y, z):
        return sum(c * x ** a * y ** b * z ** e for c, (a, b, e) in zip(cf, mons))

    x, y, z, _ = _cartesian(B)
    fs = f(x, y, z)
    fh = O.forward(O.physical_to_weighted(fs, B), B)[0]
    N = B + D // 2 + 2
    xg, wg = hermgauss(N)
    X, Y, Z = np.meshgrid(xg, xg, xg, indexing="ij")
    W = wg[:, None, None] * wg[None, :, None] * wg[None, None, :]
    Rc = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    THc = np.arccos(np.clip(Z / np.where(Rc > 0, Rc, 1), -1, 1))
    PHc = np.arctan2(Y, X)
    F = f(X, Y, Z)
    ref = np.array([np.sum(W * F * np.conj(O.basis_explicit(n, l, m, Rc, THc, PHc)))
                    for (n, l, m) in O.nlm_list(B)])
    np.testing.assert_allclose(fh, ref, atol=1e-12 * np.abs(ref).max())
    back = O.weighted_to_physical(O.inverse(fh, B)[0], B)
    np.testing.assert_allclose(back, fs, atol=1e-12 * np.abs(fs).max())


@pytest.mark.parametrize("B", [3, 8])
def test_adjoint_identities(B):
    rng = np.random.default_rng(B)
    x = inputs.random_samples(B, 1, seed=30 + B)
    y = inputs.random_coeffs(B, 1, seed=40 + B)
    lhs = np.vdot(y, O.forward(x, B))
    rhs = np.vdot(O.adjoint_forward(y, B), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    lhs = np.vdot(x, O.inverse(y, B))
    rhs = np.vdot(O.adjoint_inverse(x, B), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # against the explicit matrices of Algorithms 1/2
    H = O.sgl_matrix(B)
    w = O.sample_weights(B).reshape(-1)
    np.testing.assert_allclose(O.adjoint_forward(y, B).reshape(-1), w * (y @ H).reshape(-1), atol=1e-12)
    np.testing.assert_allclose(O.adjoint_inverse(x, B).reshape(-1), (x.reshape(-1) @ np.conj(H).T), atol=1e-11)
    del rng


@pytest.mark.parametrize("B", [3, 6])
def test_real_function_symmetry(B):
    # Def 2.1: Y_l^{-m} = (-1)^m conj(Y_l^m) and the radial part is real, so
    # H_{n,l,-m} = (-1)^m conj(H_{n,l,m}) (closed forms, arbitrary points) ...
    rng = np.random.default_rng(60 + B)
    r, th, ph = rng.uniform(0.1, 3.0, 7), rng.uniform(0.0, pi, 7), rng.uniform(0.0, 2 * pi, 7)
    for n, l, m in [(2, 1, 1), (3, 2, 1), (3, 2, 2), (B, B - 1, B - 1)]:
        np.testing.assert_allclose(OM.basis_explicit(n, l, -m, r, th, ph),
                                   (-1) ** m * np.conj(OM.basis_explicit(n, l, m, r, th, ph)), atol=1e-13)
    # ... hence the coefficients of a real function obey
    # fhat_{n,l,-m} = (-1)^m conj(fhat_{n,l,m}), which the real-function plans use
    g = inputs.random_real((2, B, 2 * B, 2 * B), seed=70 + B)
    c = O.forward(g, B)
    trip = [(n, l, m) for n in range(1, B + 1) for l in range(n) for m in range(1, l + 1)]
    ip = [O.omega(n, l, m) for n, l, m in trip]
    im = [O.omega(n, l, -m) for n, l, m in trip]
    sign = np.array([(-1.0) ** m for _, _, m in trip])
    np.testing.assert_allclose(c[:, im], sign * np.conj(c[:, ip]), atol=1e-13 * np.abs(c).max())
    m0 = [O.omega(n, l, 0) for n in range(1, B + 1) for l in range(n)]
    assert np.abs(c[:, m0].imag).max() < 1e-13 * np.abs(c).max()
    # and the inverse of such coefficients is real
    s = O.inverse(c, B)
    assert np.abs(s.imag).max() < 1e-13 * np.abs(s).max()
    # the same on the paper's grid (2B half-range Gauss-Hermite radii): the
    # symmetry comes from the angular part alone, whatever the radial rule
    gh = inputs.random_real((2, 2 * B, 2 * B, 2 * B), seed=80 + B)
    ch = O.forward(gh, B, rule="hermite")
    np.testing.assert_allclose(ch[:, im], sign * np.conj(ch[:, ip]), atol=1e-13 * np.abs(ch).max())
    assert np.abs(ch[:, m0].imag).max() < 1e-13 * np.abs(ch).max()
    sh = O.inverse(ch, B, rule="hermite")
    assert np.abs(sh.imag).max() < 1e-13 * np.abs(sh).max()


def test_forward_then_inverse_is_projector():
    # R10: on arbitrary (non-bandlimited) samples inverse(forward(.)) is an
    # orthogonal projector in the w-weighted inner product
    B = 6
    g = inputs.random_samples(B, 1, seed=77)
    p1 = O.inverse(O.forward(g, B), B)
    p2 = O.inverse(O.forward(p1, B), B)
    np.testing.assert_allclose(p2, p1, atol=1e-12 * np.abs(p1).max())


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# ---------------------------------------------------------------------------

def _clear_caches():
    OM.legendre_table.cache_clear()
    OM.radial_table.cache_clear()
    OM.laguerre_rule.cache_clear()
    OM.half_range_hermite_rule.cache_clear()


def _closed_form_ok(B=3):
    try:
        test_closed_form_coefficients(B)
        return True
    except AssertionError:
        return False


def test_pins_catch_planted_mistakes(monkeypatch):
    assert _closed_form_ok()
    orig_sphere = OM.sphere_rule
    orig_fft = np.fft.fft

    # 1. sphere weights without the azimuthal factor pi/B (R2 dropped)
    def no_pi_over_b(B):
        th, ph, beta = orig_sphere(B)
        return th, ph, beta * B / pi
    monkeypatch.setattr(OM, "sphere_rule", no_pi_over_b)
    _clear_caches()
    assert not _closed_form_ok()
    monkeypatch.setattr(OM, "sphere_rule", orig_sphere)

    # 2. phi-DFT with the wrong sign
    monkeypatch.setattr(OM.np.fft, "fft", lambda a, axis=-1: np.conj(orig_fft(np.conj(a), axis=axis)))
    _clear_caches()
    assert not _closed_form_ok()
    monkeypatch.setattr(OM.np.fft, "fft", orig_fft)

    # 3. Legendre table without the Condon-Shortley phase
    orig_leg = OM.legendre_table.__wrapped__

    def no_cs(B):
        lam = orig_leg(B).copy()
        for m in range(1, B, 2):
            lam[m] = -lam[m]
        return lam
    monkeypatch.setattr(OM, "legendre_table", no_cs)
    no_cs.cache_clear = lambda: None
    assert not _closed_form_ok()
    monkeypatch.undo()
    _clear_caches()

    # 4. radial recurrence with a wrong sign on the three-term coupling
    orig_rad = OM.radial_table.__wrapped__

    def bad_radial(B, rule="laguerre"):
        T = orig_rad(B, rule).copy()
        T[:, 1::2, :] *= -1.0  # flips every second n: breaks the r^2 pin
        return T
    monkeypatch.setattr(OM, "radial_table", bad_radial)
    bad_radial.cache_clear = lambda: None
    assert not _closed_form_ok()
    monkeypatch.undo()
    _clear_caches()
    assert _closed_form_ok()
