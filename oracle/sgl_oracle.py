"""Plain FP64 CPU oracle for the spherical Gauss-Laguerre (SGL) Fourier transform.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
it is called by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``.  It shares no code with the CUDA library.

What it computes (Prestin & Wuelker, "Fast Fourier Transforms for Spherical
Gauss-Laguerre Basis Functions"):

* the SGL basis ``H_nlm = N_nl R_nl(r) Y_lm(theta, phi)`` (Def 1.2, Def 2.1),
  index set ``|m| <= l < n <= B`` (Cor 1.3);
* the quadrature of the SGL sampling theorem (Thm 3.4), i.e. the forward
  transform ``fhat_nlm = sum_{i,j,k} w_ijk f(x_ijk) conj(H_nlm(x_ijk))``, and
  the reconstruction (inverse) ``f(x) = sum fhat_nlm H_nlm(x)`` (Algorithm 2);
* the adjoints of both, from the matrix form of Sect. 3.4;
* the same forward transform with the Legendre sums taken by the seminaive
  algorithm (Eq. DCT, Eq. dct_trick; ``forward_seminaive``);
* the midpoint rule on a Cartesian grid that the Discussion describes as the
  current practice (``midpoint``), with the closed-form basis.

Readings taken where the paper is silent or differs from the grid used here
(each is listed in the design notes with its reason):

R1  radial rule: B generalized Gauss-Laguerre nodes in ``t = r^2`` with
    alpha = 1/2 (weight ``t^{1/2} e^{-t}``), so that
    ``int_0^inf p(r) r^2 e^{-r^2} dr = 1/2 sum_i w_i p(sqrt(t_i))``; exact for
    the bandlimit-B integrands of Eq. (zwischenstufe) because, after the exact
    angular projection, the radial integrand for fixed l is a polynomial of
    degree ``<= 2B-2-l`` in t.
R2  sphere weights: Thm 3.1's ``b_j`` sums to 2; the azimuthal factor
    ``pi/B`` is applied, ``beta_j = (pi/B) b_j``.
R3  Lemma 3.7 recurs the *normalized* radial functions ``N_nl R_nl``.
R4  the Legendre functions are carried fully normalized (``Lambda_lm =
    Y_lm e^{-i m phi}``) with the Condon-Shortley phase of Def 2.1 and
    ``Y_{l,-m} = (-1)^m conj(Y_lm)``.
R5  samples are Gaussian-weighted: ``ftil(x) = exp(-r^2/2) f(x)``; the radial
    table is ``T_nl(i) = N_nl R_nl(r_i) exp(-t_i/2)`` and the radial weight
    ``what_i = (w_i/2) exp(t_i)`` (the symmetric form of the paper's
    ``a_i exp(r_i^2)`` modification, Sect. 3.2 and Sect. 5).
R6  phi-DFT sign ``e^{-i m phi}`` forward, ``e^{+i m phi}`` inverse, no 1/N;
    the Nyquist bin ``m = B`` is not a coefficient (dropped forward, zero
    inverse).

The paper's own grid (``rule="hermite"`` wherever a function takes ``rule``):
the radii are the 2B nodes of the half-range Gauss-Hermite rule of order 2B
(Thm 3.3, used in Eq. zwischenstufe_2), ``int_0^inf p(r) e^{-r^2} dr =
sum_i a_i p(r_i)``, so the radial weight is ``a_i r_i^2`` in place of
``w_i / 2``.  The rule is computed in high precision (mpmath): the recurrence
coefficients of the orthogonal polynomials from the moments
``int_0^inf r^k e^{-r^2} dr = Gamma((k+1)/2)/2`` by Chebyshev's algorithm,
the nodes as eigenvalues of the Jacobi matrix polished by Newton steps on the
recurrence, the weights from the Christoffel function ``1/sum_k p_k(r_i)^2``
of the orthonormal polynomials.  The paper leaves the method open (it cites
special recurrences of the literature); any method gives the same unique Gauss
rule.

Layouts (Sect. 3.4 index maps with ``i < R``, R = B radii, 2B on the paper's
grid):
  samples ``[batch][i][j][k]``: psi = 4B^2 i + 2B j + k, complex128;
  coefficients ``[batch][omega]``: omega = n(n-1)(2n-1)/6 + l(l+1) + m.
"""
from __future__ import annotations

from functools import lru_cache
from math import lgamma, log, pi, sqrt

import numpy as np

__all__ = [
    "coeff_count", "omega", "nlm_list",
    "sphere_rule", "laguerre_rule", "half_range_hermite_rule", "radial_rule", "n_radial", "radial_weights", "grid",
    "legendre_table", "radial_table",
    "laguerre_explicit", "legendre_rodrigues", "basis_explicit",
    "forward", "inverse", "forward_direct", "inverse_direct", "sgl_matrix",
    "adjoint_forward", "adjoint_inverse", "sample_weights",
    "physical_to_weighted", "weighted_to_physical", "cartesian_midpoints", "midpoint",
    "dct_matrix", "legendre_cosine_coeffs", "forward_seminaive",
]


# ---------------------------------------------------------------------------
# index maps (Sect. 3.4)
# ---------------------------------------------------------------------------

def coeff_count(B: int) -> int:
    """Omega = B(B+1)(2B+1)/6, the number of SGL coefficients (Sect. 3.4)."""
    return B * (B + 1) * (2 * B + 1) // 6


def omega(n: int, l: int, m: int) -> int:
    """Linear coefficient index omega(n,l,m) of Sect. 3.4."""
    return n * (n - 1) * (2 * n - 1) // 6 + l * (l + 1) + m


def nlm_list(B: int):
    """All (n, l, m) with |m| <= l < n <= B, in omega order."""
    out = []
    for n in range(1, B + 1):
        for l in range(n):
            for m in range(-l, l + 1):
                out.append((n, l, m))
    return out


# ---------------------------------------------------------------------------
# quadrature rules (Thm 3.1, Lemma 3.2; Thm 3.3 restated for t = r^2)
# ---------------------------------------------------------------------------

def sphere_rule(B: int):
    """Equiangular rule of order L = B (Thm 3.1).

    Returns theta_j = (2j+1) pi / 4B, phi_k = k pi / B (j, k < 2B) and the
    weights beta_j = (pi/B) b_j with b_j the closed form of Thm 3.1 (R2).
    """
    j = np.arange(2 * B)
    theta = (2 * j + 1) * pi / (4 * B)
    phi = np.arange(2 * B) * pi / B
    l = np.arange(B)
    inner = np.sin(np.outer(2 * j + 1, 2 * l + 1) * pi / (4 * B)) / (2 * l + 1)
    b = np.sin(theta) * (2.0 / B) * inner.sum(axis=1)
    beta = (pi / B) * b
    return theta, phi, beta


def _laguerre_pair(n: int, alpha: float, t: np.ndarray):
    """(L_n^(alpha)(t), L_{n-1}^(alpha)(t)) by the three-term recurrence
    Eq. (laguerre_recursion)."""
    prev = np.zeros_like(t)
    cur = np.ones_like(t)
    for k in range(n):
        nxt = ((2 * k + alpha + 1 - t) * cur - (k + alpha) * prev) / (k + 1)
        prev, cur = cur, nxt
    return cur, prev


_PI_LD = np.longdouble("3.14159265358979323846264338327950288419716939937510")


@lru_cache(maxsize=None)
def laguerre_rule(B: int, alpha: float = 0.5):
    """Generalized Gauss-Laguerre rule with B nodes for t^alpha e^{-t} (R1).

    Nodes: eigenvalues of the Jacobi matrix of the recurrence
    Eq. (laguerre_recursion) (a library eigensolver), polished by Newton steps
    on L_B^(alpha) evaluated by that recurrence.  Weights: the Christoffel
    form w_i = Gamma(B+alpha+1) t_i / (B! (B+alpha)^2 L_{B-1}(t_i)^2),
    evaluated in logarithms.  The polishing and the weights are computed in
    extended precision (NumPy longdouble), as the paper precomputes nodes and
    weights in high precision (Sect. 4): in double precision the smallest
    nodes keep relative errors near 1e-13 and their weights near 1e-11.
    """
    k = np.arange(B, dtype=np.float64)
    off = np.sqrt(np.arange(1, B) * (np.arange(1, B) + alpha))
    jac = np.diag(2 * k + alpha + 1) + np.diag(off, 1) + np.diag(off, -1)
    t = np.sort(np.linalg.eigvalsh(jac)).astype(np.longdouble)
    a = np.longdouble(alpha)
    for _ in range(6):
        ln, ln1 = _laguerre_pair(B, a, t)
        dln = (B * ln - (B + a) * ln1) / t
        t = t - ln / dln
    _, ln1 = _laguerre_pair(B, a, t)
    # log(Gamma(B+alpha+1)/B!) = log Gamma(alpha+1) + sum_{k<=B} log((k+alpha)/k)
    ks = np.arange(1, B + 1, dtype=np.longdouble)
    lg_ratio = np.sum(np.log((ks + a) / ks))
    if alpha == 0.5:
        lg_ratio += np.log(np.sqrt(_PI_LD) / 2)
    else:
        lg_ratio += np.longdouble(lgamma(alpha + 1))
    logw = lg_ratio + np.log(t) - 2 * np.log(B + a) - 2 * np.log(np.abs(ln1))
    return t.astype(np.float64), logw.astype(np.float64)


@lru_cache(maxsize=None)
def half_range_hermite_rule(N: int):
    """Gauss rule of order N for the weight e^{-r^2} on [0, inf) (Thm 3.3):
    nodes r_i and log a_i (float64), computed in high precision as stated in
    the module header."""
    import mpmath as mp
    with mp.workdps(2 * N + 60):  # Chebyshev's algorithm loses about 1.7 N digits
        mu = [mp.gamma(mp.mpf(k + 1) / 2) / 2 for k in range(2 * N)]
        alpha, beta = [mp.mpf(0)] * N, [mp.mpf(0)] * N
        sig_prev, sig = [mp.mpf(0)] * (2 * N), list(mu)
        alpha[0], beta[0] = mu[1] / mu[0], mu[0]
        for k in range(1, N):
            new = [mp.mpf(0)] * (2 * N)
            for l in range(k, 2 * N - k):
                new[l] = sig[l + 1] - alpha[k - 1] * sig[l] - beta[k - 1] * sig_prev[l]
            alpha[k] = new[k + 1] / new[k] - sig[k] / sig[k - 1]
            beta[k] = new[k] / sig[k - 1]
            sig_prev, sig = sig, new
    off = np.array([float(mp.sqrt(b)) for b in beta[1:]])
    jac = np.diag([float(a) for a in alpha]) + np.diag(off, 1) + np.diag(off, -1)
    x0 = np.sort(np.linalg.eigvalsh(jac))
    r = np.empty(N)
    loga = np.empty(N)
    with mp.workdps(50):
        sb = [mp.sqrt(b) for b in beta]
        for i, x in enumerate(x0):
            x = mp.mpf(float(x))
            for _ in range(4):  # Newton on the monic p_N
                pm, p, dpm, dp = mp.mpf(0), mp.mpf(1), mp.mpf(0), mp.mpf(0)
                for k in range(N):
                    bk = beta[k] if k > 0 else 0
                    pn = (x - alpha[k]) * p - bk * pm
                    dpn = p + (x - alpha[k]) * dp - bk * dpm
                    pm, p, dpm, dp = p, pn, dp, dpn
                x = x - p / dp
            qm, q = mp.mpf(0), 1 / sb[0]  # orthonormal polynomials
            s = q * q
            for k in range(N - 1):
                qn = ((x - alpha[k]) * q - (sb[k] if k > 0 else 0) * qm) / sb[k + 1]
                qm, q = q, qn
                s += q * q
            r[i] = float(x)
            loga[i] = float(-mp.log(s))
    return r, loga


def n_radial(B: int, rule: str = "laguerre") -> int:
    """Radii of the grid: B (R1) or 2B (the paper's grid)."""
    return {"laguerre": B, "hermite": 2 * B}[rule]


def radial_rule(B: int, rule: str = "laguerre"):
    """(t_i = r_i^2, log q_i) with int_0^inf p(r) r^2 e^{-r^2} dr =
    sum_i q_i p(r_i) for the radial degrees of bandlimit B: q_i = w_i / 2 on
    the B Gauss-Laguerre nodes (R1), q_i = a_i r_i^2 on the paper's 2B
    half-range Gauss-Hermite nodes (Eq. zwischenstufe_2)."""
    if rule == "laguerre":
        t, logw = laguerre_rule(B)
        return t, logw - log(2.0)
    if rule == "hermite":
        r, loga = half_range_hermite_rule(2 * B)
        return r * r, loga + 2 * np.log(r)
    raise ValueError(rule)


def radial_weights(B: int, rule: str = "laguerre"):
    """r_i, t_i = r_i^2 and the modified radial weights
    what_i = q_i exp(t_i) (R1, R5)."""
    t, logq = radial_rule(B, rule)
    what = np.exp(logq + t)
    return np.sqrt(t), t, what


def grid(B: int, rule: str = "laguerre"):
    """(r_i, theta_j, phi_k, what_i, beta_j) of the sampling grid."""
    r, _, what = radial_weights(B, rule)
    theta, phi, beta = sphere_rule(B)
    return r, theta, phi, what, beta


def sample_weights(B: int, rule: str = "laguerre") -> np.ndarray:
    """w_psi = what_i * beta_j as an (R, 2B, 2B) array (Sect. 3.4)."""
    _, _, what = radial_weights(B, rule)
    _, _, beta = sphere_rule(B)
    return np.broadcast_to(what[:, None, None] * beta[None, :, None], (len(what), 2 * B, 2 * B))


# ---------------------------------------------------------------------------
# basis tables (Def 2.1 + Eq. legendre_recurrence; Lemma 3.7)
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def legendre_table(B: int) -> np.ndarray:
    """Lam[m, l, j] = Y_lm(theta_j, phi) e^{-i m phi} for 0 <= m <= l < B.

    The normalized form of Eq. (legendre_recurrence) (R4).  Seed:
    Lam_mm = (-1)^m sqrt((2m+1)/4pi * prod_{k<=m} (2k-1)/(2k)) sin^m theta,
    formed in logarithms; Lam_{m+1,m} = sqrt(2m+3) cos theta Lam_mm.
    Entries with l < m are zero.  Negative orders follow from
    Lam_{l,-m} = (-1)^m Lam_{l,m}.
    """
    theta, _, _ = sphere_rule(B)
    x = np.cos(theta)
    logsin = np.log(np.sin(theta))
    lam = np.zeros((B, B, 2 * B))
    logprod = 0.0
    for m in range(B):
        if m > 0:
            logprod += log((2 * m - 1) / (2 * m))
        seed = np.exp(0.5 * log((2 * m + 1) / (4 * pi)) + 0.5 * logprod + m * logsin)
        lam[m, m] = -seed if (m % 2) else seed
        if m + 1 < B:
            lam[m, m + 1] = sqrt(2 * m + 3) * x * lam[m, m]
        for l in range(m + 1, B - 1):
            # Lam_{l+1,m} from Lam_{l,m} and Lam_{l-1,m}
            a = sqrt((2 * l + 1) * (2 * l + 3) / ((l + 1 - m) * (l + 1 + m)))
            c = sqrt((2 * l + 3) * (l + m) * (l - m) / ((2 * l - 1) * (l + 1 - m) * (l + 1 + m)))
            lam[m, l + 1] = a * x * lam[m, l] - c * lam[m, l - 1]
    return lam


@lru_cache(maxsize=None)
def radial_table(B: int, rule: str = "laguerre") -> np.ndarray:
    """T[l, n-1, i] = N_nl R_nl(r_i) exp(-t_i/2) for 0 <= l < n <= B, i < R.

    Lemma 3.7 read for the normalized functions (R3), seed
    sqrt(2/Gamma(l+3/2)) r^l formed in logarithms together with exp(-t/2).
    Entries with n <= l are zero.
    """
    _, t, _ = radial_weights(B, rule)
    R = len(t)
    logt = np.log(t)
    T = np.zeros((B, B, R))
    for l in range(B):
        seed = np.exp(0.5 * log(2.0) - 0.5 * lgamma(l + 1.5) + 0.5 * l * logt - 0.5 * t)
        prev = np.zeros(R)
        cur = seed
        T[l, l] = cur  # n = l + 1
        for n in range(l + 1, B):
            # R_{n+1,l} from R_{n,l} and R_{n-1,l}
            a = (2 * n - l - 0.5 - t) / sqrt((n + 0.5) * (n - l))
            c = sqrt((n - 0.5) / (n + 0.5) * (n - l - 1) / (n - l))
            nxt = a * cur - c * prev
            prev, cur = cur, nxt
            T[l, n] = cur
    return T


# ---------------------------------------------------------------------------
# independent closed-form evaluators (used only at small B)
# ---------------------------------------------------------------------------

def laguerre_explicit(k: int, alpha: float, t) -> np.ndarray:
    """L_k^(alpha)(t) by the explicit sum Eq. (associated_laguerre_explicit)."""
    t = np.asarray(t, dtype=np.float64)
    total = np.zeros_like(t)
    for j in range(k + 1):
        logbin = lgamma(k + alpha + 1) - lgamma(k - j + 1) - lgamma(alpha + j + 1)
        total = total + ((-1) ** j) * np.exp(logbin - lgamma(j + 1)) * t ** j
    return total


def legendre_rodrigues(l: int, m: int, x) -> np.ndarray:
    """P_lm(x) by the Rodrigues form of Def 2.1, 0 <= m <= l, with exact
    integer polynomial coefficients (small l only)."""
    from math import comb
    # (x^2 - 1)^l = sum_q C(l,q) (-1)^(l-q) x^(2q)
    coef = {2 * q: comb(l, q) * (-1) ** (l - q) for q in range(l + 1)}
    for _ in range(l + m):  # differentiate l+m times
        coef = {p - 1: c * p for p, c in coef.items() if p > 0}
    x = np.asarray(x, dtype=np.float64)
    poly = np.zeros_like(x)
    for p, c in coef.items():
        poly = poly + float(c) * x ** p
    from math import factorial
    pref = (-1) ** m / (2.0 ** l * factorial(l))
    return pref * (1 - x * x) ** (m / 2.0) * poly


def basis_explicit(n: int, l: int, m: int, r, theta, phi) -> np.ndarray:
    """H_nlm(r, theta, phi) of Def 1.2 from the closed forms (small B only)."""
    from math import factorial
    r = np.asarray(r, dtype=np.float64)
    am = abs(m)
    norm_nl = sqrt(2.0 * factorial(n - l - 1) / np.exp(lgamma(n + 0.5)))
    radial = norm_nl * laguerre_explicit(n - l - 1, l + 0.5, r * r) * r ** l
    cy = sqrt((2 * l + 1) / (4 * pi) * factorial(l - am) / factorial(l + am))
    lam = cy * legendre_rodrigues(l, am, np.cos(theta))
    if m < 0:
        lam = lam * (-1) ** am
    return radial * lam * np.exp(1j * m * np.asarray(phi))


# ---------------------------------------------------------------------------
# sample conventions (R5)
# ---------------------------------------------------------------------------

def physical_to_weighted(f: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    _, t, _ = radial_weights(B, rule)
    return f * np.exp(-0.5 * t)[:, None, None]


def weighted_to_physical(g: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    _, t, _ = radial_weights(B, rule)
    return g * np.exp(0.5 * t)[:, None, None]


# ---------------------------------------------------------------------------
# transforms
# ---------------------------------------------------------------------------

def _as_batch_samples(samples: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    s = np.asarray(samples, dtype=np.complex128)
    return s.reshape(-1, n_radial(B, rule), 2 * B, 2 * B)


def _as_batch_coeffs(coeffs: np.ndarray, B: int) -> np.ndarray:
    c = np.asarray(coeffs, dtype=np.complex128)
    return c.reshape(-1, coeff_count(B))


def _sphere_coeffs_to_sgl(S: np.ndarray, B: int, what, rule: str = "laguerre") -> np.ndarray:
    """Radial stage (DRT of Eq. DRT_matrix), all l:  fhat_nlm =
    sum_i T_nl(i) what_i S[b, i, l, m].  S is [b, i, l, m+B-1]."""
    T = radial_table(B, rule)
    nb = S.shape[0]
    out = np.zeros((nb, coeff_count(B)), dtype=np.complex128)
    for l in range(B):
        Tl = T[l, l:, :] * what[None, :]                 # (B-l, i)
        X = S[:, :, l, B - 1 - l:B + l]                  # (b, i, 2l+1)
        Y = np.einsum("ni,bim->bnm", Tl, X)              # (b, B-l, 2l+1)
        for n in range(l + 1, B + 1):
            o = omega(n, l, -l)
            out[:, o:o + 2 * l + 1] = Y[:, n - l - 1, :]
    return out


def forward(samples: np.ndarray, B: int, weights: bool = True, rule: str = "laguerre") -> np.ndarray:
    """Forward SGL transform of weighted samples (Thm 3.4), separated form.

    Steps of Eq. (SGL-Sampling-Theorem_rearranged) with the inner spherical
    sum split as in Eq. (SFFT_rearranged): a phi-DFT of every ring (library
    FFT), the Legendre sum over j per order m (Eq. DLT), then the radial sum
    over i per (l, m) (Eq. DRT).  ``weights=False`` drops what_i and beta_j,
    which is the adjoint of the inverse (Sect. 3.4).
    """
    f = _as_batch_samples(samples, B, rule)
    nb, R = f.shape[0], f.shape[1]
    _, _, what = radial_weights(B, rule)
    _, _, beta = sphere_rule(B)
    if not weights:
        what = np.ones_like(what)
        beta = np.ones_like(beta)
    lam = legendre_table(B)
    G = np.fft.fft(f, axis=-1)                           # G[b,i,j,(m mod 2B)]
    S = np.zeros((nb, R, B, 2 * B - 1), dtype=np.complex128)
    for m in range(-(B - 1), B):
        am = abs(m)
        sign = (-1.0) ** am if m < 0 else 1.0
        A = sign * lam[am, am:, :] * beta[None, :]       # (B-|m|, j)
        Gm = G[:, :, :, m % (2 * B)]                     # (b, i, j)
        S[:, :, am:, m + B - 1] = np.einsum("lj,bij->bil", A, Gm)
    return _sphere_coeffs_to_sgl(S, B, what, rule)


def inverse(coeffs: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    """Inverse SGL transform (Algorithm 4 steps): weighted samples
    ftil(x_psi) = sum fhat_nlm T_nl(i) Lam_lm(theta_j) e^{i m phi_k}."""
    c = _as_batch_coeffs(coeffs, B)
    nb = c.shape[0]
    T = radial_table(B, rule)
    R = T.shape[2]
    lam = legendre_table(B)
    S = np.zeros((nb, R, B, 2 * B - 1), dtype=np.complex128)  # [b,i,l,m]
    for l in range(B):
        Tl = T[l, l:, :]                                  # (B-l, i)
        X = np.zeros((nb, B - l, 2 * l + 1), dtype=np.complex128)
        for n in range(l + 1, B + 1):
            o = omega(n, l, -l)
            X[:, n - l - 1, :] = c[:, o:o + 2 * l + 1]
        S[:, :, l, B - 1 - l:B + l] = np.einsum("ni,bnm->bim", Tl, X)
    G = np.zeros((nb, R, 2 * B, 2 * B), dtype=np.complex128)  # [b,i,j,m mod 2B]
    for m in range(-(B - 1), B):
        am = abs(m)
        sign = (-1.0) ** am if m < 0 else 1.0
        A = sign * lam[am, am:, :]                       # (B-|m|, j)
        G[:, :, :, m % (2 * B)] = np.einsum("lj,bil->bij", A, S[:, :, am:, m + B - 1])
    # sum_m G e^{+i m phi_k}; the Nyquist bin stays zero (R6)
    return np.fft.ifft(G, axis=-1) * (2 * B)


def sgl_matrix(B: int, rule: str = "laguerre") -> np.ndarray:
    """Htil[omega, psi] = T_nl(i) Lam_lm(theta_j) e^{i m phi_k}, the weighted
    basis samples (matrix form of Sect. 3.4), from the recurrence tables."""
    T = radial_table(B, rule)
    lam = legendre_table(B)
    _, phi, _ = sphere_rule(B)
    rows = []
    for (n, l, m) in nlm_list(B):
        am = abs(m)
        lm = lam[am, l, :] * ((-1.0) ** am if m < 0 else 1.0)
        h = T[l, n - 1, :][:, None, None] * lm[None, :, None] * np.exp(1j * m * phi)[None, None, :]
        rows.append(h.reshape(-1))
    return np.array(rows)


def forward_direct(samples: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    """Naive forward transform, Algorithm 1: for every coefficient the full
    triple sum over the grid, O(B^7).  Small B only."""
    R = n_radial(B, rule)
    f = _as_batch_samples(samples, B, rule).reshape(-1, 4 * R * B * B)
    H = sgl_matrix(B, rule)
    w = sample_weights(B, rule).reshape(-1)
    return (f * w[None, :]) @ np.conj(H).T


def inverse_direct(coeffs: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    """Naive inverse transform, Algorithm 2: every sample summed over all
    coefficients, O(B^7).  Small B only."""
    c = _as_batch_coeffs(coeffs, B)
    H = sgl_matrix(B, rule)
    return (c @ H).reshape(-1, n_radial(B, rule), 2 * B, 2 * B)


# ---------------------------------------------------------------------------
# the seminaive Legendre transform (Eq. DCT, Eq. dct_trick)
# ---------------------------------------------------------------------------

def dct_matrix(N: int) -> np.ndarray:
    """C_N of Eq. (DCT): row k = sqrt(1/N) or sqrt(2/N) times cos(k theta_j),
    theta_j = (2j+1) pi / 2N."""
    j = np.arange(N)
    C = np.cos(np.outer(np.arange(N), (2 * j + 1) * pi / (2 * N)))
    C[0] *= sqrt(1.0 / N)
    C[1:] *= sqrt(2.0 / N)
    return C


def legendre_cosine_coeffs(B: int) -> np.ndarray:
    """Q[m, l, k] = [C_2B q_lm]_k, q_lm = Lambda_lm(theta_j) / w_m(theta_j) on the
    2B rings, w_m = 1 for even m and sin(theta) for odd m: q_lm is then a
    cosine polynomial of degree l (even m) or l - 1 (odd m) in theta, so by
    the property stated after Eq. (DCT) its entries vanish beyond that degree
    (reading for odd m: the factor sin(theta) goes with the data)."""
    theta, _, _ = sphere_rule(B)
    lam = legendre_table(B)                         # [m, l, j]
    w = np.where(np.arange(B)[:, None] % 2 == 1, np.sin(theta)[None, :], 1.0)  # [m, j]
    C = dct_matrix(2 * B)
    return np.einsum("kj,mlj->mlk", C, lam / w[:, None, :])


def forward_seminaive(samples: np.ndarray, B: int, weights: bool = True, rule: str = "laguerre") -> np.ndarray:
    """The forward transform with the Legendre sums of Eq. (DLT) taken by the
    seminaive algorithm: per order m, the DCT C_2B of the data t_j = beta_j
    w_m(theta_j) G_j over all 2B rings (a library DCT as the step), then for
    every l the inner product of Eq. (dct_trick) over the first deg + 1 DCT
    coefficients only.  The phi-FFT and the radial sum as in forward()."""
    f = _as_batch_samples(samples, B, rule)
    nb, R = f.shape[0], f.shape[1]
    _, _, what = radial_weights(B, rule)
    theta, _, beta = sphere_rule(B)
    if not weights:
        what = np.ones_like(what)
        beta = np.ones_like(beta)
    Q = legendre_cosine_coeffs(B)
    C = dct_matrix(2 * B)
    G = np.fft.fft(f, axis=-1)                            # G[b,i,j,(m mod 2B)]
    S = np.zeros((nb, R, B, 2 * B - 1), dtype=np.complex128)
    for m in range(-(B - 1), B):
        am = abs(m)
        sign = (-1.0) ** am if m < 0 else 1.0
        w = np.sin(theta) if am % 2 else np.ones_like(theta)
        T = np.einsum("kj,bij->bik", C, G[:, :, :, m % (2 * B)] * (beta * w)[None, None, :])
        for l in range(am, B):
            deg = l if am % 2 == 0 else l - 1
            S[:, :, l, m + B - 1] = sign * T[:, :, :deg + 1] @ Q[am, l, :deg + 1]
    return _sphere_coeffs_to_sgl(S, B, what, rule)


# ---------------------------------------------------------------------------
# the midpoint rule on a Cartesian grid (the practice of the Discussion)
# ---------------------------------------------------------------------------

def cartesian_midpoints(M: int, L: float):
    """x, y, z (each (M, M, M), index [ix, iy, iz]) of the cell midpoints of
    [-L, L]^3 with M cells per axis, and the cell volume."""
    h = 2.0 * L / M
    c = -L + (np.arange(M) + 0.5) * h
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z, h ** 3


def midpoint(f: np.ndarray, B: int, M: int, L: float) -> np.ndarray:
    """fhat_nlm ~= sum_k f(x_k) conj(H_nlm(x_k)) exp(-|x_k|^2) dV: the midpoint
    rule for the inner product Eq. (inner_product) on the cells of [-L, L]^3,
    H_nlm from the closed forms (small B only).  f: (batch, M, M, M) physical
    samples."""
    f = np.asarray(f, dtype=np.complex128).reshape(-1, M, M, M)
    x, y, z, dV = cartesian_midpoints(M, L)
    r = np.sqrt(x * x + y * y + z * z)
    theta = np.arccos(np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0))
    phi = np.arctan2(y, x)
    w = np.exp(-r * r) * dV
    out = np.zeros((f.shape[0], coeff_count(B)), dtype=np.complex128)
    for (n, l, m) in nlm_list(B):
        h = basis_explicit(n, l, m, r, theta, phi)
        out[:, omega(n, l, m)] = np.einsum("bxyz,xyz->b", f, np.conj(h) * w)
    return out


def adjoint_forward(y: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    """Adjoint of the forward map: F_fwd^H y = diag(w_psi) F_inv y (Sect. 3.4)."""
    return inverse(y, B, rule) * sample_weights(B, rule)[None]


def adjoint_inverse(g: np.ndarray, B: int, rule: str = "laguerre") -> np.ndarray:
    """Adjoint of the inverse map: F_inv^H g = the forward without weights."""
    return forward(g, B, weights=False, rule=rule)
