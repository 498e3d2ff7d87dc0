"""The seeded input generators shared by the tests, smoke() and bench.py:
shapes, determinism, the coefficient-slot order and the workload recipes."""
import numpy as np

import oracle as O
from paper_1604_05140_gb300 import inputs


def test_coefficient_count_and_slot_degrees_follow_the_index_map():
    # Omega = B(B+1)(2B+1)/6 and slot omega carries the degree n of the
    # paper's index map omega(n, l, m) (Sect. 3.4)
    for B in (1, 2, 5, 16, 128):
        assert inputs.n_coeffs(B) == B * (B + 1) * (2 * B + 1) // 6 == O.coeff_count(B)
    B = 9
    deg = inputs.degree_of_slot(B)
    assert [int(d) for d in deg] == [n for (n, l, m) in O.nlm_list(B)]


def test_random_draws_are_seeded_and_shaped():
    a = inputs.random_coeffs(6, 3, seed=5)
    assert a.shape == (3, inputs.n_coeffs(6)) and a.dtype == np.complex128
    assert np.array_equal(a, inputs.random_coeffs(6, 3, seed=5))
    assert not np.array_equal(a, inputs.random_coeffs(6, 3, seed=6))
    d = inputs.random_coeffs(6, 3, seed=5, decay=True)
    np.testing.assert_allclose(d * inputs.degree_of_slot(6)[None, :], a, rtol=1e-15)
    u = inputs.random_coeffs(6, 2, seed=5, dist="uniform")
    assert np.abs(u.real).max() <= 1 and np.abs(u.imag).max() <= 1
    s = inputs.random_samples(4, 2, seed=1, scale=0.01)
    assert s.shape == (2, 4, 8, 8) and np.abs(s).max() < 0.1


def test_uneven_bandlimit_recipe():
    # 256 functions, B uniform over {16, 24, ..., 128} (15 values), seeded
    Bs = inputs.uneven_bandlimits()
    assert Bs.shape == (256,) and np.array_equal(Bs, inputs.uneven_bandlimits())
    assert set(Bs.tolist()) == set(range(16, 129, 8))
