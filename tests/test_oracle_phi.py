"""Pins of the oracle's phi (Eq. s2e5) against mathematics it does not share code with.

phi(x) = -log tanh(x/2) is evaluated here independently with mpmath (40 digits) and
with numpy's FP64 log1p/expm1; the oracle's FP32 phi must stay within 2.5 ulp of it,
be self-inverse (opening of Appendix A) and decreasing; its FP64 phi must match mpmath.
"""
import mpmath
import numpy as np
import pytest

from oracle import oracle as O

mpmath.mp.dps = 40


def phi_mp(x):
    return mpmath.log(mpmath.coth(mpmath.mpf(x) / 2))


def test_clamp_constant_is_phi_of_30():
    assert np.float32(O.xlo32()) == np.float32(float(phi_mp(30.0)))


def test_phi32_accuracy_dense_sample():
    lo = np.float32(O.xlo32()).view(np.uint32)
    hi = np.float32(30.0).view(np.uint32)
    bits = np.arange(lo, hi + 1, 97, dtype=np.uint32)
    x = bits.view(np.float32)
    y = O.phi32(x).astype(np.float64)
    ref = np.log1p(2.0 / np.expm1(x.astype(np.float64)))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert (np.abs(y - ref) / ulp).max() <= 2.5


def test_phi32_against_mpmath_and_grid_edges():
    rng = np.random.default_rng(0)
    x = np.exp(rng.uniform(np.log(2e-13), np.log(30.0), 600)).astype(np.float32)
    # segment edges: half-way between grid centres and +-1 ulp around them
    e = np.array([2.0 - 2 ** -7, 2.0, 2.03125, 1.0 + 2 ** -6, 29.96875, 1e-6], np.float32)
    x = np.concatenate([x, e, np.nextafter(e, np.float32(0)), np.nextafter(e, np.float32(40))])
    y = O.phi32(x)
    for xi, yi in zip(x, y):
        ref = float(phi_mp(float(xi)))
        assert abs(float(yi) - ref) <= 2.5 * float(np.spacing(np.float32(ref))), xi


def test_phi32_clamps_and_special_values():
    y = O.phi32(np.array([0.0, 1e-30, 40.0, np.inf, np.nan], np.float32))
    xlo = np.float32(O.xlo32())
    assert y[0] == y[1] == y[4] == O.phi32(np.array([xlo], np.float32))[0]
    assert y[2] == y[3] == xlo
    assert abs(float(y[0]) - 30.0) < 1e-5


def test_phi32_self_inverse_and_decreasing():
    x = np.linspace(0.01, 12.0, 20001).astype(np.float32)
    y = O.phi32(x)
    z = O.phi32(y)
    # phi is its own inverse; the round trip is well conditioned on this range
    assert np.max(np.abs(z - x) / x) < 3e-5
    assert (np.diff(y.astype(np.float64)) <= np.spacing(y[:-1]).astype(np.float64)).all()


def test_phi64_matches_mpmath():
    x = np.array([1e-12, 1e-6, 0.01, 0.3, 1.0, 2.5, 7.0, 20.0, 45.0])
    y = O.phi64(x)
    for xi, yi in zip(x, y):
        ref = float(phi_mp(xi))
        assert abs(yi - ref) <= 4e-16 * abs(ref) + 1e-300


def test_table_values_are_phi_at_the_centres():
    tab = O.phi_table()
    assert tab.shape == (1858, 4)
    # the first coefficient is fl32(phi(centre)); check a spread of centres with mpmath
    for i in list(range(0, 1409, 97)) + [1408, 1409, 1500, 1857]:
        if i < 1409:
            m = float(np.uint32((2688 + i) << 18).view(np.float32))
            h = 2.0 ** (np.frexp(m)[1] - 1)
        else:
            m = (32 + i - 1409) / 16.0
            h = 1.0 / 16.0
        assert tab[i, 0] == np.float32(float(phi_mp(m)))
        d1 = -h / float(mpmath.sinh(mpmath.mpf(m)))
        assert tab[i, 1] == np.float32(d1)
