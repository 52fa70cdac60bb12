"""Weighted CBP in the oracle: forward reduces to CBP, adjoint equals finite differences.

The adjoint (reverse mode through the sequential sweeps) is checked against central
FP64 finite differences (step 1e-6) of the mean BCE loss, on a Z=4 lift of the 12x24
base matrix, for the weights and for the channel LLRs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_05286_gb300 import inputs as I


@pytest.fixture(scope="module")
def small():
    qc = I.relift(I.code_576(), 4)
    return qc, O.OracleCode(qc.base, qc.Z)


def bce(soft, x):
    return np.logaddexp(0.0, -(1.0 - 2.0 * x) * soft).mean()


def bce_grad(soft, x):
    z = -(1.0 - 2.0 * x) * soft
    return (-(1.0 - 2.0 * x) / (1.0 + np.exp(-z))) / soft.size


def test_unit_weights_give_cbp(small):
    qc, oc = small
    fr = I.make_frames(qc, 40, 1.5, seed=8)
    for T in (1, 3, 10):
        ones = np.ones((T, qc.mb))
        a = oc.weighted(fr.llr, ones, T, precision=32)
        b = oc.decode(fr.llr, alg="cbp_sp", max_iter=T, stop="none")["soft"]
        assert np.array_equal(a, b)
        a64 = oc.weighted(fr.llr.astype(np.float64), ones, T)
        b64 = oc.decode(fr.llr.astype(np.float64), alg="cbp_sp", max_iter=T, stop="none",
                        precision=64)["soft"]
        assert np.array_equal(a64, b64)


def test_zero_weights_leave_the_channel_llrs(small):
    qc, oc = small
    fr = I.make_frames(qc, 4, 1.0, seed=9)
    L = fr.llr.astype(np.float64)
    for T in (1, 5):
        assert np.array_equal(oc.weighted(L, np.zeros((T, qc.mb)), T), L)


def test_single_check_closed_form():
    """One parity check, one sweep: Lambda_v = L_v + w * 2 atanh(prod_{u != v} tanh(L_u / 2))."""
    oc = O.OracleCode(np.zeros((1, 5), np.int32), 1)
    L = np.array([[0.7, -1.2, 2.0, 0.3, -0.9]])
    for w in (1.0, 0.6, 1.7):
        out = oc.weighted(L, np.array([[w]]), 1)[0]
        for v in range(5):
            ext = 2.0 * np.arctanh(np.prod(np.tanh(np.delete(L[0], v) / 2.0)))
            assert abs(out[v] - (L[0, v] + w * ext)) < 1e-12


@pytest.mark.parametrize("T,ebn0", [(4, 0.5), (10, 1.0)])
def test_adjoint_matches_finite_differences(small, T, ebn0):
    qc, oc = small
    fr = I.make_frames(qc, 3, ebn0, seed=20 + T)
    L = fr.llr.astype(np.float64)
    x = fr.codewords.astype(np.float64)
    w = 1.0 + 0.1 * np.random.default_rng(T).standard_normal((T, qc.mb))
    gw, gl = oc.weighted_grad(L, w, T, bce_grad(oc.weighted(L, w, T), x))
    h = 1e-6
    rng = np.random.default_rng(1)
    for _ in range(12):
        i, j = int(rng.integers(T)), int(rng.integers(qc.mb))
        wp, wm = w.copy(), w.copy()
        wp[i, j] += h
        wm[i, j] -= h
        fd = (bce(oc.weighted(L, wp, T), x) - bce(oc.weighted(L, wm, T), x)) / (2 * h)
        assert abs(fd - gw[i, j]) <= 1e-5 * max(abs(fd), 1e-4), (i, j, fd, gw[i, j])
    big = np.argsort(-np.abs(gl).ravel())[:8]
    for idx in big:
        f, v = divmod(int(idx), qc.N)
        Lp, Lm = L.copy(), L.copy()
        Lp[f, v] += h
        Lm[f, v] -= h
        fd = (bce(oc.weighted(Lp, w, T), x) - bce(oc.weighted(Lm, w, T), x)) / (2 * h)
        assert abs(fd - gl[f, v]) <= 1e-5 * abs(fd) + 1e-9, (f, v, fd, gl[f, v])
