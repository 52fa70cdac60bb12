"""The paper-literal stop of Eq. (s4e24) with the Step 3 output, in the oracle.

Pins: special cases whose outcome follows from the rule by hand, and an independent
pure-Python decoder in the layered (tanh-product) form of the same recursion on a small
lift, which evaluates the rule from its own quantities.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_05286_gb300 import inputs as I


@pytest.fixture(scope="module")
def c576():
    qc = I.code_576()
    return qc, O.OracleCode(qc.base, qc.Z)


def test_noiseless_frames_stop_after_one_sweep(c576):
    # every V2C message keeps the codeword's sign, so every check update leaves
    # Omega > 0 and flips nothing: the M-th update is the last of sweep 1
    qc, oc = c576
    cw = I.make_frames(qc, 8, 3.0, seed=3).codewords
    llr = np.where(cw == 1, -8.0, 8.0).astype(np.float32)
    for prec in (32, 64):
        r = oc.decode(llr, alg="cbp_sp", max_iter=10, stop="window", precision=prec)
        assert np.all(r["iters"] == 1) and np.array_equal(r["hard"], cw)


def test_wrong_channel_sign_on_a_weight_one_variable_never_stops(c576):
    # the V2C message of a weight-1 variable is its channel LLR (its only check is both
    # c_j and c_i), so a wrong channel sign keeps that check's Omega negative for good:
    # the window never fills, although the posterior corrects the bit
    qc, oc = c576
    llr = np.full((1, qc.N), 6.0, np.float32)      # all-zero codeword
    col = int(np.nonzero((qc.base >= 0).sum(0) == 1)[0][0])
    llr[0, col * qc.Z + 5] = -0.5
    r = oc.decode(llr, alg="cbp_sp", max_iter=12, stop="window")
    assert r["iters"][0] == -12
    assert not r["hard"].any()
    s = oc.decode(llr, alg="cbp_sp", max_iter=12, stop="syndrome")
    assert s["iters"][0] == 1 and not s["hard"].any()


def _rows(qc):
    rows = []
    for r in range(qc.mb):
        for i in range(qc.Z):
            rows.append([c * qc.Z + (i + int(qc.base[r, c])) % qc.Z
                         for c in range(qc.nb) if qc.base[r, c] >= 0])
    return rows


def _window_layered(rows, L, max_iter):
    """Layered BP with C2V messages from the tanh rule (Eq. s3e2) and the window stop.

    CBP's posterior at check c_i's visit (Eq. s4e20) is the layered posterior after the
    update of v's previous check and before c_i's; Omega_ci > 0 iff the V2C messages into
    c_i have an even number of negative signs."""
    M = len(rows)
    lam = [float(x) for x in L]
    pneg = [x < 0.0 for x in L]
    R = [[0.0] * len(vs) for vs in rows]
    win = 0
    for t in range(1, max_iter + 1):
        for m, vs in enumerate(rows):
            flip = False
            q = []
            for k, v in enumerate(vs):
                neg = lam[v] < 0.0
                flip |= neg != pneg[v]
                pneg[v] = neg
                q.append(lam[v] - R[m][k])
            odd = sum(x < 0.0 for x in q) % 2
            th = [math.tanh(x / 2.0) for x in q]
            for k, v in enumerate(vs):
                p = 1.0
                for j, x in enumerate(th):
                    if j != k:
                        p *= x
                p = min(max(p, -1.0 + 1e-16), 1.0 - 1e-16)
                R[m][k] = 2.0 * math.atanh(p)
                lam[v] = q[k] + R[m][k]
            win = win + 1 if (odd == 0 and not flip) else 0
            if win >= M:
                return t, np.array(pneg, np.uint8)
    return -max_iter, np.array(pneg, np.uint8)


def test_window_stop_equals_layered_formulation_fp64():
    qc = I.relift(I.code_576(), 4)          # N = 96, M = 48
    oc = O.OracleCode(qc.base, qc.Z)
    rows = _rows(qc)
    fr = I.make_frames(qc, 60, 3.5, seed=11)
    r = oc.decode(fr.llr.astype(np.float64), alg="cbp_sp", max_iter=15, stop="window",
                  precision=64)
    for f in range(fr.llr.shape[0]):
        t, hard = _window_layered(rows, fr.llr[f].astype(np.float64), 15)
        assert r["iters"][f] == t, f"frame {f}"
        assert np.array_equal(r["hard"][f], hard), f"frame {f}"
    # the rule must have fired in some frames and run out in others
    assert (r["iters"] > 0).any() and (r["iters"] < 0).any()


def test_window_stop_is_for_the_log_tanh_decoder_only(c576):
    qc, oc = c576
    llr = I.make_frames(qc, 2, 2.0, seed=1).llr
    for alg in ("cbp_nms", "lbp_nms", "fbp_sp"):
        with pytest.raises(Exception):
            oc.decode(llr, alg=alg, max_iter=5, stop="window")
