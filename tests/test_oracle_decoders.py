"""Pins of the oracle's decoders against results fixed by the paper and by mathematics.

* Closed form of the check-belief, Eqs. (s4e1)/(s4e3): Omega_c = 2 atanh(prod tanh(Q/2)).
* Appendix A, Eq. (ae7): psi^- recovers the belief of the other inputs.
* CBP is layered BP with deferred C2V messages (Eqs. s4e9-s4e14): same FP32 operations,
  so CBP == LBP bit for bit (sum-product and normalized min-sum).
* On cycle-free graphs BP gives exact bit marginals: brute force over all codewords.
* Noiseless codewords, channel/decoder sign symmetry, zero syndrome of decoded words.
* Operation counts per iteration: Tables I and II.
"""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_05286_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALGS32 = ["cbp_sp", "cbp_nms", "lbp_nms", "fbp_sp", "lbp_sp"]


@pytest.fixture(scope="module")
def c576():
    code = I.code_576()
    return code, O.OracleCode(code.base, code.Z)


@pytest.fixture(scope="module")
def frames576(c576):
    code, _ = c576
    return I.make_frames(code, 120, 2.0, seed=1200)


# --------------------------------------------------------------------------- closed forms
def closed_form_omega(q):
    return 2.0 * np.arctanh(np.prod(np.tanh(np.asarray(q) / 2.0)))


@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_check_belief_equals_closed_form(c576, frames576, sweeps):
    code, oc = c576
    llr = frames576.llr[3].astype(np.float64) * 0.5      # moderate LLRs: atanh well conditioned
    S, sig, q, r = oc.trace(llr, sweeps)
    echk, evar = oc.edges()
    omega = np.where(sig == 1, -1.0, 1.0) * O.phi64(S)
    for m in range(0, code.M, 7):
        qs = q[echk == m]
        ref = closed_form_omega(qs)
        if abs(ref) < 12:
            assert abs(omega[m] - ref) <= 1e-9 * max(1.0, abs(ref))


def test_first_row_belief_in_channel_llrs(c576, frames576):
    code, oc = c576
    llr = frames576.llr[0].astype(np.float64) * 0.5
    S, sig, q, r = oc.trace(llr, 1)
    for m in range(code.Z):                      # row 0: every variable is first-visited
        vs = code.check_rows()[m]
        ref = closed_form_omega(llr[vs])
        omega = (-1.0 if sig[m] else 1.0) * O.phi64(np.array([S[m]]))[0]
        assert abs(omega - ref) <= 1e-10 * max(1.0, abs(ref))
        # Pr(S_c = 0 | Y) = (1 + prod tanh(L/2)) / 2 and Omega is its log-odds, Eq. (s4e1)
        p0 = (1.0 + np.prod(np.tanh(llr[vs] / 2.0))) / 2.0
        assert abs(np.log(p0 / (1.0 - p0)) - omega) <= 1e-9 * max(1.0, abs(omega))


def test_b2v_is_extrinsic_belief(c576, frames576):
    """Eq. (ae7): the stored C2V of (c, v) is the belief of c without v."""
    code, oc = c576
    llr = frames576.llr[5].astype(np.float64) * 0.5
    S, sig, q, r = oc.trace(llr, 1)
    echk, evar = oc.edges()
    checked = 0
    for e in range(0, code.E, 5):
        if r[e] == 0.0:
            continue                              # not yet revisited in sweep 1
        m = echk[e]
        others = q[(echk == m) & (np.arange(code.E) != e)]
        ref = closed_form_omega(others)
        if abs(ref) < 12:
            assert abs(r[e] - ref) <= 1e-9 * max(1.0, abs(ref))
            checked += 1
    assert checked > 50


# --------------------------------------------------------------------------- equivalences
@pytest.mark.parametrize("pair", [("cbp_sp", "lbp_sp"), ("cbp_nms", "lbp_nms")])
def test_cbp_equals_layered_bp_bitwise_fp32(c576, frames576, pair):
    _, oc = c576
    a = oc.decode(frames576.llr, alg=pair[0], max_iter=30)
    b = oc.decode(frames576.llr, alg=pair[1], max_iter=30)
    assert np.array_equal(a["hard"], b["hard"])
    assert np.array_equal(a["iters"], b["iters"])
    assert np.array_equal(a["soft"].view(np.uint32) & 0x7FFFFFFF, b["soft"].view(np.uint32) & 0x7FFFFFFF)
    assert np.array_equal(a["soft"], b["soft"])


def test_cbp_equals_layered_bp_fp64(c576, frames576):
    _, oc = c576
    llr = frames576.llr.astype(np.float64)
    a = oc.decode(llr, alg="cbp_sp", precision=64)
    b = oc.decode(llr, alg="lbp_sp", precision=64)
    assert np.array_equal(a["hard"], b["hard"]) and np.array_equal(a["iters"], b["iters"])
    assert np.abs(a["soft"] - b["soft"]).max() <= 1e-12 * np.abs(b["soft"]).max()


def test_s_domain_equals_literal_omega_recursion(c576, frames576):
    """The S = sum phi(|Q|) storage against the paper's psi^+/psi^- recursion on Omega."""
    _, oc = c576
    llr = frames576.llr[:40].astype(np.float64)
    a = oc.decode(llr, alg="cbp_sp", precision=64, max_iter=20)
    b = oc.decode(llr, alg="cbp_sp_omega", precision=64, max_iter=20)
    assert np.array_equal(a["hard"], b["hard"]) and np.array_equal(a["iters"], b["iters"])
    assert np.abs(a["soft"] - b["soft"]).max() < 1e-6


def test_fp32_oracle_tracks_fp64_oracle():
    code = I.code_576()
    oc = O.OracleCode(code.base, code.Z)
    fr = I.make_frames(code, 200, 2.5, seed=1250)
    a = oc.decode(fr.llr, alg="cbp_sp")
    b = oc.decode(fr.llr.astype(np.float64), alg="cbp_sp", precision=64)
    same = (a["hard"] == b["hard"]).all(axis=1)
    assert same.mean() >= 0.97
    conv = (a["iters"] > 0) & (b["iters"] > 0) & same
    assert (a["iters"][conv] == b["iters"][conv]).mean() >= 0.97


# --------------------------------------------------------------------------- trees
def _tree_codes():
    one_check = np.zeros((1, 5), np.int32)                      # single parity check
    t = -np.ones((5, 10), np.int32)
    for r, vs in enumerate([(0, 1, 2), (2, 3, 4), (4, 5, 6), (1, 7), (6, 8, 9)]):
        t[r, list(vs)] = 0
    lift = t.copy()                                              # Z=3 lift of a tree: a forest
    rng = np.random.default_rng(4)
    lift[lift >= 0] = rng.integers(0, 3, size=(lift >= 0).sum())
    return [(one_check, 1), (t, 1), (lift, 3)]


def exact_llr(H, L):
    """log Pr(x_v=0|y) / Pr(x_v=1|y) by enumerating every codeword of H."""
    code = I.QCCode(H, 1)
    enc = I.GF2Encoder(code)
    info = np.array(list(itertools.product([0, 1], repeat=enc.K)), np.uint8)
    cws = enc.encode(info)
    assert not code.syndrome(cws).any()
    logp = (L[None, :] * (1.0 - 2.0 * cws) / 2.0).sum(axis=1)
    out = np.empty(H.shape[1])
    for v in range(H.shape[1]):
        a, b = logp[cws[:, v] == 0], logp[cws[:, v] == 1]
        out[v] = np.logaddexp.reduce(a) - np.logaddexp.reduce(b)
    return out


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("alg", ["cbp_sp", "lbp_sp", "fbp_sp", "cbp_sp_omega"])
def test_exact_marginals_on_trees(k, alg):
    base, Z = _tree_codes()[k]
    code = I.QCCode(base, Z)
    H = code.dense_H().astype(np.int32) - 1   # as a Z=1 base matrix: 0 / -1
    oc = O.OracleCode(base, Z)
    rng = np.random.default_rng(10 + k)
    for _ in range(3):
        L = rng.normal(1.0, 1.5, size=code.N)
        ref = exact_llr(H, L)
        r = oc.decode(L[None], alg=alg, precision=64, max_iter=14, stop="none")
        assert np.abs(r["soft"][0] - ref).max() < 1e-9


def test_nms_single_check_by_hand():
    oc = O.OracleCode(np.zeros((1, 3), np.int32), 1)
    L = np.array([[1.0, -2.5, 4.0]], np.float32)
    for alg in ("cbp_nms", "lbp_nms"):
        r = oc.decode(L, alg=alg, max_iter=1, stop="none", alpha=0.75)
        # Lambda_v = L_v + alpha * sgn(prod of the others) * min |others|
        assert r["soft"][0].tolist() == [1.0 - 0.75 * 2.5, -2.5 + 0.75 * 1.0, 4.0 - 0.75 * 1.0]
        assert r["iters"][0] == 1 and r["hard"][0].tolist() == [1, 1, 0]


def test_nms_two_checks_two_sweeps_by_hand():
    """Layered normalized min-sum (Sec. II-B, Eqs. s2e10/s2e12 with the alpha of the min-sum
    literature) worked by hand on two checks sharing two variables, alpha = 0.75, two sweeps.
    Every value is a short binary fraction, so the FP32 and FP64 oracles must give exactly
    these numbers.  CBP min-sum (Eqs. s4e18xx/s4e21xx, reading of the garbled text: unscaled
    minima, first of equal minima wins) sends the same messages later, so it must too.

    Checks: c0 = (v0, v1, v2), c1 = (v1, v2, v3); L = (2, -1, 3, 0.5).
    Sweep 1, c0: Q = L = (2, -1, 3); min1 = 1 (v1), min2 = 2, one negative sign.
        R = (-0.75*1, +0.75*2, -0.75*1) = (-0.75, 1.5, -0.75); Lambda = (1.25, 0.5, 2.25, 0.5)
      c1: Q = (0.5, 2.25, 0.5); min1 = 0.5 (v1, first of the tie), min2 = 0.5 (v3), all +.
        R = (0.375, 0.375, 0.375); Lambda = (1.25, 0.875, 2.625, 0.875)
    Sweep 2, c0: Q = Lambda - R_old = (2, -0.625, 3.375); min1 = 0.625 (v1), min2 = 2.
        R = (-0.46875, 1.5, -0.46875); Lambda = (1.53125, 0.875, 2.90625, 0.875)
      c1: Q = (0.5, 2.53125, 0.5); min1 = min2 = 0.5.  R = (0.375, 0.375, 0.375)
        Lambda = (1.53125, 0.875, 2.90625, 0.875)
    A mistake in where alpha is applied (to the stored minima, to the rebuilt old message
    only, or twice) changes these numbers."""
    oc = O.OracleCode(np.array([[0, 0, 0, -1], [-1, 0, 0, 0]], np.int32), 1)
    L = np.array([[2.0, -1.0, 3.0, 0.5]])
    want = {1: [1.25, 0.875, 2.625, 0.875], 2: [1.53125, 0.875, 2.90625, 0.875]}
    for alg in ("lbp_nms", "cbp_nms"):
        for prec in (32, 64):
            for sweeps, ref in want.items():
                r = oc.decode(L, alg=alg, max_iter=sweeps, stop="none", alpha=0.75,
                              precision=prec)
                assert r["soft"][0].tolist() == ref, (alg, prec, sweeps)


def layered_nms_by_exclusion(H_rows, L, alpha, sweeps):
    """Textbook layered normalized min-sum in FP64, written from the definition with
    explicit exclusion: the message of check m to its k-th variable is
    alpha * prod_{j != k} sgn(q_j) * min_{j != k} |q_j| (no min1/min2/argmin bookkeeping);
    checks in ascending order, Lambda updated after each check (Eqs. s2e10, s2e12)."""
    lam = L.astype(np.float64).copy()
    R = [np.zeros(len(r)) for r in H_rows]
    for _ in range(sweeps):
        for m, vs in enumerate(H_rows):
            q = lam[vs] - R[m]
            neg = q < 0.0
            for k in range(len(vs)):
                others = [j for j in range(len(vs)) if j != k]
                mag = min(abs(q[j]) for j in others)
                sign = np.logical_xor.reduce(neg[others])
                R[m][k] = -(alpha * mag) if sign else alpha * mag
            lam[vs] = q + R[m]
    return lam


@pytest.mark.parametrize("alpha", [0.75, 0.625, 1.0])
def test_nms_equals_the_exclusion_definition(alpha):
    """Both min-sum oracles (FP64) against layered NMS by explicit exclusion, bit for bit,
    on the Z = 4 lift of the 576-bit base matrix over several sweeps."""
    base = I.code_576().base
    lift = np.where(base >= 0, base % 4, -1).astype(np.int32)
    code = I.QCCode(lift, 4)
    H = code.dense_H()
    rows = [np.flatnonzero(H[m]) for m in range(H.shape[0])]
    oc = O.OracleCode(lift, 4)
    rng = np.random.default_rng(31)
    for trial in range(4):
        L = rng.normal(1.2, 2.0, size=code.N)
        for sweeps in (1, 3, 6):
            ref = layered_nms_by_exclusion(rows, L, alpha, sweeps)
            for alg in ("lbp_nms", "cbp_nms"):
                r = oc.decode(L[None], alg=alg, max_iter=sweeps, stop="none", alpha=alpha,
                              precision=64)
                assert np.array_equal(r["soft"][0], ref), (alg, trial, sweeps)


# --------------------------------------------------------------------------- fixed points, symmetry
@pytest.mark.parametrize("alg", ALGS32)
def test_noiseless_codeword_decodes_in_one_sweep(c576, alg):
    code, oc = c576
    enc = I.GF2Encoder(code)
    rng = np.random.default_rng(21)
    cw = enc.encode(rng.integers(0, 2, size=(4, enc.K), dtype=np.uint8))
    L = (20.0 * (1.0 - 2.0 * cw)).astype(np.float32)
    r = oc.decode(L, alg=alg, max_iter=10)
    assert (r["iters"] == 1).all()
    assert np.array_equal(r["hard"], cw)
    r2 = oc.decode(L, alg=alg, max_iter=5, stop="none")   # further sweeps keep the word
    assert np.array_equal(r2["hard"], cw) and (r2["iters"] == 5).all()


@pytest.mark.parametrize("alg", ALGS32)
def test_sign_symmetry_bitwise(c576, alg):
    code, oc = c576
    fr = I.make_frames(code, 30, 2.0, seed=1300, encoder="zero")
    enc = I.GF2Encoder(code)
    cw = enc.encode(np.random.default_rng(3).integers(0, 2, size=(30, enc.K), dtype=np.uint8))
    flip = (1.0 - 2.0 * cw).astype(np.float32)
    a = oc.decode(fr.llr, alg=alg)
    b = oc.decode(fr.llr * flip, alg=alg)
    assert np.array_equal(a["iters"], b["iters"])
    assert np.array_equal(a["hard"] ^ cw, b["hard"])
    assert np.array_equal(a["soft"] * flip, b["soft"])


@pytest.mark.parametrize("alg", ALGS32)
def test_converged_words_satisfy_all_checks(c576, frames576, alg):
    code, oc = c576
    r = oc.decode(frames576.llr, alg=alg, max_iter=30)
    ok = r["iters"] > 0
    assert ok.sum() > 20
    assert not code.syndrome(r["hard"][ok]).any()
    assert code.syndrome(r["hard"][~ok]).any(axis=1).all()
    assert ((np.abs(r["iters"]) >= 1) & (np.abs(r["iters"]) <= 30)).all()


# --------------------------------------------------------------------------- Tables I, II
def test_operation_counts_match_tables_1_and_2(c576, frames576):
    code, oc = c576
    g = json.load(open(os.path.join(GOLDEN, "paper_tables_1_2_cbp.json")))
    E = code.E
    ev = {"E": E, "0": 0}
    per_sweep = {}
    for alg in ("cbp_sp", "lbp_sp"):
        c1 = oc.decode(frames576.llr[:1], alg=alg, max_iter=1, stop="none")["counts"]
        c2 = oc.decode(frames576.llr[:1], alg=alg, max_iter=2, stop="none")["counts"]
        per_sweep[alg] = {k: c2[k] - c1[k] for k in c1}
    cbp, lbp = per_sweep["cbp_sp"], per_sweep["lbp_sp"]
    u = g["updates_per_iteration"]
    assert cbp["v2c"] == ev[u["CBP"]["V2C"]] and cbp["c2v"] == ev[u["CBP"]["C2V"]]
    assert cbp["b2v"] == ev[u["CBP"]["B2V"]] and cbp["c2b"] == ev[u["CBP"]["C2B"]]
    assert lbp["v2c"] == ev[u["LBP"]["V2C"]] and lbp["c2v"] == ev[u["LBP"]["C2V"]]
    assert lbp["b2v"] == ev[u["LBP"]["B2V"]] and lbp["c2b"] == ev[u["LBP"]["C2B"]]
    w = g["calculations_per_update"]["CBP"]
    assert cbp["sums"] == w["V2C_sums"] * cbp["v2c"]
    assert cbp["products"] == w["B2V_products"] * cbp["b2v"] + w["C2B_products"] * cbp["c2b"]


# --------------------------------------------------------------------------- argument handling
def test_rejects_degenerate_codes():
    with pytest.raises(ValueError):
        O.OracleCode(np.array([[0, -1], [0, 0]], np.int32), 1)    # a degree-1 check
    with pytest.raises(ValueError):
        O.OracleCode(np.array([[0, 0, -1]], np.int32), 1)         # a variable in no check
    with pytest.raises(ValueError):
        O.OracleCode(np.array([[0, 4]], np.int32), 4)             # shift out of range


def test_empty_batch_and_one_sweep(c576, frames576):
    _, oc = c576
    r = oc.decode(frames576.llr[:0], alg="cbp_sp")
    assert r["hard"].shape == (0, 576)
    r = oc.decode(frames576.llr[:5], alg="cbp_sp", max_iter=1)
    assert (np.abs(r["iters"]) == 1).all()


def test_threads_do_not_change_results(c576, frames576):
    _, oc = c576
    a = oc.decode(frames576.llr, alg="cbp_sp", threads=1)
    b = oc.decode(frames576.llr, alg="cbp_sp", threads=4)
    for k in ("hard", "iters", "soft"):
        assert np.array_equal(a[k], b[k])
    assert a["counts"] == b["counts"]


@pytest.mark.parametrize("alg", ["cbp_sp", "fbp_sp"])
def test_noiseless_posteriors_grow_until_saturation(c576, alg):
    # with every channel LLR of the right sign, every message keeps that sign and the
    # update maps are increasing in the incoming magnitudes: starting from R = 0, the
    # posterior magnitudes can only grow from sweep to sweep (until phi saturates)
    code, oc = c576
    cw = np.zeros((2, code.N), np.uint8)
    L = np.full((2, code.N), 1.5, np.float64)
    L[1] = np.linspace(0.2, 3.0, code.N)
    prev = None
    for t in range(1, 7):
        r = oc.decode(L, alg=alg, max_iter=t, stop="none", precision=64)
        assert np.array_equal(r["hard"], cw)
        mag = np.abs(r["soft"])
        if prev is not None:
            assert np.all(mag >= prev - 1e-12), f"sweep {t}"
        prev = mag
    assert prev.min() > 3.0


# ------------------------------------------------------- flooding schedule on a loopy code
def textbook_bp(rows, L, sweeps, layered=False):
    """Sum-product BP as the textbook writes it (Sec. II, Eqs. s3e1, s3e2, s2e6), FP64, in
    the tanh form (the oracle uses the phi form).  Flooding: every check forms its V2C
    messages from the posteriors of the previous iteration minus its own old message, its
    C2V messages by the tanh rule over the other edges, and the posteriors are summed once
    all checks are done.  layered=True: the checks in ascending order, each updating its
    variables' posteriors at once (layered BP, Sec. II-B)."""
    L = np.asarray(L, np.float64)
    R = [np.zeros(len(vs)) for vs in rows]
    lam = L.copy()
    for _ in range(sweeps):
        for m, vs in enumerate(rows):
            q = lam[vs] - R[m]
            th = np.tanh(q / 2.0)
            new = np.empty(len(vs))
            for k in range(len(vs)):
                new[k] = 2.0 * np.arctanh(np.prod(np.delete(th, k)))
            if layered:
                lam[vs] = q + new
            R[m] = new
        if not layered:
            lam = L.copy()
            for m, vs in enumerate(rows):
                np.add.at(lam, vs, R[m])
    return lam


@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_fbp_equals_textbook_flooding_on_a_loopy_code(c576, sweeps):
    # On a cycle-free graph every schedule reaches the same exact marginals, so the tree
    # pins cannot see the schedule.  On the 576-bit code (girth 6 at least, many cycles)
    # the oracle's FP64 flooding BP must equal the textbook flooding recursion, and a
    # layered update would not.
    code, oc = c576
    rows = code.check_rows()
    fr = I.make_frames(code, 6, 1.0, seed=1300 + sweeps)
    r = oc.decode(fr.llr.astype(np.float64), alg="fbp_sp", precision=64, max_iter=sweeps,
                  stop="none")
    for f in range(fr.llr.shape[0]):
        ref = textbook_bp(rows, fr.llr[f], sweeps)
        assert np.abs(r["soft"][f] - ref).max() < 1e-6
        if sweeps > 1 or f == 0:  # the layered schedule differs after its first check
            lay = textbook_bp(rows, fr.llr[f], sweeps, layered=True)
            assert np.abs(r["soft"][f] - lay).max() > 1e-2


@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_cbp_flushed_posterior_equals_textbook_layered_bp(c576, sweeps):
    # CBP's flushed posterior after t sweeps is the posterior of layered BP after t sweeps
    # (Eqs. s4e9-s4e14: CBP defers each C2V message to the variable's next check).  The
    # layered recursion written above in the textbook tanh form, FP64, on the loopy 576-bit
    # code, against the oracle's CBP (S domain, phi form, deferred messages).
    code, oc = c576
    rows = code.check_rows()
    fr = I.make_frames(code, 6, 1.0, seed=1400 + sweeps)
    r = oc.decode(fr.llr.astype(np.float64), alg="cbp_sp", precision=64, max_iter=sweeps,
                  stop="none")
    for f in range(fr.llr.shape[0]):
        ref = textbook_bp(rows, fr.llr[f], sweeps, layered=True)
        assert np.abs(r["soft"][f] - ref).max() < 1e-6
