"""Seeded inputs: committed codes, both encoders and the channel model."""
import numpy as np
import pytest

from paper_2305_05286_gb300 import inputs as I


@pytest.mark.parametrize("fn,N,M,E,Z", [(I.code_576, 576, 288, 1416, 24),
                                         (I.code_2304, 2304, 1152, 5664, 96),
                                         (I.code_2304_hb, 2304, 1152, 5856, 96),
                                         (I.code_26112, 26112, 17664, 141312, 384)])
def test_committed_codes(fn, N, M, E, Z):
    c = fn()
    assert (c.N, c.M, c.E, c.Z) == (N, M, E, Z)
    assert I.is_lower_triangular(c) == (fn is not I.code_2304_hb)
    assert ((c.base >= 0).sum(axis=1) >= 2).all()
    assert ((c.base >= 0).sum(axis=0) >= 1).all()


def _has_any_4cycle(base, Z):
    mb, nb = base.shape
    for r in range(mb):
        for c in range(nb):
            s = base[r, c]
            if s >= 0:
                b = base.copy()
                b[r, c] = -1
                if I.four_cycle_at(b, Z, r, c, int(s)):
                    return True
    return False


def test_code_576_has_no_4cycles_and_column_weights():
    c = I.code_576()
    assert not _has_any_4cycle(c.base, c.Z)
    w = (c.base >= 0).sum(axis=0)
    assert (w[:12] == 3).all()          # systematic part: column weight 3
    assert w[23] == 1 and (w[12:23] == 2).all()   # lower bidiagonal parity


def test_four_cycle_detector_on_a_planted_cycle():
    b = -np.ones((2, 2), np.int32)
    b[0, 0], b[0, 1], b[1, 0] = 3, 5, 1
    assert I.four_cycle_at(b, 8, 1, 1, 3)      # 3 - 5 + 3 - 1 = 0
    assert not I.four_cycle_at(b, 8, 1, 1, 4)


def test_encoders_agree_and_give_codewords():
    c = I.code_576()
    enc = I.GF2Encoder(c)
    assert enc.K == 288
    rng = np.random.default_rng(5)
    info = rng.integers(0, 2, size=(50, enc.K), dtype=np.uint8)
    a = enc.encode(info)
    b = I.encode_lower_triangular(c, info)
    assert np.array_equal(a, b)
    assert not c.syndrome(a).any()
    assert np.array_equal(a[:, :288], info)   # systematic


def test_large_code_encoder_gives_codewords():
    c = I.code_26112()
    rng = np.random.default_rng(7)
    info = rng.integers(0, 2, size=(2, 22 * 384), dtype=np.uint8)
    x = I.encode_lower_triangular(c, info)
    assert not c.syndrome(x).any()


def test_torch_encoder_matches_numpy():
    torch = pytest.importorskip("torch")
    c = I.code_576()
    rng = np.random.default_rng(9)
    info = rng.integers(0, 2, size=(20, 288), dtype=np.uint8)
    a = I.encode_lower_triangular(c, info)
    b = I.encode_lower_triangular_torch(c, torch.from_numpy(info)).numpy()
    assert np.array_equal(a, b)


def test_channel_llr_statistics():
    c = I.code_576()
    fr = I.make_frames(c, 400, 2.0, seed=3, encoder="zero")
    s2 = I.awgn_sigma2(2.0, 0.5)
    assert abs(fr.llr.mean() - 2 / s2) < 0.02 * 2 / s2
    assert abs(fr.llr.var() - 4 / s2) < 0.03 * 4 / s2


def test_frames_are_reproducible():
    c = I.code_576()
    a = I.make_frames(c, 4, 1.5, seed=11)
    b = I.make_frames(c, 4, 1.5, seed=11)
    assert np.array_equal(a.llr, b.llr) and np.array_equal(a.codewords, b.codewords)


@pytest.mark.parametrize("fn,seed,degrees", [
    (I.code_peg_2048, 5, lambda: np.full(2048, 3)),
    (I.code_peg_irregular_2048, 6,
     lambda: I.peg_degrees(2048, {2: 0.45, 3: 0.3708, 4: 0.0307, 12: 0.1485})),
])
def test_peg_codes(fn, seed, degrees):
    qc = fn()
    assert qc.Z == 1 and qc.N == 2048 and qc.M == 1024
    H = (qc.base >= 0).astype(np.int64)
    want = np.asarray(degrees())
    # every variable keeps its degree (the committed graph places them in degree order)
    assert np.array_equal(np.sort(H.sum(0)), np.sort(want))
    # PEG keeps the graph free of 4-cycles at this size: two checks share <= 1 variable
    G = H @ H.T
    np.fill_diagonal(G, 0)
    assert G.max() <= 1
    # the committed file is what the generator gives for the seed
    rows = I.peg_graph(want, 1024, seed)
    assert rows == [list(np.nonzero(H[r])[0]) for r in range(1024)]


def test_peg_degrees_follow_the_edge_distribution():
    lam = {2: 0.45, 3: 0.3708, 4: 0.0307, 12: 0.1485}
    d = I.peg_degrees(2048, lam)
    assert d.size == 2048
    frac_edges = {i: (d == i).sum() * i / d.sum() for i in lam}
    for i in lam:
        assert abs(frac_edges[i] - lam[i]) < 0.003


def test_802_16e_parity_part_has_no_weight_one_column():
    qc = I.code_2304_hb()
    w = (qc.base >= 0).sum(0)
    assert w.min() >= 2 and w[12] == 3 and (w[13:] == 2).all()
    # its parity part is invertible: H has full rank, so K = N - M
    assert I.gf2_rank_dense(qc.dense_H()) == qc.M
    fr = I.make_frames(qc, 4, 2.0, seed=1)
    assert (qc.syndrome(fr.codewords) == 0).all()
