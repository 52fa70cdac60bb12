"""Several codes in one launch (cbp_decode_multi) against the oracle and the single-code
decoder.  Every frame must decode bit for bit as CBP-SP (Sec. IV) of its own code does."""
import ctypes as C
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_05286_gb300 import cbp, tune
from paper_2305_05286_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
# per code (in inputs.mixed_codes() order): batch and Eb/N0, chosen so that some frames
# converge within a few sweeps and others run out of sweeps
BATCHES = [37, 100, 5, 64, 0, 23, 50, 11]
EBN0 = [1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.5, 1.75]


@pytest.fixture(scope="module")
def mixed():
    qcs = I.mixed_codes()
    return qcs, [cbp.Code.from_qc(q) for q in qcs]


def frames_for(qcs, batches, seed):
    out = []
    for i, (q, b) in enumerate(zip(qcs, batches)):
        fr = I.make_frames(q, b, EBN0[i % len(EBN0)], seed=seed + i) if b else None
        out.append(np.zeros((0, q.N), np.float32) if fr is None else fr.llr)
    return out


def run_multi(codes, llrs_np, max_iter=20, **opts):
    x = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in llrs_np]
    res = cbp.decode_multi(codes, x, max_iter=max_iter, **opts)
    torch.cuda.synchronize()
    return [(cbp.unpack_bits(h, c.N).cpu().numpy(), it.cpu().numpy())
            for c, (h, it) in zip(codes, res)]


def run_single(code, llr_np, max_iter=20, stop="syndrome"):
    if llr_np.shape[0] == 0:
        return np.zeros((0, code.N), np.uint8), np.zeros((0,), np.int32)
    h, it, _ = code.decode(torch.from_numpy(llr_np).cuda(), max_iter=max_iter, stop=stop)
    torch.cuda.synchronize()
    return cbp.unpack_bits(h, code.N).cpu().numpy(), it.cpu().numpy()


def test_multi_matches_oracle_on_eight_codes(mixed):
    qcs, codes = mixed
    llrs = frames_for(qcs, BATCHES, seed=4100)
    got = run_multi(codes, llrs, max_iter=20)
    for q, a, (hard, iters) in zip(qcs, llrs, got):
        assert hard.shape == (a.shape[0], q.N)
        if a.shape[0] == 0:
            continue
        ref = O.OracleCode(q.base, q.Z).decode(a, alg="cbp_sp", max_iter=20, threads=THREADS)
        assert np.array_equal(iters, ref["iters"]), f"Z={q.Z}: iteration counts differ"
        assert np.array_equal(hard, ref["hard"]), f"Z={q.Z}: hard decisions differ"
    its = np.concatenate([g[1] for g in got])
    assert (its > 0).any() and (its < 0).any()


OPTS = [dict(),
        dict(frames_per_group=2),
        dict(chk_shared=0),
        dict(frames_per_group=2, chk_shared=0, rounds_per_chunk=1),
        dict(threads=384, ctas_per_sm=2, rounds_per_chunk=3),
        dict(rounds_per_chunk=1, ctas_per_sm=2),
        dict(tail_percent=-1),
        dict(tail_percent=100, rounds_per_chunk=8),
        dict(tail_percent=35, frames_per_group=2, rounds_per_chunk=5)]


@pytest.mark.parametrize("opts", OPTS, ids=[str(o) for o in OPTS])
def test_multi_options_equal_single_code_decode(mixed, opts):
    qcs, codes = mixed
    batches = [300, 250, 200, 150, 120, 90, 70, 60]
    llrs = frames_for(qcs, batches, seed=5200)
    got = run_multi(codes, llrs, max_iter=15, **opts)
    for c, a, (hard, iters) in zip(codes, llrs, got):
        h1, i1 = run_single(c, a, max_iter=15)
        assert np.array_equal(iters, i1), f"Z={c.Z} {opts}: iteration counts differ"
        assert np.array_equal(hard, h1), f"Z={c.Z} {opts}: hard decisions differ"


def test_multi_fixed_sweeps(mixed):
    qcs, codes = mixed
    llrs = frames_for(qcs, [20] * 8, seed=6300)
    got = run_multi(codes, llrs, max_iter=4, stop="none")
    for c, a, (hard, iters) in zip(codes, llrs, got):
        h1, i1 = run_single(c, a, max_iter=4, stop="none")
        assert np.array_equal(iters, i1) and np.array_equal(hard, h1)
        assert np.all(np.abs(iters) == 4)


def test_multi_single_item_and_repeated_codes(mixed):
    qcs, codes = mixed
    llr = frames_for(qcs[2:3], [333], seed=7100)[0]
    [(hard, iters)] = run_multi([codes[2]], [llr])
    h1, i1 = run_single(codes[2], llr)
    assert np.array_equal(iters, i1) and np.array_equal(hard, h1)
    # the same code twice in one launch, different frames
    a, b = llr[:200], llr[200:]
    (ha, ia), (hb, ib) = run_multi([codes[2], codes[2]], [a, b])
    assert np.array_equal(np.concatenate([ia, ib]), i1)
    assert np.array_equal(np.concatenate([ha, hb]), h1)


def test_multi_graph_capture_and_replay(mixed):
    qcs, codes = mixed
    batches = [64, 48, 32, 24, 16, 12, 8, 6]
    dev = torch.device("cuda")
    llrs = [torch.empty((b, c.N), dtype=torch.float32, device=dev) for c, b in zip(codes, batches)]
    hards = [torch.empty((b, c.words), dtype=torch.int32, device=dev) for c, b in zip(codes, batches)]
    its = [torch.empty((b,), dtype=torch.int32, device=dev) for b in batches]
    ws = torch.empty(cbp.multi_workspace_bytes(codes, batches), dtype=torch.uint8, device=dev)
    first = frames_for(qcs, batches, seed=8100)
    for t, a in zip(llrs, first):
        t.copy_(torch.from_numpy(a))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture (device setup, plan)
        cbp.decode_multi_into(codes, llrs, hards, its, 20, ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cbp.decode_multi_into(codes, llrs, hards, its, 20, ws)
    for seed in (8200, 8300):
        fresh = frames_for(qcs, batches, seed=seed)
        for t, a in zip(llrs, fresh):
            t.copy_(torch.from_numpy(a))
        g.replay()
        torch.cuda.synchronize()
        for c, a, h, it in zip(codes, fresh, hards, its):
            h1, i1 = run_single(c, a, max_iter=20)
            assert np.array_equal(it.cpu().numpy(), i1)
            assert np.array_equal(cbp.unpack_bits(h, c.N).cpu().numpy(), h1)


def test_multi_errors(mixed):
    qcs, codes = mixed
    L = cbp.lib()
    dev = torch.device("cuda")
    x = torch.zeros((4, codes[7].N), dtype=torch.float32, device=dev)
    h = torch.zeros((4, codes[7].words), dtype=torch.int32, device=dev)
    it = torch.zeros((4,), dtype=torch.int32, device=dev)
    items = (cbp._MultiItem * 9)()
    for i in range(9):
        items[i].code = codes[7]._h.value
        items[i].llr, items[i].hard_out, items[i].iters_out = x.data_ptr(), h.data_ptr(), it.data_ptr()
        items[i].batch = 4
    ws = torch.empty(1 << 24, dtype=torch.uint8, device=dev)
    o = cbp.multi_opts()
    # more items than one launch takes
    assert L.cbp_decode_multi(items, 9, 10, ws.data_ptr(), ws.numel(), None, C.byref(o)) == -1
    # Z = 384 does not fit a 256-thread CTA
    o = cbp.multi_opts(threads=256)
    assert L.cbp_decode_multi(items, 1, 10, ws.data_ptr(), ws.numel(), None, C.byref(o)) == -4
    # invalid options and sweep limit
    for bad in (cbp.multi_opts(frames_per_group=3), cbp.multi_opts(threads=100),
                cbp.multi_opts(threads=512, frames_per_group=2), cbp.multi_opts(ctas_per_sm=-1),
                cbp.multi_opts(tail_percent=101), cbp.multi_opts(tail_percent=-2)):
        assert L.cbp_decode_multi(items, 1, 10, ws.data_ptr(), ws.numel(), None, C.byref(bad)) == -1
    o = cbp.multi_opts()
    assert L.cbp_decode_multi(items, 1, 0, ws.data_ptr(), ws.numel(), None, C.byref(o)) == -1
    # workspace too small
    need = cbp.multi_workspace_bytes([codes[7]], [4])
    assert L.cbp_decode_multi(items, 1, 10, ws.data_ptr(), need - 1, None, C.byref(o)) == -5
    # misaligned llr
    items[0].llr = x.data_ptr() + 4
    assert L.cbp_decode_multi(items, 1, 10, ws.data_ptr(), ws.numel(), None, C.byref(o)) == -1
    # nothing to decode is not an error
    items[0].batch = 0
    assert L.cbp_decode_multi(items, 1, 10, None, 0, None, C.byref(o)) == 0
    torch.cuda.synchronize()


def test_tuner_picks_a_valid_option_set(mixed):
    qcs, codes = mixed
    batches = [128] * 8
    x = [torch.from_numpy(a).cuda() for a in frames_for(qcs, batches, seed=9100)]
    cands = tune.candidates(codes, rounds=(1, 4))
    best, table = tune.tune_multi(codes, x, max_iter=10, reps=1, cands=cands)
    assert table[0][1] == best and all(ms > 0 for ms, _ in table)
    res = cbp.decode_multi(codes, x, max_iter=10, **best)
    for c, a, (hh, ii) in zip(codes, x, res):
        h1, i1 = run_single(c, a.cpu().numpy(), max_iter=10)
        assert np.array_equal(ii.cpu().numpy(), i1)
        assert np.array_equal(cbp.unpack_bits(hh, c.N).cpu().numpy(), h1)


def test_tuner_cache(mixed, tmp_path):
    qcs, codes = mixed
    x = [torch.from_numpy(a).cuda() for a in frames_for(qcs, [64] * 8, seed=9300)]
    path = str(tmp_path / "tune.json")
    tune._CACHE.clear()
    a = tune.tuned_options(codes, x, max_iter=5, reps=1, path=path)
    tune._CACHE.clear()                      # a new process: read back from the file
    b = tune.tuned_options(codes, x, max_iter=5, reps=1, path=path)
    assert a == b and len(tune._CACHE) == 1
    # batch sizes in the same power-of-two bucket share the entry
    assert tune.cache_key(codes, [60] * 8) == tune.cache_key(codes, [64] * 8)
    assert tune.cache_key(codes, [65] * 8) != tune.cache_key(codes, [64] * 8)


def test_multi_weight1_last_instance_choice(mixed):
    # All eight mixed codes end the rows that hold their weight-1 column with it, so the
    # launch runs the instance without weight-1 branches; one code whose weight-1 column
    # comes first in its row switches the whole launch to the generic instance.
    qcs, codes = mixed
    batches = [40] * 8
    assert cbp.multi_launch_info(codes, batches)["weight1_last"] == 1
    assert cbp.multi_launch_info(codes, batches, frames_per_group=2)["weight1_last"] == 0
    base = qcs[2].base
    w1 = int(np.nonzero((base >= 0).sum(0) == 1)[0][0])
    perm = [w1] + [c for c in range(base.shape[1]) if c != w1]
    q_first = I.QCCode(np.ascontiguousarray(base[:, perm]), qcs[2].Z)
    c_first = cbp.Code.from_qc(q_first)
    codes2, qcs2 = codes[:7] + [c_first], qcs[:7] + [q_first]
    assert cbp.multi_launch_info(codes2, batches)["weight1_last"] == 0
    # a code with no frames does not decide the instance
    assert cbp.multi_launch_info(codes2, batches[:7] + [0])["weight1_last"] == 1
    llrs = frames_for(qcs2, [90, 80, 70, 60, 50, 40, 30, 120], seed=9500)
    got = run_multi(codes2, llrs, max_iter=15)
    for c, a, (hard, iters) in zip(codes2, llrs, got):
        h1, i1 = run_single(c, a, max_iter=15)
        assert np.array_equal(iters, i1) and np.array_equal(hard, h1), f"Z={c.Z}"
    ref = O.OracleCode(q_first.base, q_first.Z).decode(llrs[7], alg="cbp_sp", max_iter=15,
                                                        threads=THREADS)
    assert np.array_equal(got[7][1], ref["iters"]) and np.array_equal(got[7][0], ref["hard"])


def test_small_liftings_split_into_teams(mixed):
    # lane groups synchronise per base row only within their team; Z = 16 and Z = 32 CTAs
    # (48 and 24 groups) split into 12 teams of whole warps, Z = 384 into one per frame
    qcs, codes = mixed
    for c, groups, team in ((codes[0], 48, 4), (codes[1], 24, 2), (codes[7], 2, 1)):
        info = c.launch_info(20000)
        assert c.Z * info["team_lane_groups"] % 32 == 0
        assert (info["lane_groups_per_cta"], info["team_lane_groups"]) == (groups, team), c.Z


def test_multi_tail_of_one_round_chunks(mixed):
    # the last tail_percent % of an item's frames (whole rounds) run as one-round chunks
    qcs, codes = mixed
    B = 1600
    c_none = cbp.multi_launch_info([codes[7]], [B], tail_percent=-1)["chunks"]
    G = B // (4 * c_none)  # frames per round of this code's CTA
    assert G * 4 * c_none == B
    assert cbp.multi_launch_info([codes[7]], [B], tail_percent=100)["chunks"] == B // G
    tail = -(-(B * 20 // 100) // G) * G
    want = -(-(B - tail) // (4 * G)) + tail // G
    assert cbp.multi_launch_info([codes[7]], [B])["chunks"] == want
    assert cbp.multi_launch_info([codes[7]], [B], tail_percent=20)["chunks"] == want
