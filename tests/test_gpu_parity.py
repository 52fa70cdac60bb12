"""GPU decoders (through the C ABI) against the CPU oracle, element by element.

The oracle (FP32) and libcbp implement the same operation order and the same phi,
so hard decisions, iteration counts and soft outputs must agree bit for bit; that
is stricter than identical decisions/iterations plus soft outputs within 1e-5.
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_05286_gb300 import cbp
from paper_2305_05286_gb300 import inputs as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
ALGS = ["cbp_sp", "cbp_nms", "lbp_nms", "fbp_sp"]


def run_gpu(code, llr, alg, max_iter=30, stop="syndrome", alpha=0.75):
    x = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    hard, iters, soft = code.decode(x, max_iter=max_iter, alg=alg, alpha=alpha, stop=stop, soft=True)
    torch.cuda.synchronize()
    return (cbp.unpack_bits(hard, code.N).cpu().numpy(), iters.cpu().numpy(), soft.cpu().numpy())


def assert_parity(got, ref, what=""):
    hard, iters, soft = got
    assert np.array_equal(iters, ref["iters"]), f"{what}: iteration counts differ"
    assert np.array_equal(hard, ref["hard"]), f"{what}: hard decisions differ"
    diff = np.abs(soft.astype(np.float64) - ref["soft"].astype(np.float64))
    assert diff.max() <= 1e-5, f"{what}: soft outputs differ by {diff.max()}"
    assert np.array_equal(soft, ref["soft"]), f"{what}: soft outputs not bitwise equal"


@pytest.fixture(scope="module")
def code576():
    qc = I.code_576()
    return qc, cbp.Code.from_qc(qc), O.OracleCode(qc.base, qc.Z)


def test_phi_bitwise_equal_to_oracle():
    lo = np.float32(O.xlo32()).view(np.uint32)
    hi = np.float32(30.0).view(np.uint32)
    bits = np.arange(lo - 4096, hi + 4096, 61, dtype=np.uint32)
    x = np.concatenate([bits.view(np.float32),
                        np.array([0.0, 1e-30, 2.0, 30.0, 1e4, np.inf, np.nan], np.float32)])
    y = cbp.phi(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = O.phi32(x)
    assert np.array_equal(y.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("ebn0", [1.5, 2.0, 2.5])
@pytest.mark.parametrize("alg", ALGS)
def test_parity_576_2000_frames(code576, alg, ebn0):
    qc, code, oc = code576
    fr = I.make_frames(qc, 2000, ebn0, seed=1000 + int(round(ebn0 * 10)))
    ref = oc.decode(fr.llr, alg=alg, max_iter=30, threads=THREADS)
    assert_parity(run_gpu(code, fr.llr, alg), ref, f"{alg} @ {ebn0} dB")
    if alg == "cbp_sp":
        assert (ref["iters"] > 0).mean() > 0.5


@pytest.mark.parametrize("batch", [1, 3, 25, 151, 152, 153, 1000])
def test_ragged_batches_576(code576, batch):
    qc, code, oc = code576
    fr = I.make_frames(qc, batch, 1.75, seed=77 + batch)
    for alg in ALGS:
        ref = oc.decode(fr.llr, alg=alg, max_iter=20, threads=THREADS)
        assert_parity(run_gpu(code, fr.llr, alg, max_iter=20), ref, f"{alg} batch {batch}")


@pytest.mark.parametrize("max_iter,stop", [(1, "syndrome"), (2, "none"), (7, "none")])
def test_sweep_limits_and_fixed_sweeps(code576, max_iter, stop):
    qc, code, oc = code576
    fr = I.make_frames(qc, 300, 2.0, seed=500 + max_iter)
    for alg in ALGS:
        ref = oc.decode(fr.llr, alg=alg, max_iter=max_iter, stop=stop, threads=THREADS)
        assert_parity(run_gpu(code, fr.llr, alg, max_iter=max_iter, stop=stop), ref, alg)


@pytest.mark.parametrize("Z", [1, 4, 7, 32, 33])
def test_other_liftings(code576, Z):
    """Same base graph lifted by other Z (several frames per warp, Z > 32, Z = 1)."""
    qc = I.relift(code576[0], Z)
    code = cbp.Code.from_qc(qc)
    oc = O.OracleCode(qc.base, qc.Z)
    fr = I.make_frames(qc, 257, 2.5, seed=900 + Z, encoder="zero")
    for alg in ALGS:
        ref = oc.decode(fr.llr, alg=alg, max_iter=15, threads=THREADS)
        assert_parity(run_gpu(code, fr.llr, alg, max_iter=15), ref, f"{alg} Z={Z}")


def test_parity_2304():
    qc = I.code_2304()
    code = cbp.Code.from_qc(qc)
    oc = O.OracleCode(qc.base, qc.Z)
    fr = I.make_frames(qc, 400, 1.75, seed=6017)
    for alg in ALGS:
        ref = oc.decode(fr.llr, alg=alg, max_iter=10, threads=THREADS)
        assert_parity(run_gpu(code, fr.llr, alg, max_iter=10), ref, alg)


@pytest.fixture(scope="module")
def large():
    qc = I.code_26112()
    return qc, cbp.Code.from_qc(qc), O.OracleCode(qc.base, qc.Z)


@pytest.mark.parametrize("alg", ALGS)
def test_parity_26112_small_batch(large, alg):
    qc, code, oc = large
    llr, cw = I.make_frames_torch(qc, 96, 0.75, seed=2075)
    ref = oc.decode(llr.cpu().numpy(), alg=alg, max_iter=20, threads=THREADS)
    assert_parity(run_gpu(code, llr.cpu().numpy(), alg, max_iter=20), ref, alg)


def test_cbp_nms_with_per_edge_messages(code576, large, monkeypatch):
    """CBP min-sum with its C2V messages kept per edge (CBP_PLAN_NMS_R=1, the layout of the
    log-tanh kernel) instead of rebuilt from (min1, min2, argmin, sign bits): bitwise equal
    to the oracle, which keeps them per edge too."""
    monkeypatch.setenv("CBP_PLAN_NMS_R", "1")
    qc, code, oc = code576
    fr = I.make_frames(qc, 700, 2.0, seed=1717)
    ref = oc.decode(fr.llr, alg="cbp_nms", max_iter=30, threads=THREADS)
    assert_parity(run_gpu(code, fr.llr, "cbp_nms"), ref, "cbp_nms per-edge R, 576")
    qc, code, oc = large
    llr, _ = I.make_frames_torch(qc, 96, 2.5, seed=2076)
    ref = oc.decode(llr.cpu().numpy(), alg="cbp_nms", max_iter=20, threads=THREADS)
    assert_parity(run_gpu(code, llr.cpu().numpy(), "cbp_nms", max_iter=20), ref,
                  "cbp_nms per-edge R, 26112")


def gpu_syndrome(qc, hard_bits):
    """H x^T on the GPU with torch gathers (independent of libcbp)."""
    rows = torch.from_numpy(np.stack([np.pad(r, (0, 32 - len(r)), constant_values=-1)
                                      for r in qc.check_rows()])).cuda()
    valid = rows >= 0
    g = hard_bits[:, rows.clamp(min=0)] * valid
    return g.sum(dim=2) & 1


def test_full_size_26112_sampled(large):
    """65536 frames in the benchmark's launch configuration; 12 frames re-decoded by the oracle."""
    qc, code, oc = large
    B = 65536
    info = code.launch_info(B)  # two 384-lane frames per SM, weight-1-last instance
    assert info["weight1_last"] == 1 and info["frames_per_sm"] == 2
    assert 0 < info["shared_bytes"] <= 227 * 1024
    llr, cw = I.make_frames_torch(qc, B, 1.0, seed=2100)
    hard, iters, soft = code.decode(llr, max_iter=20, alg="cbp_sp", soft=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pick = np.concatenate([[0, 1, B // 2, B - 2, B - 1], rng.choice(B, 7, replace=False)])
    sub = llr[torch.from_numpy(pick).cuda()].cpu().numpy()
    ref = oc.decode(sub, alg="cbp_sp", max_iter=20, threads=THREADS)
    got = (cbp.unpack_bits(hard[pick], qc.N).cpu().numpy(), iters[pick].cpu().numpy(),
           soft[pick].cpu().numpy())
    assert_parity(got, ref, "26112 sampled")
    # properties at full size: converged frames satisfy every check, others do not
    bitsu = cbp.unpack_bits(hard[:2048], qc.N).to(torch.int32)
    syn = gpu_syndrome(qc, bitsu).any(dim=1).cpu().numpy()
    it = iters[:2048].cpu().numpy()
    assert not syn[it > 0].any() and syn[it < 0].all()
    assert ((np.abs(iters.cpu().numpy()) >= 1) & (np.abs(iters.cpu().numpy()) <= 20)).all()


def test_full_size_26112_at_the_operating_point(large):
    """The benchmark's launch (65536 frames of the 26112-bit code at 2.5 dB, the bench's
    own frames) against the oracle on 4 frames of every frame slot: the slot's first frame,
    its second (the first reload), one from the middle of its run and its last, so every
    slot and several reload rounds are compared bit for bit (hard decisions, iteration
    counts, soft outputs)."""
    qc, code, oc = large
    B = 65536
    info = code.launch_info(B)
    slots = info["ctas"] * info["lane_groups_per_cta"] * info["frames_per_lane_group"]
    assert info["frame_parallel"] == 0 and slots >= 152
    llr, cw = I.make_frames_torch(qc, B, 2.5, seed=2000)
    hard, iters, soft = code.decode(llr, max_iter=20, alg="cbp_sp", soft=True)
    torch.cuda.synchronize()
    k = np.arange(slots)
    last = k + ((B - 1 - k) // slots) * slots
    pick = np.unique(np.concatenate([k, k + slots, k + 100 * slots, last]))
    assert pick.size >= 1024 and pick.max() < B
    idx = torch.from_numpy(pick).cuda()
    ref = oc.decode(llr[idx].cpu().numpy(), alg="cbp_sp", max_iter=20, threads=THREADS)
    got = (cbp.unpack_bits(hard[idx], qc.N).cpu().numpy(), iters[idx].cpu().numpy(),
           soft[idx].cpu().numpy())
    assert_parity(got, ref, "26112 at 2.5 dB, every slot")
    it = iters.cpu().numpy()
    assert (it != 0).all() and np.abs(it).max() <= 20 and np.abs(it).mean() > 3


@pytest.mark.parametrize("alg", ALGS)
def test_sign_symmetry_on_gpu(code576, alg):
    qc, code, oc = code576
    fr = I.make_frames(qc, 200, 2.0, seed=31, encoder="zero")
    enc = I.GF2Encoder(qc)
    cw = enc.encode(np.random.default_rng(8).integers(0, 2, size=(200, enc.K), dtype=np.uint8))
    flip = (1.0 - 2.0 * cw).astype(np.float32)
    a = run_gpu(code, fr.llr, alg)
    b = run_gpu(code, fr.llr * flip, alg)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[0] ^ cw, b[0])
    assert np.array_equal(a[2] * flip, b[2])


def test_tree_code_on_gpu():
    base = -np.ones((5, 10), np.int32)
    for r, vs in enumerate([(0, 1, 2), (2, 3, 4), (4, 5, 6), (1, 7), (6, 8, 9)]):
        base[r, list(vs)] = 0
    code = cbp.Code(base, 1)
    oc = O.OracleCode(base, 1)
    llr = np.random.default_rng(2).normal(1.0, 1.5, size=(64, 10)).astype(np.float32)
    for alg in ALGS:
        assert_parity(run_gpu(code, llr, alg, max_iter=12, stop="none"),
                      oc.decode(llr, alg=alg, max_iter=12, stop="none"), alg)


def test_error_paths(code576):
    qc, code, oc = code576
    x = torch.zeros((8, qc.N), dtype=torch.float32, device="cuda")
    hard = torch.full((8, code.words), 7, dtype=torch.int32, device="cuda")
    iters = torch.full((8,), 7, dtype=torch.int32, device="cuda")
    need = code.workspace_bytes(8)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    L = cbp.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert L.cbp_decode(code._h, x.data_ptr(), hard.data_ptr(), iters.data_ptr(), 30, 8,
                        ws.data_ptr(), need - 1, s) == -5
    assert L.cbp_decode(code._h, x.data_ptr() + 4, hard.data_ptr(), iters.data_ptr(), 30, 8,
                        ws.data_ptr(), need, s) == -1
    assert L.cbp_decode(code._h, x.data_ptr(), hard.data_ptr(), iters.data_ptr(), 0, 8,
                        ws.data_ptr(), need, s) == -1
    assert L.cbp_decode(code._h, x.data_ptr(), hard.data_ptr(), iters.data_ptr(), 30, 0,
                        ws.data_ptr(), need, s) == 0
    torch.cuda.synchronize()
    assert (hard == 7).all() and (iters == 7).all()     # nothing launched
    big = np.zeros((1, 40), np.int32)                    # row degree 40 > 32
    bigc = cbp.Code(np.vstack([big, big]), 3)
    with pytest.raises(cbp.CbpError):
        bigc.workspace_bytes(4, alg="lbp_nms")
    assert bigc.workspace_bytes(4, alg="cbp_sp") > 0     # CBP has no per-row pool limit
    with pytest.raises(cbp.CbpError) as e:               # one lane per thread: Z <= 1024
        cbp.Code(qc.base.clip(max=0), 1025)
    assert e.value.status == -4


def test_wide_rows_cbp_only():
    """Row degree 40: CBP has no per-row register pool, so it decodes; the oracle agrees."""
    rng = np.random.default_rng(12)
    base = np.where(rng.random((4, 48)) < 0.85, rng.integers(0, 8, (4, 48)), -1).astype(np.int32)
    base[:, :2] = 0
    base[0, 2:] = np.where(base[0, 2:] < 0, 3, base[0, 2:])
    qc = I.QCCode(base, 8)
    code = cbp.Code.from_qc(qc)
    oc = O.OracleCode(base, 8)
    llr = (3.0 + 2.0 * rng.standard_normal((40, qc.N))).astype(np.float32)
    for alg in ("cbp_sp", "cbp_nms"):
        assert_parity(run_gpu(code, llr, alg, max_iter=8), oc.decode(llr, alg=alg, max_iter=8), alg)


def test_edge_ceiling_runs_and_checks_its_sink():
    import ctypes as C
    r = cbp.edge_ceiling(iters=64)
    assert r["ctas"] >= torch.cuda.get_device_properties(0).multi_processor_count
    assert r["edge_updates_per_s"] > 1e9
    n, used = C.c_int64(), C.c_int()
    small = torch.empty(512, dtype=torch.float32, device="cuda")
    rc = cbp.lib().cbp_edge_ceiling(2, 8, small.data_ptr(), small.numel(), None, C.byref(n),
                                    C.byref(used))
    assert rc == -1 and n.value == 0   # two CTAs need 1024 sink floats: nothing launched
    torch.cuda.synchronize()


@pytest.mark.parametrize("chunk", [1, 7, 100, 5000])
def test_decode_host_matches_device_decode(code576, chunk):
    qc, code, _ = code576
    fr = I.make_frames(qc, 333, 1.75, seed=4242)
    host = torch.from_numpy(fr.llr).pin_memory()
    for alg in ("cbp_sp", "lbp_nms"):
        h_ref, i_ref, _ = code.decode(host.cuda(), max_iter=20, alg=alg)
        h, i = code.decode_host(host, max_iter=20, alg=alg, chunk=chunk)
        assert not h.is_cuda and torch.equal(i, i_ref.cpu()) and torch.equal(h, h_ref.cpu())
    # pageable host memory works too (copies serialise)
    h, i = code.decode_host(torch.from_numpy(fr.llr), max_iter=20, chunk=64)
    h_ref, i_ref, _ = code.decode(host.cuda(), max_iter=20)
    assert torch.equal(i, i_ref.cpu()) and torch.equal(h, h_ref.cpu())


@pytest.mark.parametrize("alpha", [0.625, 0.8125, 1.0])
def test_min_sum_normalisations(code576, alpha):
    qc, code, oc = code576
    fr = I.make_frames(qc, 400, 2.25, seed=900 + int(alpha * 1000))
    for alg in ("cbp_nms", "lbp_nms"):
        ref = oc.decode(fr.llr, alg=alg, max_iter=30, alpha=alpha, threads=THREADS)
        assert_parity(run_gpu(code, fr.llr, alg, alpha=alpha), ref, f"{alg} alpha {alpha}")


@pytest.mark.parametrize("ebn0", [2.0, 3.0, 4.5])
def test_paper_literal_window_stop(code576, ebn0):
    qc, code, oc = code576
    fr = I.make_frames(qc, 700, ebn0, seed=1300 + int(ebn0 * 10))
    ref = oc.decode(fr.llr, alg="cbp_sp", max_iter=25, stop="window", threads=THREADS)
    x = torch.from_numpy(fr.llr).cuda()
    hard, iters, _ = code.decode(x, max_iter=25, alg="cbp_sp", stop="window")
    torch.cuda.synchronize()
    assert np.array_equal(iters.cpu().numpy(), ref["iters"])
    assert np.array_equal(cbp.unpack_bits(hard, code.N).cpu().numpy(), ref["hard"])


@pytest.mark.parametrize("Z", [1, 7, 32, 96])
def test_paper_literal_window_stop_liftings(Z):
    # Z = 1: one lane per group, many groups per team; 7: warps straddle groups; 32/96:
    # whole warps; noiseless-ish frames make the window fill in the middle of rows
    qc = I.relift(I.code_576(), Z)
    code = cbp.Code.from_qc(qc)
    oc = O.OracleCode(qc.base, qc.Z)
    for ebn0, seed in ((3.5, 1), (6.0, 2)):
        fr = I.make_frames(qc, 300, ebn0, seed=seed + Z)
        ref = oc.decode(fr.llr, alg="cbp_sp", max_iter=15, stop="window", threads=THREADS)
        hard, iters, _ = code.decode(torch.from_numpy(fr.llr).cuda(), max_iter=15, stop="window")
        torch.cuda.synchronize()
        assert np.array_equal(iters.cpu().numpy(), ref["iters"]), f"Z={Z} {ebn0} dB"
        assert np.array_equal(cbp.unpack_bits(hard, code.N).cpu().numpy(), ref["hard"])


def test_window_stop_option_checks(code576):
    qc, code, _ = code576
    x = torch.zeros((4, code.N), dtype=torch.float32, device="cuda")
    for alg in ("cbp_nms", "lbp_nms", "fbp_sp"):
        with pytest.raises(cbp.CbpError):
            code.decode(x, max_iter=5, alg=alg, stop="window")
    with pytest.raises(cbp.CbpError):   # no soft output in this mode
        code.decode(x, max_iter=5, stop="window", soft=True)


@pytest.mark.parametrize("fn", [I.code_peg_2048, I.code_peg_irregular_2048])
def test_peg_codes_all_decoders(fn):
    # a general sparse code as Z = 1: one lane per group, 1024 base rows of degree ~6
    qc = fn()
    code = cbp.Code.from_qc(qc)
    oc = O.OracleCode(qc.base, qc.Z)
    fr = I.make_frames(qc, 96, 1.75, seed=77)
    for alg, stop in (("cbp_sp", "syndrome"), ("cbp_sp", "window"), ("fbp_sp", "syndrome"),
                      ("lbp_nms", "syndrome"), ("cbp_nms", "syndrome")):
        ref = oc.decode(fr.llr, alg=alg, max_iter=40, stop=stop, alpha=1.0, threads=THREADS)
        hard, iters, _ = code.decode(torch.from_numpy(fr.llr).cuda(), max_iter=40, alg=alg,
                                     alpha=1.0, stop=stop)
        torch.cuda.synchronize()
        assert np.array_equal(iters.cpu().numpy(), ref["iters"]), f"{alg} {stop}"
        assert np.array_equal(cbp.unpack_bits(hard, code.N).cpu().numpy(), ref["hard"])


def test_device_status_reports_non_finite_llrs(code576):
    qc, code, _ = code576
    fr = I.make_frames(qc, 40, 2.0, seed=31)
    assert code.device_status() == 0
    clean = run_gpu(code, fr.llr, "cbp_sp")
    assert code.device_status() == 0          # finite input: nothing to report
    bad = fr.llr.copy()
    bad[7, 100] = np.nan
    bad[21, 3] = np.inf
    for alg in ALGS:
        got = run_gpu(code, bad, alg)
        assert code.device_status() == cbp.STATUS_NONFINITE_LLR, alg
        assert code.device_status() == 0      # read and cleared
        if alg == "cbp_sp":                   # the other frames are not affected
            keep = np.ones(40, bool)
            keep[[7, 21]] = False
            assert np.array_equal(got[1][keep], clean[1][keep])
            assert np.array_equal(got[0][keep], clean[0][keep])
    w = torch.ones((3, qc.mb), device="cuda")
    cbp.weighted_cbp(code, torch.from_numpy(bad).cuda(), w, 3)
    torch.cuda.synchronize()
    assert code.device_status() == cbp.STATUS_NONFINITE_LLR


@pytest.mark.parametrize("chk,fpt", [("0", "1"), ("1", "1"), ("0", "2"), ("1", "2")])
def test_every_cbp_sp_layout_variant(code576, monkeypatch, chk, fpt):
    # the planner picks one variant per code; force each in turn (check state in shared
    # memory or the workspace, one or two interleaved frames per lane group)
    qc, code, oc = code576
    monkeypatch.setenv("CBP_PLAN_CHK", chk)
    monkeypatch.setenv("CBP_PLAN_FPT", fpt)
    info = code.launch_info(777)
    assert info["check_state_shared"] == int(chk) and info["frames_per_lane_group"] == int(fpt)
    fr = I.make_frames(qc, 777, 2.0, seed=4000 + int(chk) * 10 + int(fpt))
    for alg in ("cbp_sp", "cbp_nms"):
        if alg == "cbp_nms" and fpt == "2":
            continue                      # min-sum kernels run one frame per lane group
        ref = oc.decode(fr.llr, alg=alg, max_iter=25, threads=THREADS)
        assert_parity(run_gpu(code, fr.llr, alg, max_iter=25), ref, f"{alg} chk {chk} fpt {fpt}")


@pytest.mark.parametrize("chk,fpt", [("0", "1"), ("1", "1"), ("1", "2")])
@pytest.mark.parametrize("pos", [0, 11])
def test_weight1_column_not_last_in_its_row(monkeypatch, pos, chk, fpt):
    # Every code above ends the rows holding a weight-1 column with that column, and the
    # planner then runs the kernel instance without weight-1 branches in its edge loop.
    # Moving the weight-1 column to the front (or the middle) of the base matrix makes
    # the generic instance run; the oracle decodes the permuted code on its own terms.
    base = I.code_576().base
    w1 = int(np.nonzero((base >= 0).sum(0) == 1)[0][0])
    perm = [c for c in range(base.shape[1]) if c != w1]
    perm.insert(pos, w1)
    qc = I.QCCode(np.ascontiguousarray(base[:, perm]), 24)
    monkeypatch.setenv("CBP_PLAN_CHK", chk)
    monkeypatch.setenv("CBP_PLAN_FPT", fpt)
    code = cbp.Code.from_qc(qc)
    info = code.launch_info(300)
    assert info["weight1_last"] == 0 and info["check_state_shared"] == int(chk)
    fr = I.make_frames(qc, 300, 2.0, seed=4300 + pos)
    ref = O.OracleCode(qc.base, qc.Z).decode(fr.llr, alg="cbp_sp", max_iter=25, threads=THREADS)
    assert (ref["iters"] < 0).any() and (ref["iters"] > 1).any()
    assert_parity(run_gpu(code, fr.llr, "cbp_sp", max_iter=25), ref, f"weight-1 column at {pos}")


@pytest.mark.parametrize("Z", [512, 1000, 1024])
def test_lifts_above_384(Z):
    # Z = 512: one lane group in a 768-thread CTA (idle lanes, one CTA-wide team);
    # Z = 1000: only the 1024-thread instance fits, and Z is off the warp grid;
    # Z = 1024: the largest lifting the library takes (every thread of the CTA a lane)
    qc = I.relift(I.code_576(), 24)
    qc = I.QCCode(qc.base, Z)             # same shifts (all < 24), lifted by Z
    code = cbp.Code.from_qc(qc)
    oc = O.OracleCode(qc.base, qc.Z)
    assert code.launch_info(40)["threads_per_cta"] > 384
    fr = I.make_frames(qc, 40, 2.0, seed=Z)
    ref = oc.decode(fr.llr, alg="cbp_sp", max_iter=20, threads=THREADS)
    assert_parity(run_gpu(code, fr.llr, "cbp_sp", max_iter=20), ref, f"Z={Z}")


def test_concurrent_streams_and_host_threads(code576):
    # the header's promise: calls with distinct outputs and workspaces may run concurrently
    import threading

    qc, code, _ = code576
    frs = [I.make_frames(qc, 600, 2.0, seed=7000 + i).llr for i in range(4)]
    ref = [run_gpu(code, a, "cbp_sp") for a in frs]
    streams = [torch.cuda.Stream() for _ in frs]
    xs = [torch.from_numpy(a).cuda() for a in frs]
    outs = [(torch.empty((600, code.words), dtype=torch.int32, device="cuda"),
             torch.empty((600,), dtype=torch.int32, device="cuda")) for _ in frs]
    wss = [torch.empty(code.workspace_bytes(600), dtype=torch.uint8, device="cuda") for _ in frs]
    torch.cuda.synchronize()

    def work(i):
        with torch.cuda.stream(streams[i]):
            code.decode_into(xs[i], outs[i][0], outs[i][1], max_iter=30, workspace=wss[i],
                             stream=streams[i])

    threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    for (h, it), (rh, ri, _) in zip(outs, ref):
        assert np.array_equal(it.cpu().numpy(), ri)
        assert np.array_equal(cbp.unpack_bits(h, code.N).cpu().numpy(), rh)


def test_decode_from_host_memory_on_another_stream(code576):
    # the copy runs on the current stream and the decoding on `stream`: the decoding must
    # wait for the copy, and the results must wait for the decoding
    qc, code, _ = code576
    fr = I.make_frames(qc, 3000, 2.0, seed=7300)
    ref = run_gpu(code, fr.llr, "cbp_sp")
    s = torch.cuda.Stream()
    for pinned in (True, False):
        host = torch.from_numpy(fr.llr)
        host = host.pin_memory() if pinned else host
        h, it, _ = code.decode(host, max_iter=30, stream=s)
        torch.cuda.synchronize()
        assert not h.is_cuda and np.array_equal(it.numpy(), ref[1])
        assert np.array_equal(cbp.unpack_bits(h, code.N).numpy(), ref[0])


def test_decode_host_with_the_window_stop(code576):
    qc, code, oc = code576
    fr = I.make_frames(qc, 250, 3.0, seed=7100)
    ref = oc.decode(fr.llr, alg="cbp_sp", max_iter=25, stop="window", threads=THREADS)
    h, i = code.decode_host(torch.from_numpy(fr.llr).pin_memory(), max_iter=25, stop="window",
                            chunk=64)
    assert np.array_equal(i.numpy(), ref["iters"])
    assert np.array_equal(cbp.unpack_bits(h, code.N).numpy(), ref["hard"])


FP_CASES = [("576", 2000, 2.0, "syndrome"), ("576", 257, 1.5, "none"),
            ("2304", 300, 1.75, "syndrome"), ("z4", 1000, 2.5, "syndrome"),
            ("z1", 333, 2.5, "syndrome"), ("peg", 700, 2.0, "syndrome")]


@pytest.mark.parametrize("name,batch,ebn0,stop", FP_CASES)
def test_frame_parallel_kernel(monkeypatch, name, batch, ebn0, stop):
    # One frame per thread, the whole sequential schedule per thread, state element-major
    # with the frame slot innermost.  The planner picks it where the lane-parallel plan
    # would keep few lanes busy (the Z = 1 PEG code); elsewhere it is forced on.  Bit for
    # bit against the oracle, soft output too.
    qc = {"576": I.code_576, "2304": I.code_2304, "peg": I.code_peg_2048,
          "z4": lambda: I.relift(I.code_576(), 4), "z1": lambda: I.relift(I.code_576(), 1)}[name]()
    code = cbp.Code.from_qc(qc)
    if name == "peg":  # the planner's choice is the wavefront kernel; without it, this one
        assert code.launch_info(batch)["level_schedule"] == 1
        monkeypatch.setenv("CBP_PLAN_LEVEL", "0")
        assert code.launch_info(batch)["frame_parallel"] == 1
        monkeypatch.setenv("CBP_PLAN_FP", "0")
        assert code.launch_info(batch)["frame_parallel"] == 0
    else:
        assert code.launch_info(batch)["frame_parallel"] == 0
    monkeypatch.setenv("CBP_PLAN_FP", "1")
    info = code.launch_info(batch)
    assert info["frame_parallel"] == 1 and info["threads_per_cta"] == 256
    fr = I.make_frames(qc, batch, ebn0, seed=4700 + batch, encoder="gf2" if qc.N <= 4096 else "tri")
    ref = O.OracleCode(qc.base, qc.Z).decode(fr.llr, alg="cbp_sp", max_iter=20, stop=stop,
                                             threads=THREADS)
    assert_parity(run_gpu(code, fr.llr, "cbp_sp", max_iter=20, stop=stop), ref, f"{name} fp")
    assert (ref["iters"] > 0).any()


LEVEL_CASES = [("peg", 700, 2.0, "syndrome", 64, "1"), ("peg", 129, 2.5, "none", 32, "0"),
               ("peg", 300, 2.0, "syndrome", 96, "0"),
               ("pegirr", 333, 1.75, "syndrome", 64, "0"), ("pegirr", 64, 1.5, "syndrome", 128, "1"),
               ("z1", 500, 2.5, "syndrome", 64, "1"), ("z4", 300, 2.0, "syndrome", 96, "0"),
               ("576", 257, 1.5, "syndrome", 64, "1"), ("2304", 100, 1.75, "syndrome", 64, "0")]


@pytest.mark.parametrize("name,batch,ebn0,stop,lanes,shrec", LEVEL_CASES)
def test_level_schedule_kernel(monkeypatch, name, batch, ebn0, stop, lanes, shrec):
    # The checks of the expanded graph by level (a check's level is one more than that of
    # the previous check of any of its variables), a level's checks on parallel lanes of one
    # group per frame.  The planner picks it for the Z = 1 PEG codes; elsewhere it is forced
    # on.  Lane groups of 32 to 128 lanes, levels wider and narrower than a group, edge
    # records in shared or global memory, frames past a group's first, stop modes, soft
    # output: bit for bit against the oracle.
    qc = {"576": I.code_576, "2304": I.code_2304, "peg": I.code_peg_2048,
          "pegirr": I.code_peg_irregular_2048,
          "z4": lambda: I.relift(I.code_576(), 4), "z1": lambda: I.relift(I.code_576(), 1)}[name]()
    code = cbp.Code.from_qc(qc)
    if name.startswith("peg"):
        info = code.launch_info(batch)
        assert info["level_schedule"] == 1 and info["frame_parallel"] == 0
    monkeypatch.setenv("CBP_PLAN_LEVEL", "1")
    monkeypatch.setenv("CBP_LVL_LANES", str(lanes))
    monkeypatch.setenv("CBP_LVL_SHREC", shrec)
    info = code.launch_info(batch)
    assert info["level_schedule"] == 1 and info["threads_per_cta"] % lanes == 0
    fr = I.make_frames(qc, batch, ebn0, seed=4900 + batch, encoder="gf2" if qc.N <= 4096 else "tri")
    ref = O.OracleCode(qc.base, qc.Z).decode(fr.llr, alg="cbp_sp", max_iter=20, stop=stop,
                                             threads=THREADS)
    assert_parity(run_gpu(code, fr.llr, "cbp_sp", max_iter=20, stop=stop), ref, f"{name} level")
    if stop == "syndrome":
        assert (ref["iters"] > 0).any()


LBP_LEVEL_CASES = [("peg", 700, 2.0, 0.75, 96, "1"), ("peg", 300, 1.75, 1.0, 64, "0"),
                   ("pegirr", 333, 2.0, 0.75, 96, "1"), ("pegirr", 100, 1.5, 0.8125, 32, "0"),
                   ("576", 257, 2.0, 0.75, 64, "1"), ("z4", 300, 2.5, 0.75, 96, "0"),
                   ("2304", 100, 2.0, 1.0, 64, "1")]


@pytest.mark.parametrize("alg", ["lbp_nms", "cbp_nms", "fbp_sp"])
@pytest.mark.parametrize("name,batch,ebn0,alpha,lanes,shv", LBP_LEVEL_CASES)
def test_level_schedule_comparators(monkeypatch, alg, name, batch, ebn0, alpha, lanes, shv):
    # Layered min-sum, CBP min-sum (both on the wavefront schedule) and flooding BP (all
    # checks at once) with lane groups per frame: the planner's choice for the Z = 1 PEG
    # codes, forced elsewhere; normalisations, lane groups, edge tables in shared or global
    # memory, soft output: bit for bit against the oracle.
    qc = {"576": I.code_576, "2304": I.code_2304, "peg": I.code_peg_2048,
          "pegirr": I.code_peg_irregular_2048,
          "z4": lambda: I.relift(I.code_576(), 4)}[name]()
    code = cbp.Code.from_qc(qc)
    if name.startswith("peg"):
        assert code.launch_info(batch, alg=alg)["level_schedule"] == 1
    monkeypatch.setenv("CBP_PLAN_LEVEL", "1")
    monkeypatch.setenv("CBP_LVL_LANES", str(lanes))
    monkeypatch.setenv("CBP_LVL_SHREC", shv)
    assert code.launch_info(batch, alg=alg)["level_schedule"] == 1
    fr = I.make_frames(qc, batch, ebn0, seed=5100 + batch)
    ref = O.OracleCode(qc.base, qc.Z).decode(fr.llr, alg=alg, max_iter=20, alpha=alpha,
                                             threads=THREADS)
    got = run_gpu(code, fr.llr, alg, max_iter=20, alpha=alpha)
    assert_parity(got, ref, f"{name} {alg} level")
    assert (ref["iters"] > 0).any()


def test_level_schedule_host_decode_and_status(monkeypatch):
    # the host-buffer entry point and the non-finite-LLR status through the same kernel
    qc = I.code_peg_2048()
    code = cbp.Code.from_qc(qc)
    assert code.launch_info(700)["level_schedule"] == 1
    fr = I.make_frames(qc, 700, 2.0, seed=4810)
    host = torch.from_numpy(fr.llr).pin_memory()
    h_ref, i_ref, _ = code.decode(host.cuda(), max_iter=20)
    h, i = code.decode_host(host, max_iter=20, chunk=256)
    assert torch.equal(i, i_ref.cpu()) and torch.equal(h, h_ref.cpu())
    code.device_status()
    bad = fr.llr.copy()
    bad[5, 7] = np.nan
    code.decode(torch.from_numpy(bad).cuda(), max_iter=5)
    torch.cuda.synchronize()
    assert code.device_status() == cbp.STATUS_NONFINITE_LLR


def test_frame_parallel_kernel_on_the_26112_code(large, monkeypatch):
    # a large lifting through the frame-parallel kernel: each thread walks all 384 lanes of
    # every base row; a batch of 40 frames leaves most of the launch's slots idle
    qc, code, oc = large
    monkeypatch.setenv("CBP_PLAN_FP", "1")
    assert code.launch_info(40)["frame_parallel"] == 1
    llr, _ = I.make_frames_torch(qc, 40, 1.0, seed=2300)
    ref = oc.decode(llr.cpu().numpy(), alg="cbp_sp", max_iter=12, threads=THREADS)
    assert_parity(run_gpu(code, llr.cpu().numpy(), "cbp_sp", max_iter=12), ref, "26112 fp")
    monkeypatch.setenv("CBP_PLAN_FP", "0")
    assert code.launch_info(40)["frame_parallel"] == 0


def test_frame_parallel_host_decode_and_status(monkeypatch):
    # the host-buffer entry point and the non-finite-LLR status through the same kernel
    qc = I.relift(I.code_576(), 4)
    code = cbp.Code.from_qc(qc)
    monkeypatch.setenv("CBP_PLAN_FP", "1")
    fr = I.make_frames(qc, 700, 2.0, seed=4800)
    host = torch.from_numpy(fr.llr).pin_memory()
    h_ref, i_ref, _ = code.decode(host.cuda(), max_iter=20)
    h, i = code.decode_host(host, max_iter=20, chunk=256)
    assert torch.equal(i, i_ref.cpu()) and torch.equal(h, h_ref.cpu())
    code.device_status()
    bad = fr.llr.copy()
    bad[5, 7] = np.nan
    code.decode(torch.from_numpy(bad).cuda(), max_iter=5)
    torch.cuda.synchronize()
    assert code.device_status() == cbp.STATUS_NONFINITE_LLR


def special_llrs(rng, B, N, ebn0_llr, cw):
    """Channel LLRs with the values that exercise the edges of the arithmetic: +0 and -0,
    subnormals, values just inside and outside the phi clamp (X_LO, 2 where phi changes
    regime, 30), large finite magnitudes up to the largest float, mixed into ordinary
    LLRs so that the frames still decode."""
    x = ebn0_llr.copy()
    xlo = np.float32(O.xlo32())
    specials = np.array([0.0, -0.0, 1e-40, -1e-40, 1e-20, -1e-20, xlo, -xlo,
                         np.nextafter(xlo, np.float32(0)), 2.0, -2.0,
                         np.nextafter(np.float32(2.0), np.float32(0)), 30.0, -30.0,
                         np.nextafter(np.float32(30.0), np.float32(100)), 1e6, -1e6,
                         3.0e38, -3.0e38, np.finfo(np.float32).max, -np.finfo(np.float32).max],
                        np.float32)
    for b in range(B):
        pos = rng.choice(N, size=N // 8, replace=False)
        v = rng.choice(specials, size=pos.size)
        if b % 2 == 0:  # even frames: each value takes the sign of its transmitted bit
            # (BPSK: bit 1 is negative), so they still decode; odd frames keep random signs
            v = np.where(cw[b, pos] != 0, -np.abs(v), np.abs(v)).astype(np.float32)
        x[b, pos] = v
    x[0, :] = 0.0          # a frame of erasures: every message starts from a zero
    x[1, :] = -0.0
    return x


@pytest.mark.parametrize("alg", ALGS)
def test_special_llr_values(code576, large, alg):
    """Frames full of signed zeros, subnormals, clamp-boundary and huge finite LLRs: every
    decoder bit for bit against the oracle (hard decisions, iteration counts, soft
    outputs), on the lane-parallel kernels of the 576- and 26112-bit codes."""
    rng = np.random.default_rng(77)
    qc, code, oc = code576
    fr = I.make_frames(qc, 64, 2.0, seed=7700)
    x = special_llrs(rng, 64, qc.N, fr.llr, fr.codewords)
    ref = oc.decode(x, alg=alg, max_iter=30, threads=THREADS)
    assert_parity(run_gpu(code, x, alg), ref, f"{alg} special 576")
    qc, code, oc = large
    llr, cw = I.make_frames_torch(qc, 24, 2.5, seed=7701)
    x = special_llrs(rng, 24, qc.N, llr.cpu().numpy(), cw.cpu().numpy())
    ref = oc.decode(x, alg=alg, max_iter=20, threads=THREADS)
    assert_parity(run_gpu(code, x, alg, max_iter=20), ref, f"{alg} special 26112")


@pytest.mark.parametrize("alg", ALGS)
def test_special_llr_values_wavefront(alg):
    """The same frames through the wavefront-schedule kernels (the planner's choice for
    the Z = 1 PEG code)."""
    rng = np.random.default_rng(78)
    qc = I.code_peg_2048()
    code = cbp.Code.from_qc(qc)
    assert code.launch_info(64, alg=alg)["level_schedule"] == 1
    fr = I.make_frames(qc, 64, 2.0, seed=7800)
    x = special_llrs(rng, 64, qc.N, fr.llr, fr.codewords)
    ref = O.OracleCode(qc.base, qc.Z).decode(x, alg=alg, max_iter=20, threads=THREADS)
    assert_parity(run_gpu(code, x, alg, max_iter=20), ref, f"{alg} special peg")


@pytest.mark.parametrize("alg", ["cbp_nms", "lbp_nms", "fbp_sp"])
@pytest.mark.parametrize("pos", [0, 11])
def test_comparators_with_weight1_column_not_last(pos, alg):
    # The min-sum and flooding kernels take a weight-1 edge anywhere in its row (CBP
    # min-sum reads its slots from the per-entry lane records): the permuted code of the
    # test above, bit for bit against the oracle.
    base = I.code_576().base
    w1 = int(np.nonzero((base >= 0).sum(0) == 1)[0][0])
    perm = [c for c in range(base.shape[1]) if c != w1]
    perm.insert(pos, w1)
    qc = I.QCCode(np.ascontiguousarray(base[:, perm]), 24)
    code = cbp.Code.from_qc(qc)
    fr = I.make_frames(qc, 300, 2.0, seed=4400 + pos)
    ref = O.OracleCode(qc.base, qc.Z).decode(fr.llr, alg=alg, max_iter=25, threads=THREADS)
    assert (ref["iters"] > 1).any()
    assert_parity(run_gpu(code, fr.llr, alg, max_iter=25), ref, f"{alg}, weight-1 column at {pos}")
