"""cbp_decode_noalloc: decoding without any device allocation by the caller or the library.

Callers that cannot allocate device memory (a real-time loop, a plugin that does not own
the device's memory) use this entry point; its scratch is a fixed array inside libcbp.
Its results must equal cbp_decode's on the same inputs, call after call: the array is
shared by every call and keeps the previous call's contents.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2305_05286_gb300 import cbp
from paper_2305_05286_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _reference(code, x, max_iter):
    hard, iters, _ = code.decode(x, max_iter=max_iter, alg="cbp_sp")
    return hard, iters


def _noalloc(code, x, max_iter):
    B = x.shape[0]
    hard = torch.full((B, code.words), -1, dtype=torch.int32, device=x.device)
    iters = torch.zeros((B,), dtype=torch.int32, device=x.device)
    rc = cbp.lib().cbp_decode_noalloc(code._h, x.data_ptr(), hard.data_ptr(), iters.data_ptr(),
                                      max_iter, B, torch.cuda.current_stream().cuda_stream)
    assert rc == 0, cbp.lib().cbp_strerror(rc)
    return hard, iters


@pytest.mark.parametrize("qc_fn,frames,ebn0,max_iter", [
    (I.code_576, 3000, 2.0, 30),      # the whole batch fits the scratch at full occupancy
    (I.code_26112, 200, 2.5, 20),     # fewer frame slots than cbp_decode would use
])
def test_noalloc_matches_cbp_decode_twice(qc_fn, frames, ebn0, max_iter):
    qc = qc_fn()
    code = cbp.Code.from_qc(qc)
    for call in range(2):   # two calls in a row on different frames
        if qc.N <= 4096:
            fr = I.make_frames(qc, frames, ebn0 + 0.25 * call, seed=70 + call)
            x = torch.from_numpy(fr.llr).cuda()
        else:
            x, _ = I.make_frames_torch(qc, frames, ebn0 - 0.75 * call, seed=71 + call)
        h_ref, i_ref = _reference(code, x, max_iter)
        h, i = _noalloc(code, x, max_iter)
        torch.cuda.synchronize()
        assert torch.equal(i, i_ref), f"call {call}: iteration counts differ"
        assert torch.equal(h, h_ref), f"call {call}: hard decisions differ"


def test_noalloc_rejects_a_code_too_big_for_the_scratch():
    # 400 x 12 base rows of weight 12, Z = 1024: one frame slot needs ~21 MB > 16 MiB
    base = np.random.default_rng(3).integers(0, 1024, size=(400, 12)).astype(np.int32)
    code = cbp.Code(base, 1024)
    x = torch.zeros((1, code.N), dtype=torch.float32, device="cuda")
    hard = torch.zeros((1, code.words), dtype=torch.int32, device="cuda")
    iters = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    rc = cbp.lib().cbp_decode_noalloc(code._h, x.data_ptr(), hard.data_ptr(), iters.data_ptr(),
                                      5, 1, torch.cuda.current_stream().cuda_stream)
    assert rc == -5 and cbp.lib().cbp_strerror(rc) == b"workspace too small"
    torch.cuda.synchronize()
    assert iters.item() == 7   # nothing was launched


def test_noalloc_fewer_lane_groups_per_cta_than_cbp_decode():
    # Z = 256, 1000 base rows of degree 3 (two heavy columns, then one weight-1 column
    # per row): one frame slot needs about 6 MB of scratch, and cbp_decode runs 3 lane
    # groups per CTA, 18 MB together.  The no-alloc call drops to 2 groups per CTA (and a
    # single CTA) to fit its array, and must still decode exactly like cbp_decode.
    mb, Z = 1000, 256
    rng = np.random.default_rng(11)
    base = np.full((mb, 2 + mb), -1, dtype=np.int32)
    base[:, 0] = rng.integers(0, Z, size=mb)
    base[:, 1] = rng.integers(0, Z, size=mb)
    base[np.arange(mb), 2 + np.arange(mb)] = 0
    code = cbp.Code(base, Z)
    frames = 320
    li = code.launch_info(frames)
    # cbp_decode: 3 lane groups of one frame each per CTA, check beliefs in the workspace
    assert li["lane_groups_per_cta"] == 3 and li["frames_per_lane_group"] == 1
    assert li["check_state_shared"] == 0 and li["frame_parallel"] == 0
    g = torch.Generator(device="cuda").manual_seed(12)
    for call in range(2):
        x = 1.5 + 2.0 * torch.randn((frames, code.N), generator=g, device="cuda")
        h_ref, i_ref = _reference(code, x, 3)
        h, i = _noalloc(code, x, 3)
        torch.cuda.synchronize()
        assert torch.equal(i, i_ref), f"call {call}: iteration counts differ"
        assert torch.equal(h, h_ref), f"call {call}: hard decisions differ"
