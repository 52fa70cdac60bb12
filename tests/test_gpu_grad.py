"""Weighted (differentiable) CBP on the GPU against the FP64 oracle adjoint.

Forward: bit for bit equal to the FP32 oracle (same operations in the same order).
Backward: the adjoint kernel's dLoss/dw and dLoss/dL against the oracle's reverse-mode
adjoint (itself pinned by finite differences), relative to the largest component: 1e-3,
both with checkpoint segments that the backward recomputes and with one segment
(ckpt = T), whose tape the forward records.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_05286_gb300 import cbp
from paper_2305_05286_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def run_forward(code, llr, w, T, ckpt):
    x = torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()
    with torch.no_grad():
        s = cbp.weighted_cbp(code, x, wt, T, ckpt)
    return s.cpu().numpy()


def run_backward(code, llr, w, T, ckpt, gsoft):
    B = llr.shape[0]
    x = torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda().requires_grad_(True)
    wt = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda().requires_grad_(True)
    s = cbp.weighted_cbp(code, x, wt, T, ckpt)
    s.backward(torch.from_numpy(np.ascontiguousarray(gsoft, dtype=np.float32)).cuda())
    return wt.grad.cpu().numpy(), x.grad.cpu().numpy()


@pytest.fixture(scope="module", params=["z4", "576"])
def setup(request):
    qc = I.relift(I.code_576(), 4) if request.param == "z4" else I.code_576()
    return qc, cbp.Code.from_qc(qc), O.OracleCode(qc.base, qc.Z)


@pytest.mark.parametrize("T,ckpt", [(10, 2), (7, 3), (1, 1)])
def test_forward_bitwise(setup, T, ckpt):
    qc, code, oc = setup
    fr = I.make_frames(qc, 37, 1.5, seed=40 + T)
    w = (1.0 + 0.2 * np.random.default_rng(T).standard_normal((T, qc.mb))).astype(np.float32)
    got = run_forward(code, fr.llr, w, T, ckpt)
    ref = oc.weighted(fr.llr, w, T, precision=32)
    assert np.array_equal(got, ref)


def test_unit_weights_equal_cbp(setup):
    qc, code, oc = setup
    fr = I.make_frames(qc, 50, 2.0, seed=44)
    got = run_forward(code, fr.llr, np.ones((10, qc.mb), np.float32), 10, 2)
    hard, iters, soft = code.decode(torch.from_numpy(fr.llr).cuda(), max_iter=10, stop="none",
                                    soft=True)
    assert np.array_equal(got, soft.cpu().numpy())


@pytest.mark.parametrize("T,ckpt,ebn0", [(10, 2, 1.0), (4, 1, 0.5), (6, 4, 1.5), (8, 8, 1.0)])
def test_adjoint_matches_oracle(setup, T, ckpt, ebn0):
    qc, code, oc = setup
    fr = I.make_frames(qc, 9, ebn0, seed=60 + T)
    w = (1.0 + 0.1 * np.random.default_rng(2).standard_normal((T, qc.mb))).astype(np.float32)
    x = fr.codewords.astype(np.float64)
    soft = oc.weighted(fr.llr.astype(np.float64), w.astype(np.float64), T)
    z = -(1.0 - 2.0 * x) * soft
    gsoft = ((-(1.0 - 2.0 * x) / (1.0 + np.exp(-z))) / soft.size).astype(np.float32)
    gw, gl = run_backward(code, fr.llr, w, T, ckpt, gsoft)
    rw, rl = oc.weighted_grad(fr.llr.astype(np.float64), w.astype(np.float64), T,
                              gsoft.astype(np.float64))
    assert np.abs(gw - rw).max() <= 1e-3 * np.abs(rw).max()
    assert np.abs(gl - rl).max() <= 1e-3 * np.abs(rl).max()


def test_checkpoint_spacing_does_not_change_gradients():
    qc = I.code_576()
    code = cbp.Code.from_qc(qc)
    fr = I.make_frames(qc, 64, 1.25, seed=77)
    T = 10
    w = np.ones((T, qc.mb), np.float32)
    gsoft = np.random.default_rng(5).standard_normal(fr.llr.shape).astype(np.float32) * 1e-4
    grads = [run_backward(code, fr.llr, w, T, c, gsoft) for c in (1, 2, 5, 10)]
    for gw, gl in grads[1:]:
        assert np.abs(gw - grads[0][0]).max() <= 1e-5 * np.abs(grads[0][0]).max()
        assert np.abs(gl - grads[0][1]).max() <= 1e-5 * np.abs(grads[0][1]).max()


def test_training_step_on_the_4096_frame_batch():
    """The 576-bit code at T = 10, checkpoints every 2 sweeps, 4096 frames at Eb/N0
    uniform in [1, 3] dB: loss and gradients are finite and a small step against the
    gradient lowers the loss."""
    qc = I.code_576()
    code = cbp.Code.from_qc(qc)
    g = torch.Generator(device="cuda").manual_seed(3)
    ebn0 = 1.0 + 2.0 * torch.rand(4096, generator=g, device="cuda")
    llr, cw = I.make_frames_torch(qc, 4096, ebn0, seed=3)
    w = torch.ones((10, qc.mb), device="cuda", requires_grad=True)

    def loss_fn(w):
        s = cbp.weighted_cbp(code, llr, w, 10, 2)
        return torch.nn.functional.binary_cross_entropy_with_logits(-s, cw.float())

    loss = loss_fn(w)
    loss.backward()
    assert torch.isfinite(loss) and torch.isfinite(w.grad).all() and w.grad.abs().sum() > 0
    with torch.no_grad():
        w2 = w - 0.01 * w.grad / w.grad.abs().max()
    assert loss_fn(w2).item() < loss.item()
