"""The library's FP32 phi (Eq. s2e5, phi(x) = -log tanh(x/2)) and its derivative on the GPU.

* phi: every FP32 input from the lower clamp fl32(phi(30)) to 30, and the clamped ranges
  on both sides, bit for bit against the oracle's phi.
* derivative (the adjoint of weighted CBP): against the derivative of the oracle's cubic
  of the same grid centre, computed here in FP64 from the oracle's coefficient table;
  against the closed form -1/sinh(x) within the cubic's truncation error; 0 where the
  clamp holds.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_05286_gb300 import cbp

pytestmark = pytest.mark.gpu
CHUNK = 1 << 25


def _all_inputs():
    lo = int(np.float32(O.xlo32()).view(np.uint32))
    hi = int(np.float32(30.0).view(np.uint32))
    return lo, hi


def test_phi_exhaustive_bitwise():
    lo, hi = _all_inputs()
    n = 0
    for a in range(lo, hi + 1, CHUNK):
        b = min(a + CHUNK, hi + 1)
        bits = torch.arange(a, b, dtype=torch.int64, device="cuda").to(torch.int32)
        x = bits.view(torch.float32)
        y = cbp.phi(x).view(torch.int32).cpu().numpy()
        ref = O.phi32(x.cpu().numpy()).view(np.int32)
        bad = np.flatnonzero(y != ref)
        assert bad.size == 0, f"{bad.size} mismatches, first at bits {a + bad[0]:#x}"
        n += b - a
    assert n == hi - lo + 1 > 3.8e8
    # the clamped ranges: below the lower clamp (down to +0) and above 30 (up to +inf)
    edge = np.concatenate([np.arange(0, 1 << 20, 7, dtype=np.uint32),
                           np.arange(lo - (1 << 20), lo, 3, dtype=np.uint32),
                           np.arange(hi, hi + (1 << 20), 5, dtype=np.uint32),
                           np.array([0x7f7fffff, 0x7f800000], dtype=np.uint32)])
    x = edge.view(np.float32)
    y = cbp.phi(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), O.phi32(x).view(np.uint32))


def _cubic_derivative(x):
    """d/dx of the oracle's cubic c0 + c1 t + c2 t^2 + c3 t^3, t = (x - m) / h, at the grid
    centre m nearest to x (32 per binade below 2, k/16 from 2 to 30), in FP64."""
    tab = O.phi_table().astype(np.float64)
    xlo = np.float32(O.xlo32())
    xc = np.minimum(np.maximum(x, xlo), np.float32(30.0))
    bits = xc.view(np.uint32)
    cb = (bits + np.uint32(0x20000)) & np.uint32(0xFFFC0000)
    lo_reg = xc < np.float32(2.0)
    i_lo = (cb >> np.uint32(18)).astype(np.int64) - 2688
    e = ((cb >> np.uint32(23)) & np.uint32(0xff)).astype(np.int64) - 127
    k = np.rint(xc.astype(np.float64) * 16.0)
    i = np.where(lo_reg, i_lo, 1409 + (k.astype(np.int64) - 32))
    m = np.where(lo_reg, cb.view(np.float32).astype(np.float64), k / 16.0)
    h = np.where(lo_reg, np.ldexp(1.0, e), 1.0 / 16.0)
    t = (xc.astype(np.float64) - m) / h
    c = tab[i]
    d = (c[:, 1] + t * (2.0 * c[:, 2] + 3.0 * c[:, 3] * t)) / h
    inside = (x >= xlo) & (x <= np.float32(30.0))
    return np.where(inside, d, 0.0)


def test_phi_derivative_against_the_cubic():
    lo, hi = _all_inputs()
    worst = 0.0
    for a in range(lo, hi + 1, CHUNK * 3):
        bits = np.arange(a, min(a + CHUNK * 3, hi + 1), 3, dtype=np.uint32)
        x = bits.view(np.float32)
        y = cbp.phi_deriv(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
        ref = _cubic_derivative(x)
        rel = np.abs(y - ref) / np.abs(ref)
        worst = max(worst, float(rel.max()))
        # and the cubic's derivative is the derivative of phi up to the truncation error
        true = -1.0 / np.sinh(x.astype(np.float64))
        assert (np.abs(y - true) <= 2e-5 * np.abs(true)).all()
    assert worst <= 1e-6, worst


def test_phi_derivative_is_zero_where_the_clamp_holds():
    lo, hi = _all_inputs()
    x = np.concatenate([np.array([0.0, 1e-30], np.float32),
                        np.arange(lo - 4096, lo, dtype=np.uint32).view(np.float32),
                        np.arange(hi + 1, hi + 4096, dtype=np.uint32).view(np.float32),
                        np.array([1e4, np.inf], np.float32)])
    y = cbp.phi_deriv(torch.from_numpy(x).cuda()).cpu().numpy()
    assert (y == 0.0).all()
    inner = np.array([np.float32(O.xlo32()), np.float32(30.0)], np.float32)
    yi = cbp.phi_deriv(torch.from_numpy(inner).cuda()).cpu().numpy()
    assert (yi < 0.0).all()
