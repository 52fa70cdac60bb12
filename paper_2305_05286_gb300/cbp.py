"""Thin Python binding of libcbp (include/cbp.h): argument marshalling only.

Every decoding step runs in the CUDA kernels of libcbp.so; this module passes
torch device pointers and the current stream through ctypes.  There is no CPU
fallback: without the built library, or without a CUDA device, calls raise.

    from paper_2305_05286_gb300 import cbp, inputs
    code = cbp.Code.from_qc(inputs.code_576())
    hard, iters, soft = code.decode(llr_cuda, max_iter=30, alg="cbp_sp", soft=True)
"""
from __future__ import annotations

import ctypes as C
import threading

import torch

from . import build as _build

ALGS = {"cbp_sp": 0, "cbp_nms": 1, "lbp_nms": 2, "fbp_sp": 3}
STOPS = {"syndrome": 0, "none": 1, "window": 2}
STATUS = {0: "CBP_OK", -1: "CBP_EINVAL", -2: "CBP_ENOMEM", -3: "CBP_ECUDA",
          -4: "CBP_EUNSUPPORTED", -5: "CBP_EWORKSPACE", -6: "CBP_EDEVICE"}

# Every symbol include/cbp.h declares (checked by the ABI test).
EXPORTS = ("cbp_code_create", "cbp_code_destroy", "cbp_code_info", "cbp_workspace_bytes",
           "cbp_launch_info", "cbp_decode", "cbp_decode_ex", "cbp_host_buffer_bytes",
           "cbp_decode_host", "cbp_grad_workspace_bytes",
           "cbp_decode_weighted", "cbp_decode_grad", "cbp_decode_noalloc",
           "cbp_multi_workspace_bytes", "cbp_multi_launch_info", "cbp_decode_multi", "cbp_phi",
           "cbp_phi_deriv",
           "cbp_edge_ceiling", "cbp_device_status", "cbp_strerror")
STATUS_NONFINITE_LLR = 1
MULTI_MAX_ITEMS = 8


class CbpError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        msg = lib().cbp_strerror(status).decode()
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} ({msg})")


class _Opts(C.Structure):
    _fields_ = [("alg", C.c_int), ("alpha", C.c_float), ("stop_mode", C.c_int),
                ("soft_out", C.c_void_p)]


class _MultiItem(C.Structure):
    _fields_ = [("code", C.c_void_p), ("llr", C.c_void_p), ("hard_out", C.c_void_p),
                ("iters_out", C.c_void_p), ("batch", C.c_int)]


class _MultiOpts(C.Structure):
    _fields_ = [("frames_per_group", C.c_int), ("chk_shared", C.c_int), ("threads", C.c_int),
                ("ctas_per_sm", C.c_int), ("rounds_per_chunk", C.c_int), ("stop_mode", C.c_int),
                ("tail_percent", C.c_int)]


_lock = threading.Lock()
_lib = None


def lib(build_if_needed: bool = True):
    """Load libcbp.so from the package's _build directory (building it if stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            L = C.CDLL(path)
            P, I, Z = C.c_void_p, C.c_int, C.c_size_t
            L.cbp_code_create.restype = I
            L.cbp_code_create.argtypes = [P, I, I, I, C.POINTER(C.c_void_p)]
            L.cbp_code_destroy.restype = None
            L.cbp_code_destroy.argtypes = [P]
            L.cbp_code_info.restype = I
            L.cbp_code_info.argtypes = [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]
            L.cbp_workspace_bytes.restype = I
            L.cbp_workspace_bytes.argtypes = [P, I, C.POINTER(_Opts), C.POINTER(Z)]
            L.cbp_launch_info.restype = I
            L.cbp_launch_info.argtypes = [P, I, C.POINTER(_Opts), C.POINTER(I)]
            L.cbp_decode.restype = I
            L.cbp_decode.argtypes = [P, P, P, P, I, I, P, Z, P]
            L.cbp_decode_ex.restype = I
            L.cbp_decode_ex.argtypes = [P, P, P, P, I, I, P, Z, P, C.POINTER(_Opts)]
            L.cbp_host_buffer_bytes.restype = I
            L.cbp_host_buffer_bytes.argtypes = [P, I, C.POINTER(_Opts), C.POINTER(Z)]
            L.cbp_decode_host.restype = I
            L.cbp_decode_host.argtypes = [P, P, P, P, I, I, I, P, Z, P, C.POINTER(_Opts)]
            L.cbp_grad_workspace_bytes.restype = I
            L.cbp_grad_workspace_bytes.argtypes = [P, I, I, I, C.POINTER(Z)]
            L.cbp_decode_weighted.restype = I
            L.cbp_decode_weighted.argtypes = [P, P, P, I, I, I, P, P, Z, P]
            L.cbp_decode_grad.restype = I
            L.cbp_decode_grad.argtypes = [P, P, P, I, I, I, P, P, P, P, Z, P]
            L.cbp_decode_noalloc.restype = I
            L.cbp_decode_noalloc.argtypes = [P, P, P, P, I, I, P]
            MI, MO = C.POINTER(_MultiItem), C.POINTER(_MultiOpts)
            L.cbp_multi_workspace_bytes.restype = I
            L.cbp_multi_workspace_bytes.argtypes = [MI, I, MO, C.POINTER(Z)]
            L.cbp_multi_launch_info.restype = I
            L.cbp_multi_launch_info.argtypes = [MI, I, MO, C.POINTER(I)]
            L.cbp_decode_multi.restype = I
            L.cbp_decode_multi.argtypes = [MI, I, I, P, Z, P, MO]
            L.cbp_phi.restype = I
            L.cbp_phi.argtypes = [P, P, C.c_int64, P]
            L.cbp_phi_deriv.restype = I
            L.cbp_phi_deriv.argtypes = [P, P, C.c_int64, P]
            L.cbp_device_status.restype = I
            L.cbp_device_status.argtypes = [P, P, C.POINTER(C.c_uint32)]
            L.cbp_edge_ceiling.restype = I
            L.cbp_edge_ceiling.argtypes = [I, I, P, Z, P, C.POINTER(C.c_int64), C.POINTER(I)]
            L.cbp_strerror.restype = C.c_char_p
            L.cbp_strerror.argtypes = [I]
            _lib = L
    return _lib


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check(fn: str, rc: int):
    if rc != 0:
        raise CbpError(fn, rc)


def _opts(alg: str, alpha: float, stop: str, soft_ptr: int | None) -> _Opts:
    return _Opts(ALGS[alg], float(alpha), STOPS[stop], soft_ptr or None)


class Code:
    """A QC-LDPC code on the current CUDA device (cbp_code_create)."""

    def __init__(self, base, Z: int):
        import numpy as np

        b = np.ascontiguousarray(np.asarray(base, dtype=np.int32))
        if b.ndim != 2:
            raise ValueError("base matrix must be 2-D")
        self.base = b
        self.Z = int(Z)
        self.device = torch.cuda.current_device()
        h = C.c_void_p()
        _check("cbp_code_create",
               lib().cbp_code_create(b.ctypes.data, b.shape[0], b.shape[1], self.Z, C.byref(h)))
        self._h = h
        n, m, k, e = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check("cbp_code_info",
               lib().cbp_code_info(h, C.byref(n), C.byref(m), C.byref(k), C.byref(e)))
        self.N, self.M, self.K, self.E = n.value, m.value, k.value, e.value
        self.words = (self.N + 31) // 32
        self._ws = None

    @classmethod
    def from_qc(cls, qc) -> "Code":
        return cls(qc.base, qc.Z)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.cbp_code_destroy(h)
            self._h = None

    def device_status(self, stream=None) -> int:
        """Read and clear the handle's device status word (cbp_device_status)."""
        v = C.c_uint32()
        _check("cbp_device_status",
               lib().cbp_device_status(self._h, _stream_ptr(stream), C.byref(v)))
        return v.value

    # ------------------------------------------------------------------ workspace
    def workspace_bytes(self, batch: int, alg: str = "cbp_sp", stop: str = "syndrome") -> int:
        nb = C.c_size_t()
        o = _opts(alg, 0.75, stop, None)
        _check("cbp_workspace_bytes",
               lib().cbp_workspace_bytes(self._h, int(batch), C.byref(o), C.byref(nb)))
        return nb.value

    def workspace(self, batch: int, alg: str = "cbp_sp", stop: str = "syndrome") -> torch.Tensor:
        """A cached device workspace big enough for (batch, alg, stop)."""
        need = self.workspace_bytes(batch, alg, stop)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    def launch_info(self, batch: int, alg: str = "cbp_sp", stop: str = "syndrome") -> dict:
        """The launch plan cbp_decode_ex would use (cbp_launch_info)."""
        info = (C.c_int * 12)()
        o = _opts(alg, 0.75, stop, None)
        _check("cbp_launch_info", lib().cbp_launch_info(self._h, int(batch), C.byref(o), info))
        keys = ("frames_per_sm", "threads_per_cta", "ctas_per_sm", "lane_groups_per_cta",
                "frames_per_lane_group", "check_state_shared", "ctas", "team_lane_groups",
                "shared_bytes", "weight1_last", "frame_parallel", "level_schedule")
        return dict(zip(keys, list(info)))

    # ------------------------------------------------------------------ decode
    def decode_into(self, llr: torch.Tensor, hard: torch.Tensor, iters: torch.Tensor,
                    max_iter: int = 30, alg: str = "cbp_sp", alpha: float = 0.75,
                    stop: str = "syndrome", soft: torch.Tensor | None = None,
                    workspace: torch.Tensor | None = None, stream=None) -> None:
        """cbp_decode_ex on caller-provided device tensors (no allocation)."""
        B = llr.shape[0]
        if llr.dtype != torch.float32 or not llr.is_cuda or not llr.is_contiguous():
            raise ValueError("llr must be a contiguous float32 CUDA tensor")
        if llr.numel() != B * self.N:
            raise ValueError(f"llr must have {self.N} values per frame")
        if hard.numel() < B * self.words or iters.numel() < B:
            raise ValueError("output tensors too small")
        ws = workspace if workspace is not None else self.workspace(B, alg, stop)
        o = _opts(alg, alpha, stop, soft.data_ptr() if soft is not None else None)
        rc = lib().cbp_decode_ex(self._h, llr.data_ptr(), hard.data_ptr(), iters.data_ptr(),
                                 int(max_iter), int(B), ws.data_ptr(), ws.numel(),
                                 _stream_ptr(stream), C.byref(o))
        _check("cbp_decode_ex", rc)

    def decode(self, llr: torch.Tensor, max_iter: int = 30, alg: str = "cbp_sp",
               alpha: float = 0.75, stop: str = "syndrome", soft: bool = False, stream=None):
        """Decode [B, N] LLRs.  Returns (hard int32 [B, ceil(N/32)] bit words,
        iters int32 [B], soft float32 [B, N] or None).

        A CPU ``llr`` is copied to the device first and the results are copied back
        (the end-to-end path); a CUDA ``llr`` stays on the device.  With ``stream`` the
        decoding runs there, ordered after the current stream's work.  The code's cached
        workspace serves every call, so calls that may overlap on different streams should
        use ``decode_into`` with a workspace each."""
        host = not llr.is_cuda
        dev = torch.device(f"cuda:{self.device}")
        cur = torch.cuda.current_stream(dev)
        other = stream is not None and stream != cur  # copies on `cur`, decoding on `stream`
        x = llr.to(dev, non_blocking=True) if host else llr
        x = x.contiguous()
        B = x.shape[0]
        hard = torch.empty((B, self.words), dtype=torch.int32, device=dev)
        iters = torch.empty((B,), dtype=torch.int32, device=dev)
        sb = torch.empty((B, self.N), dtype=torch.float32, device=dev) if soft else None
        if other:
            stream.wait_stream(cur)
            for t in (x, hard, iters) + ((sb,) if sb is not None else ()):
                t.record_stream(stream)  # not reused by the allocator before `stream` is done
        self.decode_into(x, hard, iters, max_iter, alg, alpha, stop, sb, stream=stream)
        if host and other:
            cur.wait_stream(stream)
        if host:
            pin = llr.is_pinned()
            hard_h = torch.empty(hard.shape, dtype=hard.dtype, pin_memory=pin)
            iters_h = torch.empty(iters.shape, dtype=iters.dtype, pin_memory=pin)
            hard_h.copy_(hard, non_blocking=pin)
            iters_h.copy_(iters, non_blocking=pin)
            sb_h = sb.cpu() if sb is not None else None
            if pin:
                torch.cuda.current_stream(dev).synchronize()
            return hard_h, iters_h, sb_h
        return hard, iters, sb

    def decode_host(self, llr: torch.Tensor, max_iter: int = 30, alg: str = "cbp_sp",
                     alpha: float = 0.75, stop: str = "syndrome", chunk: int = 4096,
                     hard: torch.Tensor | None = None, iters: torch.Tensor | None = None,
                     stream=None, sync: bool = True):
        """Decode host LLRs [B, N] float32 with the copies overlapped with decoding
        (cbp_decode_host).  Page-locked ``llr`` (and outputs) let the copies overlap.  Returns
        host (hard int32 [B, ceil(N/32)], iters int32 [B]); with ``sync`` the call waits for
        the stream."""
        if llr.is_cuda or llr.dtype != torch.float32 or not llr.is_contiguous():
            raise ValueError("llr must be a contiguous float32 host tensor")
        B = llr.shape[0]
        if llr.numel() != B * self.N:
            raise ValueError(f"llr must have {self.N} values per frame")
        pin = llr.is_pinned()
        if hard is None:
            hard = torch.empty((B, self.words), dtype=torch.int32, pin_memory=pin)
        if iters is None:
            iters = torch.empty((B,), dtype=torch.int32, pin_memory=pin)
        if hard.is_cuda or iters.is_cuda or hard.numel() < B * self.words or iters.numel() < B:
            raise ValueError("hard/iters must be host tensors large enough for the batch")
        chunk = max(1, min(int(chunk), max(B, 1)))
        o = _opts(alg, alpha, stop, None)
        need = C.c_size_t()
        _check("cbp_host_buffer_bytes",
               lib().cbp_host_buffer_bytes(self._h, chunk, C.byref(o), C.byref(need)))
        buf = getattr(self, "_hbuf", None)
        if buf is None or buf.numel() < need.value:
            buf = torch.empty(max(need.value, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
            self._hbuf = buf
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check("cbp_decode_host",
               lib().cbp_decode_host(self._h, llr.data_ptr(), hard.data_ptr(), iters.data_ptr(),
                                     int(max_iter), int(B), chunk, buf.data_ptr(), buf.numel(),
                                     int(st.cuda_stream), C.byref(o)))
        if sync:
            st.synchronize()
        return hard, iters


def phi(x: torch.Tensor, stream=None) -> torch.Tensor:
    """The library's FP32 phi (Eq. s2e5) applied elementwise on the device (cbp_phi)."""
    if x.dtype != torch.float32 or not x.is_cuda:
        raise ValueError("x must be a float32 CUDA tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check("cbp_phi", lib().cbp_phi(x.data_ptr(), y.data_ptr(), x.numel(), _stream_ptr(stream)))
    return y


def phi_deriv(x: torch.Tensor, stream=None) -> torch.Tensor:
    """Derivative of the library's FP32 phi as evaluated (cbp_phi_deriv): the derivative of
    the cubic of each input's grid centre, 0 where the clamp holds."""
    if x.dtype != torch.float32 or not x.is_cuda:
        raise ValueError("x must be a float32 CUDA tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check("cbp_phi_deriv",
           lib().cbp_phi_deriv(x.data_ptr(), y.data_ptr(), x.numel(), _stream_ptr(stream)))
    return y


def edge_ceiling(iters: int = 4096, ctas: int = 0, stream=None) -> dict:
    """Time the CBP-SP edge-update ceiling kernel (cbp_edge_ceiling) with CUDA events:
    edge updates per second with every SM filled to its occupancy limit (ctas = 0)."""
    L = lib()
    st = stream if stream is not None else torch.cuda.current_stream()
    n, used = C.c_int64(), C.c_int()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    # 512-thread CTAs: at most 2048 / 512 = 4 per SM
    sink = torch.empty((ctas if ctas > 0 else 4 * sms) * 512, dtype=torch.float32, device="cuda")
    args = lambda it: (int(ctas), int(it), sink.data_ptr(), sink.numel(), int(st.cuda_stream),
                       C.byref(n), C.byref(used))
    _check("cbp_edge_ceiling", L.cbp_edge_ceiling(*args(16)))  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    _check("cbp_edge_ceiling", L.cbp_edge_ceiling(*args(iters)))
    e1.record(st)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    return {"edge_updates_per_s": n.value / secs, "ctas": used.value, "iters": int(iters),
            "seconds": secs}


def unpack_bits(words: torch.Tensor, N: int) -> torch.Tensor:
    """[B, ceil(N/32)] int32 bit words -> [B, N] uint8 hard decisions (bit v%32 of word v/32)."""
    w = words.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(32, device=w.device, dtype=torch.int64)
    b = (w[:, :, None] >> shifts) & 1
    return b.reshape(w.shape[0], w.shape[1] * 32)[:, :N].to(torch.uint8)


# ----------------------------------------------------------------------------- differentiable
class _WeightedCBP(torch.autograd.Function):
    """Weighted CBP as an autograd function: forward cbp_decode_weighted (checkpoints in a
    workspace kept on the context), backward cbp_decode_grad."""

    @staticmethod
    def forward(ctx, llr, weights, code, T, ckpt_every):
        if llr.dtype != torch.float32 or not llr.is_cuda or llr.dim() != 2 or llr.shape[1] != code.N:
            raise ValueError("llr must be a float32 CUDA tensor of shape [batch, N]")
        llr = llr.contiguous()
        w = weights.detach().contiguous().to(torch.float32)
        if w.numel() != int(T) * code.base.shape[0]:
            raise ValueError(f"weights must hold T x mb = {int(T) * code.base.shape[0]} values")
        B = llr.shape[0]
        need = C.c_size_t()
        _check("cbp_grad_workspace_bytes",
               lib().cbp_grad_workspace_bytes(code._h, B, int(T), int(ckpt_every), C.byref(need)))
        ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=llr.device)
        soft = torch.empty_like(llr)
        _check("cbp_decode_weighted",
               lib().cbp_decode_weighted(code._h, llr.data_ptr(), w.data_ptr(), int(T),
                                         int(ckpt_every), B, soft.data_ptr(), ws.data_ptr(),
                                         ws.numel(), _stream_ptr()))
        ctx.save_for_backward(llr, w)
        ctx.ws, ctx.code, ctx.T, ctx.ckpt = ws, code, int(T), int(ckpt_every)
        return soft

    @staticmethod
    def backward(ctx, grad_soft):
        if ctx.ws is None:
            raise RuntimeError("weighted_cbp: backward ran a second time; the checkpoints of the "
                               "forward pass are consumed by the first backward (run the "
                               "forward again instead of retain_graph=True)")
        llr, w = ctx.saved_tensors
        gs = grad_soft.contiguous().to(torch.float32)
        gw = torch.empty_like(w)
        gl = torch.empty_like(llr) if ctx.needs_input_grad[0] else None
        B = llr.shape[0]
        _check("cbp_decode_grad",
               lib().cbp_decode_grad(ctx.code._h, llr.data_ptr(), w.data_ptr(), ctx.T, ctx.ckpt,
                                     B, gs.data_ptr(), gw.data_ptr(),
                                     gl.data_ptr() if gl is not None else None,
                                     ctx.ws.data_ptr(), ctx.ws.numel(), _stream_ptr()))
        ctx.ws = None
        return gl, gw, None, None, None


def weighted_cbp(code: Code, llr: torch.Tensor, weights: torch.Tensor, T: int,
                 ckpt_every: int | None = None) -> torch.Tensor:
    """Differentiable weighted CBP: posterior LLRs [B, N] after T sweeps.

    ``weights`` [T, mb] scale the B2V messages per sweep and base row of the sending
    check (all ones = plain CBP with T sweeps).  Gradients flow to ``weights`` and
    ``llr`` through the library's adjoint kernel.  ``ckpt_every`` (default T): with T the
    forward records the backward's tape of every sweep (12 bytes per edge and sweep of
    workspace) and the backward recomputes nothing; a smaller value keeps a state
    checkpoint every ``ckpt_every`` sweeps instead and the backward recomputes each
    segment from it."""
    ck = int(T) if ckpt_every is None else int(ckpt_every)
    return _WeightedCBP.apply(llr, weights, code, int(T), ck)


# ----------------------------------------------------------------------------- several codes
def multi_opts(frames_per_group: int = 0, chk_shared: int = -1, threads: int = 0,
               ctas_per_sm: int = 0, rounds_per_chunk: int = 0,
               stop: str = "syndrome", tail_percent: int = 0) -> _MultiOpts:
    """Launch options of cbp_decode_multi (0 / -1 = the library's default; tail_percent
    -1 = no tail of one-round chunks)."""
    return _MultiOpts(int(frames_per_group), int(chk_shared), int(threads), int(ctas_per_sm),
                      int(rounds_per_chunk), STOPS[stop], int(tail_percent))


def _multi_items(codes, batches, llrs=None, hards=None, iters=None):
    if len(codes) != len(batches):
        raise ValueError("one batch size per code")
    if len(codes) > MULTI_MAX_ITEMS:
        raise ValueError(f"at most {MULTI_MAX_ITEMS} codes per launch")
    arr = (_MultiItem * max(1, len(codes)))()
    for i, (code, b) in enumerate(zip(codes, batches)):
        arr[i].code = code._h.value
        arr[i].batch = int(b)
        if llrs is not None:
            x, h, it = llrs[i], hards[i], iters[i]
            if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
                raise ValueError("llr tensors must be contiguous float32 CUDA tensors")
            if x.numel() != b * code.N or h.numel() < b * code.words or it.numel() < b:
                raise ValueError(f"item {i}: buffer sizes do not match the batch")
            arr[i].llr, arr[i].hard_out, arr[i].iters_out = (
                x.data_ptr(), h.data_ptr(), it.data_ptr())
    return arr


def multi_workspace_bytes(codes, batches, **opts) -> int:
    """Workspace bytes of one cbp_decode_multi launch (cbp_multi_workspace_bytes)."""
    nb = C.c_size_t()
    o = multi_opts(**opts)
    _check("cbp_multi_workspace_bytes",
           lib().cbp_multi_workspace_bytes(_multi_items(codes, batches), len(codes), C.byref(o),
                                           C.byref(nb)))
    return nb.value


def multi_launch_info(codes, batches, **opts) -> dict:
    """The launch cbp_decode_multi would use (cbp_multi_launch_info)."""
    info = (C.c_int * 8)()
    o = multi_opts(**opts)
    _check("cbp_multi_launch_info",
           lib().cbp_multi_launch_info(_multi_items(codes, batches), len(codes), C.byref(o), info))
    keys = ("ctas", "threads_per_cta", "shared_bytes", "ctas_per_sm", "chunks",
            "check_state_shared", "frames_per_lane_group", "weight1_last")
    return dict(zip(keys, list(info)))


def decode_multi_into(codes, llrs, hards, iters, max_iter: int = 30,
                      workspace: torch.Tensor | None = None, stream=None, **opts) -> None:
    """cbp_decode_multi on caller-provided device tensors: llrs[i] [B_i, N_i] float32,
    hards[i] [B_i, ceil(N_i/32)] int32, iters[i] [B_i] int32."""
    batches = [x.shape[0] for x in llrs]
    arr = _multi_items(codes, batches, llrs, hards, iters)
    o = multi_opts(**opts)
    if workspace is None:
        need = multi_workspace_bytes(codes, batches, **opts)
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=llrs[0].device)
    _check("cbp_decode_multi",
           lib().cbp_decode_multi(arr, len(codes), int(max_iter), workspace.data_ptr(),
                                  workspace.numel(), _stream_ptr(stream), C.byref(o)))


def decode_multi(codes, llrs, max_iter: int = 30, stream=None, **opts):
    """Decode several codes' frames in one launch.  Returns [(hard, iters)] per code."""
    hards = [torch.empty((x.shape[0], c.words), dtype=torch.int32, device=x.device)
             for c, x in zip(codes, llrs)]
    its = [torch.empty((x.shape[0],), dtype=torch.int32, device=x.device) for x in llrs]
    decode_multi_into(codes, [x.contiguous() for x in llrs], hards, its, max_iter,
                      stream=stream, **opts)
    return list(zip(hards, its))
