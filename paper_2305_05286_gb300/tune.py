"""Launch autotuner for the several-codes decoder (cbp_decode_multi).

The library's default launch shape (one 768-thread CTA per SM, four frame rounds per
chunk, the last 20 % of each item's frames in one-round chunks) is a safe choice, not
always the fastest: small lifting sizes leave lanes idle, two interleaved frames per
lane group hide more latency, and the size of chunks and of the one-round tail trade
per-chunk overhead against idle SMs at the end of the launch.  `tune_multi` times each
candidate option set on the caller's own frames with CUDA events and returns the
fastest.  All
decoding runs in libcbp; this module only chooses among its launch options.
"""
from __future__ import annotations

import itertools

import torch

from . import cbp


def candidates(codes, fpts=(1, 2), chks=(1, 0), ctas=(1, 2), rounds=(1, 2, 4, 8),
               tails=(-1, 20, 50)):
    """Option sets worth timing: every combination whose CTA can hold each code's
    lifting size (threads >= Z) and that the library can plan.  The tail of one-round
    chunks only matters when chunks hold more than one round."""
    zmax = max(c.Z for c in codes)
    out = []
    for fpt, chk, cps, r, tail in itertools.product(fpts, chks, ctas, rounds, tails):
        tmax = 384 if fpt == 2 else 768
        threads = tmax // cps if cps > 1 and tmax // cps >= zmax else tmax
        if threads < zmax or (r == 1 and tail != tails[0]):
            continue
        out.append(dict(frames_per_group=fpt, chk_shared=chk, threads=threads,
                        ctas_per_sm=cps, rounds_per_chunk=r, tail_percent=tail))
    return out


def time_multi(codes, llrs, opts: dict, max_iter: int = 30, reps: int = 3,
               warmup: int = 1) -> float:
    """Mean milliseconds of one cbp_decode_multi launch with `opts` on these frames."""
    batches = [x.shape[0] for x in llrs]
    need = cbp.multi_workspace_bytes(codes, batches, **opts)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=llrs[0].device)
    hards = [torch.empty((b, c.words), dtype=torch.int32, device=ws.device)
             for c, b in zip(codes, batches)]
    its = [torch.empty((b,), dtype=torch.int32, device=ws.device) for b in batches]
    for _ in range(warmup):
        cbp.decode_multi_into(codes, llrs, hards, its, max_iter, ws, **opts)
    st = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(st)
    for _ in range(reps):
        cbp.decode_multi_into(codes, llrs, hards, its, max_iter, ws, **opts)
    t1.record(st)
    t1.synchronize()
    return t0.elapsed_time(t1) / reps


def tune_multi(codes, llrs, max_iter: int = 30, reps: int = 3, cands=None):
    """Time every candidate; returns (best options, [(ms, options)] sorted fastest first).
    Candidates the library rejects for these codes (CBP_EUNSUPPORTED) are skipped."""
    table = []
    for o in cands if cands is not None else candidates(codes):
        try:
            ms = time_multi(codes, llrs, o, max_iter, reps)
        except cbp.CbpError as e:
            if e.status == -4:
                continue
            raise
        table.append((ms, o))
    if not table:
        raise RuntimeError("no launch option set fits these codes")
    table.sort(key=lambda t: t[0])
    return table[0][1], table


# ----------------------------------------------------------------------------- cache
_CACHE: dict = {}


def cache_key(codes, batches) -> str:
    """(GPU, codes, batch sizes rounded up to powers of two): launches that share a key
    share their best options."""
    import hashlib

    h = hashlib.sha1()
    h.update(torch.cuda.get_device_name().encode())
    for c, b in zip(codes, batches):
        h.update(c.base.tobytes())
        h.update(f"{c.Z}:{1 << max(0, int(b) - 1).bit_length()};".encode())
    return h.hexdigest()


def tuned_options(codes, llrs, max_iter: int = 30, reps: int = 3, path: str | None = None):
    """tune_multi once per cache key; later calls with the same key return the stored
    options.  ``path`` (a JSON file) keeps the cache across processes."""
    import json
    import os

    key = cache_key(codes, [x.shape[0] for x in llrs])
    if path and not _CACHE and os.path.exists(path):
        with open(path) as f:
            _CACHE.update(json.load(f))
    if key not in _CACHE:
        best, _ = tune_multi(codes, llrs, max_iter, reps)
        _CACHE[key] = best
        if path:
            with open(path, "w") as f:
                json.dump(_CACHE, f, indent=1)
    return dict(_CACHE[key])
