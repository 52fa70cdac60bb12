"""Throughput benchmark of CBP decoding on one GB300 (or N replicas under torchrun).

Workload: the 46x68 base graph lifted by Z=384 (N=26112, K=8448, rate 22/68),
65536 BPSK/AWGN frames per launch, at most 20 sweeps, syndrome stop.  One step is
one cbp_decode_ex launch over the whole batch with the LLRs resident in HBM
(6.85 GB per launch, far larger than L2).  Reported: decoded (information) Gbit/s,
FER/BER/iterations, the same-GPU comparators, an end-to-end number through host
buffers, an ALU roofline fraction, and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --sweep            # FER/BER/iterations/Gbit/s per Eb/N0 point
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CBP decoded Gbit/s at fixed FER vs same-GPU layered min-sum; % of roofline"
# Operating point: the Eb/N0 grid point (0.25 dB grid) at which layered normalized
# min-sum (alpha = 0.75) first reaches FER <= 1e-2 on this code (measured with --sweep at
# 65536 frames per point: FER 0.246 at 2.25 dB, 6.3e-4 at 2.5 dB).
EBN0_OPERATING = 2.5
# The Eb/N0 at which layered min-sum's FER is 1e-2 on this code, interpolated on log FER
# between the 0.05 dB grid points 2.40 dB (FER 1.43e-2) and 2.45 dB (3.6e-3) of
# `--sweep --sweep-lo 2.3 --sweep-hi 2.5 --sweep-step 0.05` (65536 frames per point).
# The default run also times CBP-SP and layered min-sum there: the comparison at exactly
# the fixed FER, where the 0.25 dB grid point above overshoots it twenty-fold.
EBN0_FER_1E2 = 2.41
FRAMES = 65536
MAX_ITER = 20

# Algorithmic operations per unit (the roofline numerator): only the arithmetic the
# algorithm itself needs, counted in FP32/INT32 lane operations -- no memory
# instructions, no lane indexing or addressing, no control flow.
#   phi evaluation: 20 (clamp 2, centre rounding 2, offset 1, k and offset above 2: 3,
#     regime test and selects 3, index 3, table fetch 2, Horner 3).
#   CBP-SP edge (Sec. IV-C Step 2; Tables I-II count E sums and E products per sweep):
#     2 phi + 8 simple operations (|S| - phi, the sign of R^new (2), Q* + R^new,
#     Lambda - R_old, S += phi, the sign fold, the first-visit select) = 48.
#   Posterior per variable (Eq. s4e20 read-only, then Eq. s2e7): phi + 4 (|S| - phi,
#     sign, add, compare) = 24.  Syndrome: 1 XOR per edge.
#   Min-sum (CBP and layered): about 10 compare/select/add operations per edge in place
#     of the two phi, 4 per variable.  Flooding BP: the CBP-SP edge count, 4 per variable.
OPS_EDGE = {"cbp_sp": 48, "cbp_nms": 10, "lbp_nms": 10, "fbp_sp": 48}
OPS_VAR = {"cbp_sp": 24, "cbp_nms": 4, "lbp_nms": 4, "fbp_sp": 4}
OPS_SYN = 1
# ncu counters of the current kernels, taken from one capture each (2432 frames of the
# 26112-bit code at 2.5 dB): DRAM bytes (read + write) and issued thread-instructions per
# frame-sweep or edge-sweep.  Each entry names the kernel instance and the capture date,
# and carries a hash of the kernel sources it was measured on: when the sources change,
# the numbers are stale and the bench line reports null instead.
CAPTURES = {
    "cbp_sp": {"kernel": "cbp_sp_kernel<0, 1, 3, 0, 768, 1>(KParams)", "date": "2026-12-04", "frames": 2432,
               "sources": "54fc0b0530641af9", "dram_bytes_per_frame_sweep": 1392182,
               "thread_inst_per_edge_sweep": 92.1, "issue_active": 0.523,
               "warps_active_per_sm": 23.9},
    "lbp_nms": {"kernel": "minsum_kernel<2, 0, 768, 0>(KParams)", "date": "2026-12-04", "frames": 2432,
               "sources": "11960eefc1b530b6", "dram_bytes_per_frame_sweep": 513578,
               "thread_inst_per_edge_sweep": 76.2, "issue_active": 0.631,
               "warps_active_per_sm": 22.3},
    "cbp_nms": {"kernel": "minsum_kernel<1, 0, 768, 0>(KParams)", "date": "2026-12-04", "frames": 2432,
               "sources": "11960eefc1b530b6", "dram_bytes_per_frame_sweep": 849329,
               "thread_inst_per_edge_sweep": 86.5, "issue_active": 0.576,
               "warps_active_per_sm": 21.7},
    "fbp_sp": {"kernel": "flood_kernel(KParams)", "date": "2026-12-04", "frames": 2432,
               "sources": "d4fcbc323157bf8c", "dram_bytes_per_frame_sweep": 789273,
               "thread_inst_per_edge_sweep": 109.7, "issue_active": 0.321,
               "warps_active_per_sm": 12.0},
}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling (every 200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_identity(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def timed_steps(torch, fn, steps, stream):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / steps  # ms per step


def frame_stats(torch, cbp, qc, hard, iters, cw):
    bits = cbp.unpack_bits(hard, qc.N)
    err = bits != cw
    fer = err.any(dim=1).float().mean().item()
    ber = err.float().mean().item()
    it = iters.abs().to(torch.float64)
    return {"fer": fer, "ber": ber, "mean_iters": it.mean().item(),
            "sweeps_total": int(it.sum().item()),
            "unconverged": int((iters < 0).sum().item())}


def alu_ops(alg, qc, sweeps_total):
    per_sweep = qc.E * (OPS_EDGE[alg] + OPS_SYN) + qc.N * OPS_VAR[alg]
    return per_sweep * sweeps_total


def kernel_source_hash(alg):
    """Hash of the kernel sources an algorithm's decoder is compiled from."""
    import hashlib

    names = ("cbp_minsum.cu" if "nms" in alg else "cbp_flood.cu" if alg == "fbp_sp"
             else "cbp_sp.cu", "cbp_kernel_common.cuh", "cbp_internal.cuh")
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2305_05286_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def capture_for(alg, code_name):
    """The ncu counters of this algorithm's kernel, if they were taken on these sources."""
    c = CAPTURES.get(alg)
    if c is None or code_name != "26112" or c["sources"] != kernel_source_hash(alg):
        return None
    return c


def roofline_entry(alg, qc, st, ms, peak_ops, code_name, traffic_arg):
    """ALU roofline of one decode: algorithmic operations per second against the issue-rate
    peak; the kernel's DRAM traffic and issued instructions from its ncu capture."""
    ops = alu_ops(alg, qc, st["sweeps_total"])
    achieved = ops / (ms / 1e3) / 1e12
    cap = capture_for(alg, code_name)
    traffic, src = traffic_arg, "--traffic"
    counters = None
    if traffic is None and cap is not None:
        traffic = cap["dram_bytes_per_frame_sweep"] * st["sweeps_total"]
        src = (f"ncu capture of {cap['kernel']} ({cap['date']}, {cap['frames']} frames), "
               "scaled by frame-sweeps")
    if traffic is None:
        src = "no capture of the current kernel sources"
    if cap is not None:
        counters = {k: cap[k] for k in ("kernel", "date", "thread_inst_per_edge_sweep",
                                        "issue_active", "warps_active_per_sm")}
    return {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "T lane-ops/s",
            "frac": achieved / peak_ops, "traffic": traffic, "traffic_source": src,
            "units": {"edge_sweeps": qc.E * st["sweeps_total"],
                      "var_sweeps": qc.N * st["sweeps_total"],
                      "ops_per_edge": OPS_EDGE[alg] + OPS_SYN, "ops_per_var": OPS_VAR[alg]},
            "kernel_counters": counters}


def cpu_oracle_rate(qc, llr_host, seconds=12.0, chunk=64):
    """Time the CPU oracle (all host cores) on consecutive frames until `seconds` pass."""
    from oracle import oracle as orc

    oc = orc.OracleCode(qc.base, qc.Z)
    cores = os.cpu_count() or 1
    done, t0 = 0, time.perf_counter()
    while True:
        sub = llr_host[done:done + chunk]
        if sub.shape[0] == 0:
            break
        oc.decode(sub, alg="cbp_sp", max_iter=MAX_ITER, soft=False, threads=cores)
        done += sub.shape[0]
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    K = (qc.nb - qc.mb) * qc.Z
    return {"value": K * done / dt / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
            "sample": f"first {done} frames of the same batch, FP32 oracle, CBP-SP, "
                      f"{cores} threads, {dt:.1f} s"}


# ----------------------------------------------------------------------------
def run_reference(args, rank):
    """The CPU oracle as it stands, on the host cores, same config and metric."""
    if rank != 0:
        return
    from paper_2305_05286_gb300 import inputs as I
    from oracle import oracle as orc

    qc = I.code_26112()
    K = (qc.nb - qc.mb) * qc.Z
    per_step = args.ref_frames
    fr = I.make_frames(qc, per_step * (args.steps + args.warmup), args.ebn0, seed=9000,
                       encoder="tri")
    oc = orc.OracleCode(qc.base, qc.Z)
    cores = os.cpu_count() or 1
    times = []
    for s in range(args.warmup + args.steps):
        sub = fr.llr[s * per_step:(s + 1) * per_step]
        t0 = time.perf_counter()
        oc.decode(sub, alg="cbp_sp", max_iter=MAX_ITER, soft=False, threads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = K * per_step / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "impl": "reference",
        "config": workload_config(args, qc, note=f"{per_step} frames per step on the host cores"),
        "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} frames per step, FP32 oracle CBP-SP, {cores} threads"},
        "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --code: the decoded code (the throughput workload is the 26112-bit one)
CODES = {"26112": ("code_26112", "QC-LDPC 46x68 base, Z=384"),
         "2304": ("code_2304", "QC-LDPC 12x24 base, Z=96"),
         "576": ("code_576", "QC-LDPC 12x24 base, Z=24"),
         "peg2048": ("code_peg_2048", "regular (3,6) PEG code, Z=1"),
         "pegirr2048": ("code_peg_irregular_2048", "irregular rate-1/2 PEG code, Z=1")}


def bench_code(I, name):
    return getattr(I, CODES[name][0])()


def workload_config(args, qc, note=None):
    gb = 4.0 * qc.N * args.frames / 1e9
    c = {"workload": f"{CODES[getattr(args, 'code', '26112')][1]} (N={qc.N}, "
                     f"K={(qc.nb - qc.mb) * qc.Z}), "
                     f"{args.frames} BPSK/AWGN frames per launch at Eb/N0 {args.ebn0} dB, "
                     f"max {MAX_ITER} sweeps, syndrome stop",
         "alg": args.alg, "frames_per_launch": args.frames, "ebn0_db": args.ebn0,
         "max_iter": MAX_ITER, "parallelism": "replicas" if args.gpus > 1 else "single",
         "l2": (f"inputs larger than L2 (LLRs 4*N bytes per frame, {gb:.2f} GB per launch)"
                if gb > 0.129 else f"LLRs {gb * 1e3:.0f} MB per launch, within L2 "
                                   "(each step decodes the same frames)")}
    if note:
        c["note"] = note
    return c


def max_over_ranks(dist, ms: float) -> float:
    """The slowest rank's time (the whole job waits for it); ms itself on one rank."""
    if not dist:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def frame_seed(rank: int) -> int:
    """Each replica decodes its own frames."""
    return 2000 + 97 * rank


def run_ours(args, rank, world, dist):
    import torch

    from paper_2305_05286_gb300 import cbp
    from paper_2305_05286_gb300 import inputs as I

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream(dev)
    qc = bench_code(I, args.code)
    K = (qc.nb - qc.mb) * qc.Z
    code = cbp.Code.from_qc(qc)
    B = args.frames
    llr, cw = I.make_frames_torch(qc, B, args.ebn0, seed=frame_seed(rank), device=dev,
                                  zero_codeword=not I.is_lower_triangular(qc))
    hard = torch.empty((B, code.words), dtype=torch.int32, device=dev)
    iters = torch.empty((B,), dtype=torch.int32, device=dev)
    ws = code.workspace(B, args.alg)

    def step(alg=args.alg):
        code.decode_into(llr, hard, iters, max_iter=MAX_ITER, alg=alg, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(gpu_identity(torch, local)) as clk:
        torch.cuda.synchronize()
        ms = timed_steps(torch, step, args.steps, stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(dist, ms)
    st = frame_stats(torch, cbp, qc, hard, iters, cw)
    iters_dev = iters.cpu()  # for the end-to-end run's check (comparators reuse `iters`)
    value = world * K * B / (ms / 1e3) / 1e9

    peaks = load_peaks()
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1455.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ops = sms * 128 * sm_mhz * 1e6 / 1e12  # T lane-ops/s at the sampled SM clock
    roofline = roofline_entry(args.alg, qc, st, ms, peak_ops, args.code, args.traffic)
    roofline["peak_source"] = f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (sampled SM clock)"
    hbm_bytes = B * (4 * qc.N + 4 * code.words + 4)
    roofline["hbm_algorithmic_GBs"] = hbm_bytes / (ms / 1e3) / 1e9
    roofline["hbm_peak_GBs"] = peaks.get("hbm_gbs")
    if args.alg == "cbp_sp":
        # measured compute ceiling: the CBP-SP edge update from registers, same phi
        ceil = cbp.edge_ceiling(iters=2048)
        rate = qc.E * st["sweeps_total"] / (ms / 1e3)
        roofline["edge_ceiling"] = {
            "ceiling_edge_updates_per_s": ceil["edge_updates_per_s"],
            "decoder_edge_updates_per_s": rate,
            "frac": rate / ceil["edge_updates_per_s"],
            "note": "cbp_edge_ceiling: 4 independent edge updates per thread, registers only, "
                    "phi table in shared memory, full occupancy"}

    comparators = {}
    if not args.no_comparators:
        # every comparator is timed like the headline decoder: the same warm-up and timed
        # steps on the same frames, with its own clock record
        for alg in ("cbp_nms", "lbp_nms", "fbp_sp"):
            if alg == args.alg:
                continue
            wsa = code.workspace(B, alg)
            f = lambda a=alg, w=wsa: code.decode_into(llr, hard, iters, max_iter=MAX_ITER,
                                                      alg=a, workspace=w)
            for _ in range(args.warmup):
                f()
            torch.cuda.synchronize()
            with ClockSampler(gpu_identity(torch, local)) as cclk:
                torch.cuda.synchronize()
                cms = timed_steps(torch, f, args.steps, stream)
                torch.cuda.synchronize()
            cs = frame_stats(torch, cbp, qc, hard, iters, cw)
            cro = roofline_entry(alg, qc, cs, cms, peak_ops, args.code, None)
            comparators[alg] = {"gbps": K * B / (cms / 1e3) / 1e9, "ms_per_step": cms,
                                "steps": args.steps, "warmup": args.warmup,
                                "fer": cs["fer"], "ber": cs["ber"], "mean_iters": cs["mean_iters"],
                                "alu_frac": cro["frac"], "kernel_counters": cro["kernel_counters"],
                                "clocks": cclk.summary(), "launch": code.launch_info(B, alg)}
            del wsa
        ws = code.workspace(B, args.alg)

    e2e = None
    if not args.no_e2e:
        host = torch.empty((B, qc.N), dtype=torch.float32, pin_memory=True)
        host.copy_(llr)
        hard_h = torch.empty((B, code.words), dtype=torch.int32, pin_memory=True)
        iters_h = torch.empty((B,), dtype=torch.int32, pin_memory=True)

        def e2e_step():  # cbp_decode_host: chunked H2D / decode / D2H, copies overlapped
            code.decode_host(host, max_iter=MAX_ITER, alg=args.alg, chunk=args.e2e_chunk,
                             hard=hard_h, iters=iters_h, sync=False)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ems = timed_steps(torch, e2e_step, args.steps, stream)
        ems = max_over_ranks(dist, ems)
        e2e = {"value": world * K * B / (ems / 1e3) / 1e9, "unit": "Gbit/s",
               "h2d_bytes_per_step": B * qc.N * 4,
               "d2h_bytes_per_step": B * code.words * 4 + B * 4, "ms_per_step": ems,
               "api": f"Code.decode_host (cbp_decode_host), chunks of {args.e2e_chunk} frames",
               "check_iters_equal_device_run": bool(torch.equal(iters_h, iters_dev))}
        del host, hard_h, iters_h

    at_fer = None
    if (not args.no_comparators and args.code == "26112" and args.alg == "cbp_sp"
            and args.ebn0 == EBN0_OPERATING):
        # the same two decoders, same steps and warm-up, at the Eb/N0 of layered min-sum's
        # FER 1e-2 (other frames of the same recipe)
        del ws
        llr2, cw2 = I.make_frames_torch(qc, B, EBN0_FER_1E2, seed=frame_seed(rank) + 1,
                                        device=dev, zero_codeword=not I.is_lower_triangular(qc))
        at_fer = {"ebn0_db": EBN0_FER_1E2}
        for alg in ("cbp_sp", "lbp_nms"):
            wsa = code.workspace(B, alg)
            f = lambda a=alg, w=wsa: code.decode_into(llr2, hard, iters, max_iter=MAX_ITER,
                                                      alg=a, workspace=w)
            for _ in range(args.warmup):
                f()
            torch.cuda.synchronize()
            with ClockSampler(gpu_identity(torch, local)) as cclk:
                torch.cuda.synchronize()
                cms = timed_steps(torch, f, args.steps, stream)
                torch.cuda.synchronize()
            cs = frame_stats(torch, cbp, qc, hard, iters, cw2)
            at_fer[alg] = {"gbps": world * K * B / (cms / 1e3) / 1e9, "ms_per_step": cms,
                           "fer": cs["fer"], "ber": cs["ber"], "mean_iters": cs["mean_iters"],
                           "clocks": cclk.summary()}
            del wsa
        at_fer["ratio"] = at_fer["cbp_sp"]["gbps"] / at_fer["lbp_nms"]["gbps"]
        del llr2, cw2

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = llr[: args.cpu_frames].cpu().numpy()
        cpu = cpu_oracle_rate(qc, sample, seconds=args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args, qc),
            "fer": st["fer"], "ber": st["ber"], "mean_iters": st["mean_iters"],
            "unconverged_frames": st["unconverged"],
            "coded_gbps": world * qc.N * B / (ms / 1e3) / 1e9,
            "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "comparators": comparators,
            "launch": code.launch_info(B, args.alg),
        }
        if "lbp_nms" in comparators:  # the metric's comparison at the fixed-FER point
            line["vs_layered_min_sum"] = {
                "ratio": value / (world * comparators["lbp_nms"]["gbps"]),
                "fer": st["fer"], "fer_layered_min_sum": comparators["lbp_nms"]["fer"],
                "mean_sweeps": st["mean_iters"],
                "mean_sweeps_layered_min_sum": comparators["lbp_nms"]["mean_iters"],
                "at_fer_1e-2": at_fer}
        print(json.dumps(line), flush=True)


def run_sweep(args):
    """FER, BER, mean sweeps and decoded Gbit/s per Eb/N0 point for each decoder, on the
    26112-bit code (65536 device frames per point by default, at most 20 sweeps) or on the
    576-bit code (2000 GF(2)-encoded frames per point, at most 30 sweeps).  Every point is
    timed over --sweep-steps launches after one warm-up, with its own clock record and ALU
    roofline fraction; one JSON line per (point, decoder)."""
    import torch

    from paper_2305_05286_gb300 import cbp
    from paper_2305_05286_gb300 import inputs as I

    qc = bench_code(I, args.code)
    K = (qc.nb - qc.mb) * qc.Z
    code = cbp.Code.from_qc(qc)
    small = qc.N <= 4096
    B = args.sweep_frames if args.sweep_frames else (2000 if small else FRAMES)
    max_iter = args.sweep_max_iter if args.sweep_max_iter else (30 if small else MAX_ITER)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    gid = gpu_identity(torch, 0)
    points = np.arange(args.sweep_lo, args.sweep_hi + 1e-9, args.sweep_step)
    for i, e in enumerate(points):
        if small:  # the parity workload's host frames (GF(2) encoder)
            fr = I.make_frames(qc, B, float(e), seed=1000 + int(round(float(e) * 10)))
            llr = torch.from_numpy(fr.llr).cuda()
            cw = torch.from_numpy(fr.codewords).cuda()
        else:
            llr, cw = I.make_frames_torch(qc, B, float(e), seed=2000 + i,
                                          zero_codeword=not I.is_lower_triangular(qc))
        hard = torch.empty((B, code.words), dtype=torch.int32, device="cuda")
        iters = torch.empty((B,), dtype=torch.int32, device="cuda")
        for alg in args.sweep_algs.split(","):
            ws = code.workspace(B, alg)
            f = lambda: code.decode_into(llr, hard, iters, max_iter=max_iter, alg=alg,
                                         alpha=args.alpha, workspace=ws)
            f()
            torch.cuda.synchronize()
            # enough launches for the clock sampler (one sample per 200 ms) to see the load
            first = timed_steps(torch, f, 1, stream)
            steps = max(args.sweep_steps, int(np.ceil(args.sweep_min_ms / max(first, 1e-3))))
            with ClockSampler(gid) as clk:
                ms = timed_steps(torch, f, steps, stream)
                torch.cuda.synchronize()
            st = frame_stats(torch, cbp, qc, hard, iters, cw)
            clocks = clk.summary()
            peak = sms * 128 * (clocks["sm_mhz"] or 2070.0) * 1e6 / 1e12
            ro = roofline_entry(alg, qc, st, ms, peak, args.code, None)
            row = {"code": f"{qc.mb}x{qc.nb} Z={qc.Z} (N={qc.N}, K={K})", "ebn0_db": round(float(e), 3),
                   "alg": alg, "alpha": args.alpha if "nms" in alg else None, "frames": B,
                   "max_iter": max_iter, "fer": st["fer"], "ber": st["ber"],
                   "mean_iters": st["mean_iters"], "gbps": K * B / (ms / 1e3) / 1e9,
                   "ms_per_launch": ms, "launches": steps,
                   "alu_frac": ro["frac"], "clocks": clocks}
            print(json.dumps(row), flush=True)
            del ws
        del llr, cw


def run_learned(args):
    """Learned-weight CBP on the 2304-bit code (12x24 base, Z=96, seed 4): train the
    T x mb B2V scales (init 1.0) with Adam on fresh frames at Eb/N0 ~ U[1, 3] dB, then
    compare FER and decoded Gbit/s against plain CBP and layered min-sum at T sweeps."""
    import torch

    from paper_2305_05286_gb300 import cbp
    from paper_2305_05286_gb300 import inputs as I

    qc = {"2304": I.code_2304, "2304hb": I.code_2304_hb}[args.learned_code]()
    zero = not I.is_lower_triangular(qc)  # all-zero codewords where the device encoder can't
    code = cbp.Code.from_qc(qc)
    K = (qc.nb - qc.mb) * qc.Z
    T, B = 10, args.train_frames
    w = torch.ones((T, qc.mb), device="cuda", requires_grad=True)
    opt = torch.optim.Adam([w], lr=args.lr)
    g = torch.Generator(device="cuda").manual_seed(5000)
    t0 = time.perf_counter()
    losses = []
    stream = torch.cuda.current_stream()
    step_ev = []  # CUDA events around the decoder's forward + loss and its backward
    for step in range(args.train_steps):
        ebn0 = 1.0 + 2.0 * torch.rand(B, generator=g, device="cuda")
        llr, cw = I.make_frames_torch(qc, B, ebn0, seed=5000 + step, zero_codeword=zero)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        # checkpoint spacing T: the forward records the tape, the backward recomputes nothing
        # --norm-weights: each sweep's scales divided by their mean, so training can
        # reweight the base rows of a sweep against each other but not inflate a sweep
        weff = w / w.mean(dim=1, keepdim=True) if args.norm_weights else w
        soft = cbp.weighted_cbp(code, llr, weff, T, T)
        if args.loss == "bce":
            loss = torch.nn.functional.binary_cross_entropy_with_logits(-soft, cw.float())
        elif args.loss == "soft_ber":  # mean sigmoid of the margin by which a bit is wrong
            loss = torch.sigmoid(soft * (2.0 * cw.float() - 1.0)).mean()
        else:  # soft frame-error rate: 1 - prod over the bits of sigmoid(-margin), per frame
            m = soft * (2.0 * cw.float() - 1.0)
            loss = (1.0 - torch.exp(-torch.nn.functional.softplus(m).sum(dim=1))).mean()
        opt.zero_grad(set_to_none=True)
        ev[1].record(stream)
        loss.backward()
        ev[2].record(stream)
        opt.step()
        if step >= 3:  # after 3 warm-up steps
            step_ev.append(ev)
        if step % 50 == 0 or step == args.train_steps - 1:
            losses.append((step, float(loss.item())))
            print(json.dumps({"train_step": step, "loss": losses[-1][1],
                              "elapsed_s": time.perf_counter() - t0}), flush=True)
    train_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    med = lambda xs: sorted(xs)[len(xs) // 2] if xs else None  # noqa: E731
    step_ms = {"forward_loss": med([a.elapsed_time(b) for a, b, _ in step_ev]),
               "backward": med([b.elapsed_time(c) for _, b, c in step_ev]),
               "steps_timed": len(step_ev)}
    wl = (w / w.mean(dim=1, keepdim=True) if args.norm_weights else w).detach().clone()
    ones = torch.ones_like(wl)
    rows = []
    chunk = min(args.eval_frames, 16384)
    for pi, e in enumerate((1.5, 2.0, 2.5)):
        stats = {k: [0, 0, 0.0] for k in ("learned", "cbp_T", "cbp_stop", "lbp_nms")}
        done = 0
        while done < args.eval_frames:
            n = min(chunk, args.eval_frames - done)
            llr, cw = I.make_frames_torch(qc, n, e, seed=6000 + 1000 * pi + done // chunk,
                                          zero_codeword=zero)
            for name in stats:
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                with torch.no_grad():
                    if name in ("learned", "cbp_T"):
                        soft = cbp.weighted_cbp(code, llr, wl if name == "learned" else ones, T, 5)
                        bits = (soft < 0).to(torch.uint8)
                    else:
                        hard, iters, _ = code.decode(llr, max_iter=T,
                                                     alg="cbp_sp" if name == "cbp_stop" else "lbp_nms")
                        bits = cbp.unpack_bits(hard, qc.N)
                ev1.record(stream)
                ev1.synchronize()
                st = stats[name]
                st[0] += int((bits != cw).any(dim=1).sum().item())
                st[1] += int((bits != cw).sum().item())
                st[2] += ev0.elapsed_time(ev1) / 1e3
            done += n
        for name, (fe, be, secs) in stats.items():
            row = {"ebn0_db": e, "decoder": name, "frames": done, "fer": fe / done,
                   "ber": be / (done * qc.N), "gbps": K * done / secs / 1e9,
                   "sweeps": T if name != "cbp_stop" and name != "lbp_nms" else f"<= {T}"}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"code": args.learned_code, "zero_codeword": zero,
                      "learned_weights": wl.cpu().numpy().round(4).tolist(),
                      "train_steps": args.train_steps, "train_frames": B, "loss": args.loss,
                      "norm_weights": bool(args.norm_weights),
                      "lr": args.lr,
                      "train_seconds": train_s, "train_step_ms_median": step_ms,
                      "loss_first_last": [losses[0], losses[-1]]}),
          flush=True)


def run_multi_bench(args):
    """Eight QC codes (Z 16..384, rates 1/3..8/9) with log-uniform frame counts in
    [64, 16384] and Eb/N0 ~ U[1, 4] dB per frame, decoded in one persistent launch
    (cbp_decode_multi) captured in a CUDA graph with autotuned launch options; against
    a graph of one cbp_decode_ex launch per code.  The LLRs (about 94 MB) fit in L2, so
    L2 is flushed (a 512 MB write) between timed replays and only the replays are timed."""
    import torch

    from paper_2305_05286_gb300 import cbp, tune
    from paper_2305_05286_gb300 import inputs as I

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    qcs = I.mixed_codes()
    codes = [cbp.Code.from_qc(q) for q in qcs]
    rng = np.random.default_rng(3)
    batches = [int(b) for b in np.exp(rng.uniform(np.log(64), np.log(16384), size=len(qcs)))]
    g = torch.Generator(device="cuda").manual_seed(3)
    llrs, cws = [], []
    for i, (q, b) in enumerate(zip(qcs, batches)):
        ebn0 = 1.0 + 3.0 * torch.rand(b, generator=g, device=dev)
        x, cw = I.make_frames_torch(q, b, ebn0, seed=3100 + i, device=dev)
        llrs.append(x.contiguous())
        cws.append(cw)
    Ks = [(q.nb - q.mb) * q.Z for q in qcs]
    info_bits = sum(k * b for k, b in zip(Ks, batches))
    hards = [torch.empty((b, c.words), dtype=torch.int32, device=dev) for c, b in zip(codes, batches)]
    its = [torch.empty((b,), dtype=torch.int32, device=dev) for b in batches]

    t0 = time.perf_counter()
    if args.no_tune:  # the library's default launch options (a fixed shape for profiling)
        best, table = {}, []
    else:
        best, table = tune.tune_multi(codes, llrs, MAX_ITER, reps=2)
    tune_s = time.perf_counter() - t0
    ws = torch.empty(max(cbp.multi_workspace_bytes(codes, batches, **best), 256),
                     dtype=torch.uint8, device=dev)
    wss = [c.workspace(b) for c, b in zip(codes, batches)]

    def multi():
        cbp.decode_multi_into(codes, llrs, hards, its, MAX_ITER, ws, **best)

    def per_code():
        for c, x, h, it, w in zip(codes, llrs, hards, its, wss):
            c.decode_into(x, h, it, max_iter=MAX_ITER, workspace=w)

    graphs = {}
    for name, fn in (("multi", multi), ("per_code", per_code)):
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(max(1, args.warmup)):
                fn()
        stream.wait_stream(side)
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            fn()
        graphs[name] = gr
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(gr, steps):
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gr.replay()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps

    for gr in graphs.values():
        for _ in range(args.warmup):
            gr.replay()
    torch.cuda.synchronize()
    with ClockSampler(gpu_identity(torch, 0)) as clk:
        ms_multi = timed(graphs["multi"], args.steps)
        ms_per = timed(graphs["per_code"], args.steps)
    graphs["multi"].replay()
    torch.cuda.synchronize()
    per = []
    sweeps = 0
    ops = 0
    for q, b, h, it, cw in zip(qcs, batches, hards, its, cws):
        st = frame_stats(torch, cbp, q, h, it, cw)
        sweeps += st["sweeps_total"]
        ops += alu_ops("cbp_sp", q, st["sweeps_total"])
        per.append({"code": f"{q.mb}x{q.nb} Z={q.Z}", "N": q.N, "frames": b, "fer": st["fer"],
                    "ber": st["ber"], "mean_iters": st["mean_iters"]})
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 1455.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * sm_mhz * 1e6 / 1e12
    line = {"metric": "mixed-code CBP decoded Gbit/s, one persistent launch (CUDA graph)",
            "value": info_bits / (ms_multi / 1e3) / 1e9, "unit": "Gbit/s",
            "ms_per_step": ms_multi, "steps": args.steps, "warmup": args.warmup,
            "per_code_launches": {"gbps": info_bits / (ms_per / 1e3) / 1e9, "ms_per_step": ms_per},
            "speedup_vs_per_code_launches": ms_per / ms_multi,
            "tuned_options": best, "tune_seconds": tune_s,
            "tune_table": [{"ms": ms, **o} for ms, o in table[:8]],
            "launch": cbp.multi_launch_info(codes, batches, **best),
            "roofline": {"bound": "alu", "achieved": ops / (ms_multi / 1e3) / 1e12, "peak": peak,
                         "unit": "T lane-ops/s",
                         "frac": ops / (ms_multi / 1e3) / 1e12 / peak},
            "codes": per, "info_bits_per_step": info_bits,
            "config": {"workload": "8 QC codes Z 16..384, rates 1/3..8/9, frames log-uniform "
                                   "[64, 16384] (seed 3), Eb/N0 ~ U[1, 4] dB per frame, "
                                   f"max {MAX_ITER} sweeps, syndrome stop",
                       "l2": "L2 flushed (512 MB write) before each timed replay"},
            "clocks": clocks, "dtype": "f32", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_nms_study(args):
    """CBP min-sum against CBP log-tanh: FER, BER and mean sweeps over an Eb/N0 grid on the
    576- and 2304-bit codes, CBP-NMS for several normalisations alpha, with layered NMS and
    flooding BP beside them (30 sweeps at most, syndrome stop)."""
    import torch

    from paper_2305_05286_gb300 import cbp
    from paper_2305_05286_gb300 import inputs as I

    alphas = [float(a) for a in args.alphas.split(",")]
    for name, qc in (("n576", I.code_576()), ("n2304", I.code_2304())):
        code = cbp.Code.from_qc(qc)
        B = args.study_frames
        for pi, e in enumerate(np.arange(args.sweep_lo, args.sweep_hi + 1e-9, 0.25)):
            llr, cw = I.make_frames_torch(qc, B, float(e), seed=7000 + 100 * pi + qc.Z)
            hard = torch.empty((B, code.words), dtype=torch.int32, device="cuda")
            iters = torch.empty((B,), dtype=torch.int32, device="cuda")
            runs = [("cbp_sp", 0.75), ("fbp_sp", 0.75), ("lbp_nms", 0.75)]
            runs += [("cbp_nms", a) for a in alphas]
            for alg, a in runs:
                code.decode_into(llr, hard, iters, max_iter=30, alg=alg, alpha=a,
                                 workspace=code.workspace(B, alg))
                s = frame_stats(torch, cbp, qc, hard, iters, cw)
                print(json.dumps({"code": name, "ebn0_db": round(float(e), 2), "alg": alg,
                                  "alpha": a if "nms" in alg else None, "frames": B,
                                  "fer": s["fer"], "ber": s["ber"],
                                  "mean_iters": s["mean_iters"]}), flush=True)
            del llr, cw


def run_paper_rerun(args):
    """The paper's own setting (Sec. V): rate-1/2 PEG codes of length 2048, regular (3,6)
    and irregular, BPSK/AWGN, at most 200 iterations.  FER, BER and mean sweeps of CBP
    (which equals layered BP bit for bit) with the syndrome stop and with the paper's
    window stop, CBP min-sum (alpha = 1) and flooding BP.  The codes are general sparse
    graphs, decoded as QC codes with Z = 1; frames are codewords of a GF(2) encoder."""
    import torch

    from paper_2305_05286_gb300 import cbp
    from paper_2305_05286_gb300 import inputs as I

    runs = [("cbp_sp", "syndrome"), ("cbp_sp", "window"), ("cbp_nms", "syndrome"),
            ("fbp_sp", "syndrome")]
    for name, qc in (("peg_3_6_n2048", I.code_peg_2048()),
                     ("peg_irr_n2048", I.code_peg_irregular_2048())):
        code = cbp.Code.from_qc(qc)
        for pi, e in enumerate(np.arange(args.sweep_lo, args.sweep_hi + 1e-9, 0.25)):
            fr = I.make_frames(qc, args.study_frames, float(e), seed=8000 + 10 * pi)
            llr = torch.from_numpy(fr.llr).cuda()
            cw = torch.from_numpy(fr.codewords).cuda()
            for alg, stop in runs:
                t0 = time.perf_counter()
                hard, iters, _ = code.decode(llr, max_iter=200, alg=alg, alpha=1.0, stop=stop)
                torch.cuda.synchronize()
                secs = time.perf_counter() - t0
                s = frame_stats(torch, cbp, qc, hard, iters, cw)
                ok = iters > 0
                print(json.dumps({
                    "code": name, "ebn0_db": round(float(e), 2), "alg": alg, "stop": stop,
                    "frames": args.study_frames, "fer": s["fer"], "ber": s["ber"],
                    "mean_iters": s["mean_iters"],
                    "mean_iters_stopped": float(iters[ok].abs().double().mean().item())
                    if ok.any() else None,
                    "stopped": float(ok.double().mean().item()), "seconds": secs}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alg", default="cbp_sp", choices=["cbp_sp", "cbp_nms", "lbp_nms", "fbp_sp"])
    ap.add_argument("--ebn0", type=float, default=EBN0_OPERATING)
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--sweep-frames", type=int, default=0,
                    help="frames per Eb/N0 point (0: 65536 for the 26112-bit code, 2000 for "
                         "the 576-bit code)")
    ap.add_argument("--sweep-step", type=float, default=0.25)
    ap.add_argument("--sweep-steps", type=int, default=3, help="timed launches per point")
    ap.add_argument("--sweep-min-ms", type=float, default=600.0,
                    help="at least this long a timed region per point (more launches)")
    ap.add_argument("--sweep-max-iter", type=int, default=0,
                    help="0: 20 sweeps for the 26112-bit code, 30 for the 576-bit code")
    ap.add_argument("--sweep-algs", default="cbp_sp,cbp_nms,lbp_nms,fbp_sp")
    ap.add_argument("--alpha", type=float, default=0.75,
                    help="min-sum normalisation for --sweep (the bench line uses 0.75)")
    ap.add_argument("--learned", action="store_true")
    ap.add_argument("--code", choices=sorted(CODES), default="26112",
                    help="decoded code of the throughput run (default: the 26112-bit workload)")
    ap.add_argument("--multi", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="--multi: skip the autotuner and use the library's default options")
    ap.add_argument("--nms-study", action="store_true")
    ap.add_argument("--paper-rerun", action="store_true")
    ap.add_argument("--study-frames", type=int, default=100000)
    ap.add_argument("--alphas", default="0.625,0.6875,0.75,0.8125,0.875,1.0")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--learned-code", default="2304", choices=["2304", "2304hb"])
    ap.add_argument("--train-frames", type=int, default=8192)
    ap.add_argument("--eval-frames", type=int, default=1_000_000)
    ap.add_argument("--lr", type=float, default=0.01)
    ap.add_argument("--loss", default="bce", choices=["bce", "soft_ber", "soft_fer"],
                    help="learned weights: mean BCE of the output LLRs, the mean sigmoid of "
                         "each bit's wrong-side margin (a smooth bit-error rate), or one minus "
                         "the product of the bits' sigmoid(-margin) per frame (a smooth "
                         "frame-error rate)")
    ap.add_argument("--norm-weights", action="store_true",
                    help="learned weights: each sweep's base-row scales normalised to mean 1")
    ap.add_argument("--sweep-lo", type=float, default=0.0)
    ap.add_argument("--sweep-hi", type=float, default=2.0)
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunk", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cpu-frames", type=int, default=4096)
    ap.add_argument("--ref-frames", type=int, default=64)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch from an ncu capture of the current kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td

        td.init_process_group("gloo")
        dist = td
    args.gpus = world if world > 1 else args.gpus
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.sweep:
        run_sweep(args)
    elif args.learned:
        run_learned(args)
    elif args.multi:
        run_multi_bench(args)
    elif args.nms_study:
        run_nms_study(args)
    elif args.paper_rerun:
        run_paper_rerun(args)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
