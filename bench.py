#!/usr/bin/env python3
"""Benchmark: spin SHT transforms/s (forward + inverse) at L = 1024, s = 2, B = 64 fields.

One step = one inverse transform of B fields (coefficients -> the L x (2L-1) sphere grid) followed
by one forward transform of that grid (-> coefficients), through the C ABI of libssht on inputs
already resident in HBM (each field's coefficients are larger than nothing fits in L2: the batch
is 0.5 GB of coefficients and 1.1 GB of samples, so every step streams from HBM).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ssht|reference]

Under torchrun (N > 1) every rank transforms its own B fields (weak scaling, no collective on
the data path); the time is the maximum over ranks.  Rank 0 prints one JSON line.
``--impl reference`` times the CPU oracle (the plain FP64 implementation under oracle/) on the
host cores, one field of the same workload per step, on rank 0 only.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin SHT transforms/s (fwd+inv) at L=1024 s=2 B=64; rel err vs FP64 oracle"
DEFAULT_L, DEFAULT_S, DEFAULT_B = 1024, 2, 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ssht", choices=["ssht", "reference"])
    ap.add_argument("--L", type=int, default=DEFAULT_L)
    ap.add_argument("--s", type=int, default=DEFAULT_S)
    ap.add_argument("--batch", type=int, default=DEFAULT_B)
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--delta-mode", default="recompute", choices=["recompute", "cache"])
    ap.add_argument("--no-check", action="store_true", help="skip the oracle error check")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cache-line", action="store_true")
    ap.add_argument("--no-alt", action="store_true", help="skip the other split precision's line")
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven-batch (captured graph) line")
    ap.add_argument("--no-real", action="store_true", help="skip the real spin-0 fields line")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 transform line")
    ap.add_argument("--no-tune", action="store_true", help="default contraction shape instead of the tuned one")
    ap.add_argument("--error-sweep", action="store_true",
                    help="print errors vs the FP64 oracle for L = 32 .. 2048 and every precision, then exit")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# distributed helpers
# ---------------------------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank, B):
    """First field seed of a rank: rank r transforms fields r*B .. r*B+B-1 (field b of the rank
    draws from default_rng(r*B + b)), so the shards of the ranks are disjoint."""
    return rank * B


def throughput(world, B, steps, ms):
    """Whole-job transforms/s: the fields of all ranks over the slowest rank's time."""
    return world * B * steps / (ms / 1e3)


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device):
    if world > 1:
        import torch.distributed as dist
        dist.barrier(device_ids=[device.index] if device is not None and device.type == "cuda" else None)


# ---------------------------------------------------------------------------------------------
# GPU clocks during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, fl in rows for k, v in enumerate(fl) if v.lower() == "active"})
        sm = [r[0] for r in rows]
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------------------------

def device_units():
    """SM count of the current GPU (queried) and its maximum SM clock in Hz (nvidia-smi, else the
    figure recorded beside the measured peaks)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
        clk = float(out.strip().splitlines()[0]) * 1e6
    except Exception:
        clk = None
    if not clk:
        path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        clk = float(json.load(open(path)).get("sm_max_mhz", 2070.0)) * 1e6 if os.path.exists(path) else 2.07e9
    return sms, clk


def peaks(sms=152, clk=2.07e9):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, bf16, bf16s, src = 6800.0, 1900.0, 1700.0, "fallback"
    if os.path.exists(path):
        j = json.load(open(path))
        hbm, bf16, src = float(j.get("hbm_gbs", hbm)), float(j.get("bf16_tflops", bf16)), "measured"
        bf16s = float(j.get("bf16_tflops_sustained", bf16s))
    return {
        "hbm_gbs": (hbm, src + " copy bandwidth"),
        "bf16_tflops": (bf16, src + " (burst)"),
        "bf16_tflops_sustained": (bf16s, src + " (sustained)"),
        # Not in MEASURED_PEAKS.json: derived from unit counts and the maximum SM clock.
        "fp64_tflops": (sms * 2 * 2 * clk / 1e12, "derived: %d SMs x 2 DFMA/clk x 2 flop x %.2f GHz" % (sms, clk / 1e9)),
        "fp32_tflops": (sms * 128 * 2 * clk / 1e12, "derived: %d SMs x 128 FFMA/clk x 2 flop x %.2f GHz" % (sms, clk / 1e9)),
        "tf32_tflops": (bf16s / 2.0, src + " sustained bf16 x nominal tf32/bf16 ratio 1/2"),
    }


# An FP64 FMA-chain probe on this part (independent chains, all SMs) reached 1.19 TFLOP/s, 94.5 % of
# the derived FP64 figure; it is reported beside the derived peak.
FP64_PROBE_TFLOPS = 1.19


def contraction_macs(L, s):
    """Complex x real multiply-adds of one field and one direction: sum_{l>=|s|} (2l+1)(l+1)."""
    l = np.arange(abs(s), L, dtype=np.float64)
    return float(np.sum((2 * l + 1) * (l + 1)))


def recursion_updates(L):
    """Element updates of one octant Risbo sweep: (half-step, integer-step) updates, i.e. half
    slabs (l+1)(l+4)/2 and integer slabs (l+2)(l+3)/2 summed over l = 0 .. L-2."""
    l = np.arange(0, max(L - 1, 0), dtype=np.float64)
    return float(np.sum((l + 1) * (l + 4) / 2)), float(np.sum((l + 2) * (l + 3) / 2))


def column_updates(L):
    """Updates of one sweep of the column recursion: in degree l the lane of column m walks rows
    l .. 32 floor(m/32) and updates once per row below the first, l - 32 floor(m/32) times."""
    total = 0.0
    for l in range(L):
        m = np.arange(l + 1)
        total += float(np.sum(l - 32 * (m // 32)))
    return total


def lane_updates(L):
    """Updates of one sweep of the degree-lane recursion: in degree l the lane of column m walks
    rows l .. m, l - m updates."""
    l = np.arange(L, dtype=np.float64)
    return float(np.sum(l * (l + 1) / 2))


def quadrant_entries(L):
    """Entries Delta^l_{m'm}, 0 <= m, m' <= l < L (the table, or the A operand, of one sweep)."""
    l = np.arange(L, dtype=np.float64)
    return float(np.sum((l + 1) ** 2))


def torus_M(L):
    """FFT length of the torus passes' Bluestein DFTs of length N = 2L - 1."""
    M = 128
    while M < 2 * (2 * L - 1) - 1:
        M *= 2
    return M


def fft_flops(M):
    return 5.0 * M * np.log2(M)


KERNEL_SOURCES = {
    "column_tiles_kernel": ["paper_0807_4494_gb300/csrc/delta_column.cu", "paper_0807_4494_gb300/csrc/int_mul.h",
                            "paper_0807_4494_gb300/csrc/f32_round.h"],
    "column_recursion_kernel": ["paper_0807_4494_gb300/csrc/delta_column.cu", "paper_0807_4494_gb300/csrc/int_mul.h",
                                "paper_0807_4494_gb300/csrc/f32_round.h"],
    "lane_recursion_kernel": ["paper_0807_4494_gb300/csrc/delta_column.cu", "paper_0807_4494_gb300/csrc/int_mul.h",
                                "paper_0807_4494_gb300/csrc/f32_round.h"],
    "risbo_kernel": ["paper_0807_4494_gb300/csrc/delta.cu"],
    "tc_gemm_kernel<inverse>": ["paper_0807_4494_gb300/csrc/contract_tc.cu"],
    "tc_gemm_kernel<forward>": ["paper_0807_4494_gb300/csrc/contract_tc.cu"],
    "pack_v_kernel": ["paper_0807_4494_gb300/csrc/contract_tc.cu"],
    "inverse_theta_kernel": ["paper_0807_4494_gb300/csrc/torus_pass.cu"],
    "phi_kernel<+1>": ["paper_0807_4494_gb300/csrc/torus_pass.cu"],
    "phi_kernel<-1>": ["paper_0807_4494_gb300/csrc/torus_pass.cu"],
    "forward_theta_kernel": ["paper_0807_4494_gb300/csrc/torus_pass.cu"],
    "inverse_kernel (SIMT)": ["paper_0807_4494_gb300/csrc/contract_simt.cu"],
    "project_kernel (SIMT)": ["paper_0807_4494_gb300/csrc/contract_simt.cu"],
}


def split_trace(trace, steps):
    """Per-kernel live launch times (ms) from the stage trace of `steps` inverse + forward steps of
    one plan: the torus passes are the caller-stream FFT brackets in call order (inverse theta,
    inverse phi, forward phi, forward theta), the recursion the Delta brackets, the packing of the
    inverse's data operand the caller-stream pack brackets."""
    out = {}
    fft = [t1 - t0 for name, lane, t0, t1 in trace if name == "fft" and lane == 0]
    names = ["theta_inverse", "phi_inverse", "phi_forward", "theta_forward"]
    for k, d in enumerate(fft):
        out.setdefault(names[k % 4], []).append(d)
    rec_inv = [t1 - t0 for name, lane, t0, t1 in trace if name == "delta_inverse"]
    rec = [t1 - t0 for name, lane, t0, t1 in trace if name == "delta"]
    if rec_inv:  # 3xTF32 plans: the recursions writing the A tiles of each direction
        out["recursion_inverse"] = rec_inv
        if rec:
            out["recursion_forward"] = rec
    else:
        for k, d in enumerate(rec):  # one recursion per call: the inverse's, then the forward's
            out.setdefault("recursion_inverse" if k % 2 == 0 else "recursion_forward", []).append(d)
    for name, lane, t0, t1 in trace:
        key = {("inverse", 0): "contraction_inverse",
               ("project", 0): "contraction_forward", ("pack", 0): "pack_data", ("pack", 1): "pack_a",
               ("torus", 0): "torus_glue"}.get((name, lane))
        if key:
            out.setdefault(key, []).append(t1 - t0)
    return {k: {"ms": float(np.mean(v)), "launches": len(v)} for k, v in out.items()}


def kernel_rooflines(times, L, s, B, prec, recursion, pk):
    """Achieved fraction of each kernel's bound: algorithmic work of one launch over its live
    average duration.  Algorithmic bytes count each operand once (a lower bound on DRAM traffic)."""
    N, M = 2 * L - 1, torus_M(L)
    macs = B * contraction_macs(L, s)
    quad = quadrant_entries(L)
    res = {}

    def entry(kernel, ms, flops=None, fpeak=None, fsrc=None, nbytes=None, extra=None):
        t = ms / 1e3
        e = {"kernel": kernel, "ms": ms}
        fr = {}
        if flops is not None:
            e["tflops"] = flops / t / 1e12
            e["flop_frac"] = e["tflops"] / fpeak[0]
            e["flop_peak"] = fpeak[0]
            e["flop_peak_source"] = fpeak[1]
            fr["flop"] = e["flop_frac"]
        if nbytes is not None:
            e["gbs"] = nbytes / t / 1e9
            e["hbm_frac"] = e["gbs"] / pk["hbm_gbs"][0]
            e["algorithmic_bytes"] = nbytes
            fr["hbm"] = e["hbm_frac"]
        e["bound"] = max(fr, key=fr.get) if fr else None
        if extra:
            e.update(extra)
        files = KERNEL_SOURCES.get(kernel) or KERNEL_SOURCES.get(kernel.split(" ")[0], [])
        e["traffic"] = traffic_for(kernel, files, "L=%d s=%d B=%d %s" % (L, s, B, prec))
        return e

    tc = prec in ("tf32x3", "bf16x6")
    # bytes of one real operand value in the contraction's tiles in global memory: 3xTF32 tiles
    # hold the FP32 value (split into hi + lo in shared memory), split-BF16 tiles the two parts
    tv = 4.0 if prec == "tf32x3" else 8.0
    for key, v in times.items():
        ms = v["ms"]
        if key == "recursion_inverse" and tc and recursion != "risbo" and prec == "tf32x3":
            u = lane_updates(L)
            res[key] = entry("lane_recursion_kernel", ms, 2.5 * u, pk["fp64_tflops"], None, quad * tv,
                             {"fp64_instr_frac": (1.5 * u / (ms / 1e3)) / (pk["fp64_tflops"][0] * 1e12 / 2.0),
                              "work": "%.3g updates x 1.5 FP64 instructions (2.5 flops: the rescaled relation's "
                                      "fused multiply-add, and the coefficient m alpha at every other row, made "
                                      "on the integer pipe at the others); writes the inverse's A tiles" % u,
                              "fp64_probe_tflops": FP64_PROBE_TFLOPS})
        elif key.startswith("recursion"):
            if recursion == "risbo":
                nh, ni = recursion_updates(L)
                res[key] = entry("risbo_kernel", ms, 7.0 * nh + 8.0 * ni, pk["fp64_tflops"], None, quad * 8.0,
                                 {"fp64_instr_frac": ((4.0 * nh + 5.0 * ni) / (ms / 1e3)) / (pk["fp64_tflops"][0] * 1e12 / 2.0)})
            else:
                u = column_updates(L)
                # tile output (3xTF32): the rescaled relation's FMA, and the coefficient product at
                # every other row (the integer pipe makes it at the others); FP64 table: b y and
                # the FMA, the coefficient on the integer pipe
                direct = prec == "tf32x3"
                ni, nf = (1.5, 2.5) if direct else (2.0, 3.0)
                res[key] = entry("column_tiles_kernel" if direct else "column_recursion_kernel (table)", ms,
                                 nf * u, pk["fp64_tflops"], None, quad * (tv if direct else 8.0),
                                 {"fp64_instr_frac": (ni * u / (ms / 1e3)) / (pk["fp64_tflops"][0] * 1e12 / 2.0),
                                  "work": "%.3g updates x %g FP64 instructions (%g flops); writes %s" % (
                                      u, ni, nf, "the A tiles (%d B an entry)" % tv if direct else "the FP64 table"),
                                  "fp64_probe_tflops": FP64_PROBE_TFLOPS})
        elif key in ("contraction_inverse", "contraction_forward") and tc:
            nprod, pkey = (3, "tf32_tflops") if prec == "tf32x3" else (6, "bf16_tflops_sustained")
            fwd = key.endswith("forward")
            data = B * (N * L if fwd else L * L) * 2.0 * tv
            outb = B * (L * L if fwd else N * L) * 8.0
            res[key] = entry("tc_gemm_kernel<%s>" % ("forward" if fwd else "inverse"), ms, nprod * 4.0 * macs,
                             pk[pkey], None, quad * tv + data + outb,
                             {"useful_tflops": 4.0 * macs / (ms / 1e3) / 1e12, "issued_products": nprod})
        elif key in ("contraction_inverse", "contraction_forward"):
            fwd = key.endswith("forward")
            pkey = "fp64_tflops" if prec == "fp64" else "fp32_tflops"
            res[key] = entry(("project_kernel" if fwd else "inverse_kernel") + " (SIMT)", ms, 4.0 * macs, pk[pkey], None,
                             quad * 8.0 + B * (L * L + N * L) * (16.0 if prec == "fp64" else 8.0))
        elif key == "pack_data":
            res[key] = entry("pack_v_kernel", ms, None, None, None, B * L * L * (8.0 + 2.0 * tv))
        elif key in ("theta_inverse", "phi_inverse", "phi_forward", "theta_forward") and prec != "fp64":
            rows = B * L
            nfft = 4 if key == "theta_forward" else 2
            outb = B * L * (N + 1) * (2.0 * tv if (key == "theta_forward" and tc) else 8.0)
            kern = {"theta_inverse": "inverse_theta_kernel", "phi_inverse": "phi_kernel<+1>",
                    "phi_forward": "phi_kernel<-1>", "theta_forward": "forward_theta_kernel"}[key]
            res[key] = entry(kern, ms, rows * nfft * fft_flops(M), pk["fp32_tflops"], None, B * L * N * 8.0 + outb,
                             {"work": "%d rows x %d FFTs of %d points (5 M log2 M flops each)" % (rows, nfft, M)})
    return res


def source_hash(*files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel, files, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on these sources and
    this workload."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        j = json.load(open(path)).get(kernel)
    except Exception:
        return None
    if not j or j.get("source_hash") != source_hash(*files) or j.get("workload") != workload:
        return None
    return j.get("bytes_per_launch")


# ---------------------------------------------------------------------------------------------
# the ssht arm
# ---------------------------------------------------------------------------------------------

def run_ssht(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    __graft_entry__.build()
    from paper_0807_4494_gb300 import inputs, ssht

    L, s, B = args.L, args.s, args.batch
    prec = args.precision
    if prec == "auto":
        prec = "tf32x3" if B <= 64 else "fp32"
    t_plan = time.perf_counter()
    plan = ssht.Plan(L, s, B, precision=prec, delta_mode=args.delta_mode, tune=not args.no_tune)
    plan_s = time.perf_counter() - t_plan
    tile_cfg = plan.tile_config() if prec in ("tf32x3", "bf16x6") else None
    cdt = plan.dtype
    flm_np = inputs.coeffs(L, s, B, seed=rank_seed(rank, B), spectrum="cmb")
    flm = torch.from_numpy(flm_np).to(cdt).to(device)
    grid = torch.empty(plan.grid_shape(), dtype=cdt, device=device)
    back = torch.empty(plan.coeff_shape(), dtype=cdt, device=device)
    stream = torch.cuda.current_stream()

    def step():
        plan.inverse(flm, out=grid)
        plan.forward(grid, out=back)

    sampler = ClockSampler(device.index) if rank == 0 else None
    if sampler:
        sampler.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.check()
    plan.profile(True)
    _, launches0 = plan.profile_read()
    barrier(world, device)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world, device)
    ms_local = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    trace = plan.profile_trace()
    stages, launches1 = plan.profile_read()
    plan.profile(False)
    plan.check()
    ms = max_over_ranks(ms_local, world, device)
    value = throughput(world, B, args.steps, ms)
    ms_step = ms / args.steps

    # the recursion alone, nothing beside it (in the step the forward call's sweep shares its SMs
    # with the torus passes): a few sweeps through ssht_wigner_delta, timed by the same stage events
    delta_alone_ms = None
    if rank == 0 and args.delta_mode == "recompute":
        tab = torch.empty(L * (L + 1) * (2 * L + 1) // 6, dtype=torch.float64, device=device)
        plan.wigner_delta(out=tab)
        torch.cuda.synchronize()
        plan.profile(True)
        for _ in range(3):
            plan.wigner_delta(out=tab)
            torch.cuda.synchronize()
        dst, _ = plan.profile_read()
        plan.profile(False)
        plan.check()
        if dst["delta"][1] > 0:
            delta_alone_ms = dst["delta"][0] / dst["delta"][1]
        del tab

    # end to end through the C ABI with host buffers: H2D of the coefficients, D2H of the result
    # (measured before the oracle check below keeps the host cores busy)
    e2e = None
    if not args.no_e2e:
        h_in = torch.empty(plan.coeff_shape(), dtype=cdt, pin_memory=True)
        h_in.copy_(flm.cpu())
        h_out = torch.empty(plan.coeff_shape(), dtype=cdt, pin_memory=True)

        def step_host():
            plan.inverse(h_in, out=grid)        # host -> device inside the call
            plan.forward(grid, out=h_out)       # device -> host inside the call
        for _ in range(max(1, args.warmup)):
            step_host()
        torch.cuda.synchronize()
        barrier(world, device)
        nrep = max(5, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(nrep):
            step_host()
        torch.cuda.synchronize()
        barrier(world, device)
        el = max_over_ranks(time.perf_counter() - t0, world, device)
        nbytes = B * L * L * h_in.element_size()
        e2e = {"value": world * B * nrep / el, "unit": "transforms/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": nrep,
               "how": "one stream: each step the inverse copies the pinned host coefficients to the device (copy "
                      "engines), the forward returns its result to pinned host memory and the call waits for it"}
        # Two request streams in flight, the pattern of a server: each with its own plan, CUDA stream,
        # pinned buffers and host thread, through the same calls; every step of each still copies its
        # input in and its result out inside the timed region, and one stream's copies overlap the
        # other's kernels.
        import threading
        plan2 = ssht.Plan(L, s, B, precision=prec, delta_mode=args.delta_mode)
        grid2 = torch.empty(plan2.grid_shape(), dtype=cdt, device=device)
        h_in2 = torch.empty(plan2.coeff_shape(), dtype=cdt, pin_memory=True)
        h_in2.copy_(h_in)
        h_out2 = torch.empty(plan2.coeff_shape(), dtype=cdt, pin_memory=True)
        streams = [torch.cuda.Stream(device=device), torch.cuda.Stream(device=device)]
        work = [(plan, grid, h_in, h_out), (plan2, grid2, h_in2, h_out2)]

        def run(k, n):
            p_, g_, i_, o_ = work[k]
            with torch.cuda.stream(streams[k]):
                for _ in range(n):
                    p_.inverse(i_, out=g_)
                    p_.forward(g_, out=o_)

        def both(n):
            ts = [threading.Thread(target=run, args=(k, n)) for k in range(2)]
            for t in ts:
                t.start()
            for t in ts:
                t.join()
        both(max(1, args.warmup))
        torch.cuda.synchronize()
        barrier(world, device)
        t0 = time.perf_counter()
        both(nrep)
        torch.cuda.synchronize()
        barrier(world, device)
        el2 = max_over_ranks(time.perf_counter() - t0, world, device)
        e2e["two_streams"] = {"value": world * 2 * B * nrep / el2, "unit": "transforms/s",
                              "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps_per_stream": nrep}
        plan2.close()
        del grid2, h_in2, h_out2

    # roundtrip error over the whole batch, and the oracle check on sampled fields
    rt = float((back - flm).abs().max() / flm.abs().max())
    check = None
    fields = sorted(set(range(0, B, 8)) | {B - 1})
    inv_oracle = {}

    def oracle_errors(g_dev, b_dev):
        from oracle import transforms as T
        g = g_dev.cpu().numpy()
        b_out = b_dev.cpu().numpy()
        e_inv, e_fwd = 0.0, 0.0
        for b in fields:
            if b not in inv_oracle:
                inv_oracle[b] = T.inverse(flm_np[b], L, s)
            f_or = inv_oracle[b]
            e_inv = max(e_inv, float(np.abs(g[b] - f_or).max() / np.abs(f_or).max()))
            fw_or = T.forward(g[b].astype(np.complex128), L, s)
            e_fwd = max(e_fwd, float(np.abs(b_out[b] - fw_or).max() / np.abs(fw_or).max()))
        return e_inv, e_fwd

    if rank == 0 and not args.no_check:
        e_inv, e_fwd = oracle_errors(grid, back)
        check = {"inverse": e_inv, "forward": e_fwd, "roundtrip": rt, "fields_checked": fields,
                 "measure": "max|x - oracle| / max|oracle|"}

    # the other split form of the tensor-core contraction on the same workload (3xTF32 <-> split-BF16)
    alt = None
    if not args.no_alt and prec in ("tf32x3", "bf16x6"):
        other = "bf16x6" if prec == "tf32x3" else "tf32x3"
        aplan = ssht.Plan(L, s, B, precision=other, delta_mode=args.delta_mode)
        grid2 = torch.empty_like(grid)
        back2 = torch.empty_like(back)

        def astep():
            aplan.inverse(flm, out=grid2)
            aplan.forward(grid2, out=back2)
        for _ in range(args.warmup):
            astep()
        torch.cuda.synchronize()
        barrier(world, device)
        nalt = min(args.steps, 10)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(nalt):
            astep()
        a1.record(stream)
        torch.cuda.synchronize()
        aplan.check()
        ams = max_over_ranks(a0.elapsed_time(a1), world, device)
        alt = {"precision": other, "value": world * B * nalt / (ams / 1e3), "unit": "transforms/s",
               "ms_per_step": ams / nalt, "steps": nalt,
               "roundtrip": float((back2 - flm).abs().max() / flm.abs().max())}
        if rank == 0 and not args.no_check:
            e_inv, e_fwd = oracle_errors(grid2, back2)
            alt.update({"inverse": e_inv, "forward": e_fwd, "fields_checked": fields})
        aplan.close()
        del grid2, back2

    # every kernel of the step, timed live (stage brackets on their own streams), against its
    # bound; the top-level line is the kernel that takes the most time
    sms, clk = device_units()
    pk = peaks(sms, clk)
    kern = kernel_rooflines(split_trace(trace, args.steps), L, s, B, prec, "column", pk)
    roof = None
    if kern:
        # the dominant kernel: the longest on the caller's stream, the step's critical path (the
        # recursions run beside it on the plan's second stream, their live time stretched by the
        # SMs they share; they are reported under "kernels")
        path = [k for k in kern if not k.startswith("recursion")] or list(kern)
        dom = max(path, key=lambda k: kern[k]["ms"])
        e = kern[dom]
        if e["bound"] == "hbm":
            roof = {"bound": "hbm", "achieved": e["gbs"], "peak": pk["hbm_gbs"][0], "unit": "GB/s",
                    "frac": e["hbm_frac"], "peak_source": pk["hbm_gbs"][1]}
        else:
            roof = {"bound": "tensor" if e["kernel"].startswith("tc_gemm") else "alu", "achieved": e["tflops"],
                    "peak": e["flop_peak"], "unit": "TFLOP/s", "frac": e["flop_frac"],
                    "peak_source": e["flop_peak_source"]}
        roof.update({"kernel": e["kernel"], "stage": dom, "ms_per_launch": e["ms"], "traffic": e["traffic"]})
        if delta_alone_ms and dom.startswith("recursion"):
            u = column_updates(L)
            roof["alone"] = {"ms": delta_alone_ms, "achieved": 4.0 * u / (delta_alone_ms / 1e3) / 1e12,
                             "note": "the table-writing sweep timed by itself (ssht_wigner_delta)"}
    stage_ms = {k: round(v[0] / args.steps, 4) for k, v in stages.items() if v[1] > 0}

    # column pairing along theta (two phi-frequency columns of opposite parity in one DFT): the
    # inverse theta pass transforms pairs, the adjoint's theta pass one column at a time, each
    # with two FFTs of the same length -- their time per column shows what the pairing saves
    pairing = None
    if prec != "fp64":
        plan.profile(True)
        adj_out = torch.empty(plan.coeff_shape(), dtype=cdt, device=device)
        for _ in range(3):
            plan.adjoint(grid, out=adj_out)
        atrace = plan.profile_trace()
        plan.profile(False)
        plan.check()
        afft = [t1 - t0 for name, lane, t0, t1 in atrace if name == "fft" and lane == 0]
        theta_adj = float(np.mean(afft[1::2])) if len(afft) >= 2 else None
        theta_inv = kern.get("theta_inverse", {}).get("ms")
        if theta_adj and theta_inv:
            cols = B * (2 * L - 1)
            pairing = {"theta_inverse_paired_ms": theta_inv, "theta_adjoint_unpaired_ms": theta_adj,
                       "us_per_column_paired": 1e3 * theta_inv / cols, "us_per_column_unpaired": 1e3 * theta_adj / cols,
                       "unpaired_over_paired": theta_adj / theta_inv,
                       "note": "same DFT length and FFT count per transformed sequence; the adjoint's theta pass "
                               "also writes the data tiles, the inverse's the phi input"}
        del adj_out

    # the plain FP64 GPU transform of the same workload (the mixed-precision form must beat it)
    fp64_line = None
    if not args.no_fp64 and prec != "fp64":
        fp64_line = run_fp64(args, torch, inputs, ssht, world, device, stream, rank, pk, inv_oracle, flm_np)

    # the plan-time Delta cache (the paper's timing protocol: precomputed Delta in memory)
    cache_line = None
    if not args.no_cache_line and args.delta_mode == "recompute":
        t0 = time.perf_counter()
        cplan = ssht.Plan(L, s, B, precision=prec, delta_mode="cache")
        build_s = time.perf_counter() - t0

        def cstep():
            cplan.inverse(flm, out=grid)
            cplan.forward(grid, out=back)
        for _ in range(args.warmup):
            cstep()
        torch.cuda.synchronize()
        barrier(world, device)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            cstep()
        c1.record(stream)
        torch.cuda.synchronize()
        cms = max_over_ranks(c0.elapsed_time(c1), world, device)
        cache_line = {"value": world * B * args.steps / (cms / 1e3), "unit": "transforms/s",
                      "ms_per_step": cms / args.steps, "plan_build_s": build_s}
        cplan.close()

    # the uneven batch: 256 fields, L ~ U{128,256,512,1024}, s ~ U{0,+-1,+-2}, N(0,1) coefficients,
    # one group (buckets by (L, s), shared Delta per L, tuned contraction per bucket), inverse +
    # forward captured into one CUDA graph and replayed
    uneven = None
    if not args.no_uneven:
        uneven = run_uneven(args, torch, inputs, ssht, world, device, stream, rank)

    # the paper's real workload: real spin-0 fields (U[-1,1] coefficients with the reality
    # condition), 2B real fields per step, two per complex transform
    real_line = None
    if not args.no_real and prec in ("tf32x3", "bf16x6", "fp32", "fp64"):
        real_line = run_real(args, torch, inputs, ssht, world, device, stream, rank, prec)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(L, s, flm_np[0])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32"}.get(prec, prec) + " (Delta recursion f64)",
            "data": "synthetic: sf_lm ~ CN(0, 1/(l+1)^2) (Re, Im each N(0, 1/(2(l+1)^2))), seeds rank*B .. rank*B+B-1",
            "config": {"workload": "L=%d s=%d B=%d fwd+inv per step" % (L, s, B), "L": L, "s": s, "batch": B,
                       "precision": prec, "delta_mode": args.delta_mode, "parallelism": "dp%d (independent fields)" % world,
                       "contraction_shape": tile_cfg, "plan_create_s": plan_s,
                       "l2": "inputs larger than L2 (%.2f GB of coefficients, %.2f GB of samples per step)" % (
                           flm.numel() * flm.element_size() / 1e9, grid.numel() * grid.element_size() / 1e9)},
            "rel_err": check,
            "alt_precision": alt,
            "roofline": roof,
            "kernels": kern,
            "stage_ms_per_step": stage_ms,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": int(launches1 - launches0),
            "fp64": fp64_line,
            "theta_pairing": pairing,
            "delta_cache": cache_line,
            "uneven_batch": uneven,
            "real_fields": real_line,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_fp64(args, torch, inputs, ssht, world, device, stream, rank, pk, inv_oracle, flm_np):
    """The plain FP64 GPU transform on the same band-limit and spin: B fields (the headline batch)
    and one field, with the FP64 contractions' live rooflines and the errors of field 0."""
    L, s = args.L, args.s
    res = {}
    for B in sorted({args.batch, 1}, reverse=True):
        plan = ssht.Plan(L, s, B, precision="fp64")
        flm = torch.from_numpy(flm_np[:B]).to(torch.complex128).to(device)
        grid = torch.empty(plan.grid_shape(), dtype=torch.complex128, device=device)
        back = torch.empty(plan.coeff_shape(), dtype=torch.complex128, device=device)

        def step():
            plan.inverse(flm, out=grid)
            plan.forward(grid, out=back)
        step()
        torch.cuda.synchronize()
        nrep = 3 if B > 1 else 5
        plan.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nrep):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        trace = plan.profile_trace()
        plan.profile(False)
        plan.check()
        ms = max_over_ranks(e0.elapsed_time(e1), world, device)
        # FP64 plans make the same table in both calls; the forward call's sweep waits beside the
        # inverse's cuFFT passes for room on the SMs, so its bracket measures that wait: the
        # inverse call's bracket is the sweep
        times = {k: v for k, v in split_trace(trace, nrep).items()
                 if k in ("recursion_inverse", "contraction_inverse", "contraction_forward")}
        line = {"batch": B, "value": throughput(world, B, nrep, ms), "unit": "transforms/s", "ms_per_step": ms / nrep,
                "steps": nrep, "kernels": kernel_rooflines(times, L, s, B, "fp64", "column", pk)}
        if rank == 0 and not args.no_check:
            from oracle import transforms as T
            if 0 not in inv_oracle:
                inv_oracle[0] = T.inverse(flm_np[0], L, s)
            f_or = inv_oracle[0]
            g0 = grid[0].cpu().numpy()
            fw = T.forward(g0, L, s)
            line["inverse"] = float(np.abs(g0 - f_or).max() / np.abs(f_or).max())
            line["forward"] = float(np.abs(back[0].cpu().numpy() - fw).max() / np.abs(fw).max())
        res["B%d" % B] = line
        plan.close()
        del flm, grid, back
        torch.cuda.empty_cache()
    return res


def run_real(args, torch, inputs, ssht, world, device, stream, rank, prec):
    L, nreal = args.L, 2 * args.batch
    plan = ssht.Plan(L, 0, nreal, precision=prec, delta_mode=args.delta_mode, real=True)
    flm_np = inputs.coeffs(L, 0, nreal, seed=rank_seed(rank, nreal), spectrum="paper", real=True)
    flm = torch.from_numpy(flm_np).to(plan.dtype).to(device)
    f = torch.empty(plan.grid_shape(), dtype=plan.grid_dtype, device=device)
    back = torch.empty(plan.coeff_shape(), dtype=plan.dtype, device=device)

    def step():
        plan.inverse(flm, out=f)
        plan.forward(f, out=back)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world, device)
    nrep = min(args.steps, 10)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nrep):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    plan.check()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    res = {"workload": "L=%d s=0, %d real fields per step (U[-1,1] with the reality condition), two per complex "
                       "transform" % (L, nreal), "precision": prec, "value": throughput(world, nreal, nrep, ms),
           "unit": "transforms/s", "ms_per_step": ms / nrep, "steps": nrep,
           "roundtrip": float((back - flm).abs().max() / flm.abs().max())}
    if rank == 0 and not args.no_check:
        from oracle import transforms as T
        f_or = T.inverse(flm_np[0], L, 0)
        res["inverse"] = float(np.abs(f[0].cpu().numpy() - f_or.real).max() / np.abs(f_or).max())
    plan.close()
    return res


def run_uneven(args, torch, inputs, ssht, world, device, stream, rank):
    n = 256
    Ls, ss = inputs.uneven_batch(n, seed=rank_seed(rank, n))
    t0 = time.perf_counter()
    g = ssht.Group(Ls, ss, precision="fp32", delta_mode="recompute", tune=True)
    build_s = time.perf_counter() - t0
    flms = [inputs.coeffs(L, s_, 1, seed=rank_seed(rank, n) + i)[0] for i, (L, s_) in enumerate(zip(Ls, ss))]
    flat = g.pack_coeffs([torch.from_numpy(x).to(torch.complex64).to(device) for x in flms])
    f = g.empty_grid()
    back = g.empty_coeffs()
    g.capture(flat, f, back)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    barrier(world, device)
    nrep = min(args.steps, 10)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nrep):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    g.check()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device)
    res = {"fields": n, "value": throughput(world, n, nrep, ms), "unit": "transforms/s", "ms_per_step": ms / nrep,
           "steps": nrep, "graph": "one CUDA graph per step (inverse + forward of all fields)",
           "group_build_s": build_s,
           "buckets": [{"L": L, "s": s_, "fields": c, "contraction": {0: "fp64", 1: "fp32", 2: "tf32x3", 3: "bf16x6"}[p]}
                       for (L, s_, c, p) in g.buckets()],
           "roundtrip": float((back - flat).abs().max() / flat.abs().max())}
    if rank == 0 and not args.no_check:
        # the first field of every (L, s) bucket against the oracle, inverse and forward
        from oracle import transforms as T
        fs, bs = g.unpack_grid(f), g.unpack_coeffs(back)
        e_inv, e_fwd, seen = 0.0, 0.0, set()
        for i, (Lq, sq_) in enumerate(zip(Ls, ss)):
            if (Lq, sq_) in seen:
                continue
            seen.add((Lq, sq_))
            f_or = T.inverse(flms[i], Lq, sq_)
            fi = fs[i].cpu().numpy()
            e_inv = max(e_inv, float(np.abs(fi - f_or).max() / np.abs(f_or).max()))
            fw = T.forward(fi.astype(np.complex128), Lq, sq_)
            e_fwd = max(e_fwd, float(np.abs(bs[i].cpu().numpy() - fw).max() / np.abs(fw).max()))
        res["rel_err"] = {"inverse": e_inv, "forward": e_fwd, "buckets_checked": len(seen),
                          "fields_checked": "the first field of every (L, s) bucket"}
    g.close()
    return res


def cpu_baseline(L, s, flm1):
    """The oracle, as it stands, on the host cores: one field of the workload, inverse + forward."""
    from oracle import transforms as T
    t0 = time.perf_counter()
    f = T.inverse(flm1, L, s)
    T.forward(f, L, s)
    el = time.perf_counter() - t0
    return {"value": 1.0 / el, "unit": "transforms/s", "cores": T.num_threads(), "kind": "oracle",
            "sample": "1 field of the L=%d s=%d workload (field 0), inverse + forward, FP64, %.1f s" % (L, s, el)}


# ---------------------------------------------------------------------------------------------
# the reference arm: the CPU oracle
# ---------------------------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import _lib
    from oracle import transforms as T
    from paper_0807_4494_gb300 import inputs
    _lib.build()
    L, s = args.L, args.s
    flm = inputs.coeffs(L, s, 1, seed=0, spectrum="cmb")[0]

    def step():
        f = T.inverse(flm, L, s)
        T.forward(f, L, s)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic: field 0 of the workload",
        "config": {"workload": "L=%d s=%d B=%d fwd+inv per step" % (L, s, args.batch), "L": L, "s": s,
                   "batch": args.batch, "sample": "1 field per step"},
        "cpu_baseline": {"value": value, "unit": "transforms/s", "kind": "oracle", "cores": T.num_threads(),
                         "sample": "1 field of the workload per step (inverse + forward), FP64 C/OpenMP + numpy.fft"},
        "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def error_sweep(args):
    """Error vs band-limit (max-norm relative, vs the FP64 oracle) of every precision, one field of
    the CMB-like spectrum (seed 0) per L: inverse, forward of the GPU's own grid, roundtrip."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from oracle import transforms as T
    from paper_0807_4494_gb300 import inputs, ssht
    # the single-field FP64 configuration: Re/Im iid N(0,1), spins 0 and 2 separately, L = 32 .. 512
    for s in (0, 2):
        for L in (32, 64, 128, 256, 512):
            flm = inputs.coeffs(L, s, 1, seed=0)
            f_or = np.ascontiguousarray(T.inverse(flm[0], L, s))
            plan = ssht.Plan(L, s, 1, precision="fp64")
            x = torch.from_numpy(flm).cuda()
            f = plan.inverse(x)
            back = plan.forward(f)
            plan.check()
            f0 = f[0].cpu().numpy()
            fw = T.forward(f_or, L, s)
            print(json.dumps({"L": L, "s": s, "spectrum": "flat N(0,1)", "precision": "fp64",
                              "inverse": float(np.abs(f0 - f_or).max() / np.abs(f_or).max()),
                              "forward_of_oracle_grid": float(np.abs(plan.forward(torch.from_numpy(f_or[None]).cuda())[0].cpu().numpy() - fw).max() / np.abs(fw).max()),
                              "roundtrip": float((back - x).abs().max() / x.abs().max())}), flush=True)
            plan.close()
    s = args.s
    for L in (32, 64, 128, 256, 512, 1024, 2048):
        flm = inputs.coeffs(L, s, 1, seed=0, spectrum="cmb")
        f_or = T.inverse(flm[0], L, s)
        for prec in ("fp64", "fp32", "tf32x3", "bf16x6"):
            plan = ssht.Plan(L, s, 1, precision=prec)
            x = torch.from_numpy(flm).to(plan.dtype).cuda()
            f = plan.inverse(x)
            back = plan.forward(f)
            plan.check()
            f0 = f[0].cpu().numpy()
            fw = T.forward(f0.astype(np.complex128), L, s)
            line = {"L": L, "s": s, "spectrum": "cmb CN(0, 1/(l+1)^2)", "precision": prec,
                    "inverse": float(np.abs(f0 - f_or).max() / np.abs(f_or).max()),
                    "forward": float(np.abs(back[0].cpu().numpy() - fw).max() / np.abs(fw).max()),
                    "roundtrip": float((back - x).abs().max() / x.abs().max())}
            if prec == "fp64" and L <= 2048:
                # the same inverse with the paper's Risbo recursion for Delta
                rplan = ssht.Plan(L, s, 1, precision="fp64", recursion="risbo")
                fr = rplan.inverse(x)[0].cpu().numpy()
                rplan.check()
                rplan.close()
                line["inverse_risbo_recursion"] = float(np.abs(fr - f_or).max() / np.abs(f_or).max())
            if prec == "fp64":
                # the paper's triangular forward of the same grid: its five error metrics against
                # the coefficients the grid was made from, next to the quadrature forward's
                tri = plan.forward_triangular(f)[0].cpu().numpy()
                line["triangular_forward_vs_true"] = T.error_metrics(flm[0], tri)
                line["quadrature_forward_vs_true"] = T.error_metrics(flm[0], back[0].cpu().numpy())
            print(json.dumps(line), flush=True)
            plan.close()
            del f, back, x
            torch.cuda.empty_cache()


def main():
    args = parse()
    if args.error_sweep:
        error_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ssht(args)


if __name__ == "__main__":
    main()
