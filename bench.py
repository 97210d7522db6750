"""Throughput benchmark of the fast discrete Walsh transform pipeline on GB300.

Workload (default): p = 2, s = 32, m = 24 (N = 16,777,216 net points), a batch
of 32 FP32 product functions f(x) = prod_j (1 + (x_j - 1/2)/j^2) evaluated on
the net on the device, spectral weight prod_j (1 + k_j)^-2.  One step is the
whole hot path over the batch: forward transform (Algorithm 1), scaling,
weighting, the truncation / superposition variance classes with the effective
dimensions, and the inverse transform (Algorithm 2) -- one dwt_interpolate
call.  The plan (net, K(C) tables) is built once beforehand and timed apart.

Inputs (2 GiB) are larger than the 126 MB L2, so no flush is needed between
steps.  Multi-GPU: each rank runs its own batch on its own GPU with no
collective (the functions are independent), scaling is "weak".

``--impl reference`` times the CPU oracle (the FP64 restatement of the paper
in oracle/) on a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "net points/s (p=2, m=24, s=32, batch 32: forward + weight + effdim + inverse)"
UNIT = "points/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, pg, device):
    """The slowest rank's time: every rank returns the maximum (replicas finish
    when the last one does).  pg is torch.distributed or None."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world_size, max_ms):
    """Units processed by all ranks per second of the slowest rank's time."""
    return units_per_rank * world_size / (max_ms / 1e3)


def rank_requests(count, rank):
    """The serving requests of one rank: disjoint request ids per rank."""
    import synthetic as S
    return S.serving_requests(count, first=rank * count)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms while the timed
    region runs.  Samples carry the host time they were read; ``mark`` records
    the timed region's bounds, so the summary reports the samples inside it and
    those of the whole sampled window (the timed region padded by untimed
    replays of the same step before and after it)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.region = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the sampler is running (first line read) before the timed region starts
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
            self.lines.clear()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        self.region = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _parse(lines):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return sm, mx, reasons

    def summary(self):
        sm, mx, reasons = self._parse([ln for _, ln in self.lines])
        inside = [ln for _, ln in self.lines]
        if self.region:
            # a sample read at host time t describes the GPU during the preceding period
            t0, t1 = self.region
            inside = [ln for t, ln in self.lines if t0 < t <= t1 + self.PERIOD_MS / 1e3]
        smi, _, reasons_i = self._parse(inside)
        return {"sm_mhz": statistics.median(smi) if smi else (statistics.median(sm) if sm else None),
                "sm_max_mhz": mx, "reasons": sorted(reasons | reasons_i), "samples": len(smi),
                "samples_window": len(sm), "period_ms": self.PERIOD_MS,
                "window": "the timed region padded by about 0.3 s of untimed replays of the same step on each side"}


def _bind_to_gpu_node(local):
    """Run this process on the CPUs next to GPU ``local`` (from the PCI device's
    local_cpulist), so that page-locked host buffers allocated afterwards sit in
    that socket's memory.  Returns the CPU list, or None if it is unknown."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(local)
        bdf = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bdf) as fh:
            spec = fh.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except Exception:
        return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def run_reference(args):
    """The CPU oracle on a bounded sample of the same workload (one function)."""
    import numpy as np

    import oracle
    import synthetic as S

    ws, rank, _ = _dist()
    if rank != 0:
        return
    w = S.workload_p2_m24(batch=1)
    p, m, s = w["p"], w["m"], w["s"]
    N = p ** m
    oracle.lib()
    # input function: oracle net points and the product function (untimed)
    Y = oracle.net_points(p, m, w["C"])
    f = oracle.eval_product(p, m, Y, w["coef"][0])
    del Y
    # The timed oracle work (Algorithm 1, weight, class sums, Algorithm 2) does not
    # depend on the table values, so the plan-time K(C) tables (excluded from the
    # metric on both arms) are replaced by constants of the same shape here.
    W = np.ones(N)
    cls = np.zeros((N, 2), dtype=np.uint8)
    # one function of the batch per thread on every host core this process may
    # use (the oracle's C routines release the interpreter lock); at most four
    # timed steps of about 4 s each, so the arm ends within a minute or two
    import concurrent.futures as cf
    threads = max(1, min(len(os.sched_getaffinity(0)), 32))
    steps = max(1, min(args.steps, 4))
    times = []
    with cf.ThreadPoolExecutor(threads) as ex:
        for _ in range(steps):
            t0 = time.perf_counter()
            list(ex.map(lambda _: oracle.interpolate(p, m, f, W, cls, s)[3], range(threads)))
            times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    value = threads * N / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": 0, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "p2_m24_s32_b32", "p": 2, "m": 24, "s": 32, "global_batch": 32,
                   "l2": "inputs larger than L2",
                   "subsample": {"functions_per_step": threads, "of_batch": 32, "steps": len(times),
                                 "steps_asked": args.steps, "warmup": 0,
                                 "tables": "K(C) weight and class tables replaced by constants (plan time is "
                                           "excluded on both arms; the timed arithmetic does not depend on them)"}},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d of the 32 functions (N=2^24) per step, one per thread, forward+weight+class "
                                   "sums+inverse in FP64; K(C) tables replaced by constants" % threads},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(acc_in=None):
    """Oracle time on a bounded sample of the workload: one function on one thread,
    then one function per thread on every host core this process may use (the
    oracle's C routines release the interpreter lock, so the threads run in
    parallel).  About 10-20 s in total.  With acc_in (GPU outputs for function 0
    of the workload) it also returns their deviation from the FP64 oracle."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    import synthetic as S

    w = S.workload_p2_m24(batch=1)
    p, m, s = w["p"], w["m"], w["s"]
    N = p ** m
    Y = oracle.net_points(p, m, w["C"])
    f = oracle.eval_product(p, m, Y, w["coef"][0])
    del Y
    W = np.ones(N)
    cls = np.zeros((N, 2), dtype=np.uint8)
    t0 = time.perf_counter()
    oracle.interpolate(p, m, f, W, cls, s)
    t1 = time.perf_counter() - t0
    threads = max(1, min(len(os.sched_getaffinity(0)), 32))
    with cf.ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda _: oracle.interpolate(p, m, f, W, cls, s)[3], range(threads)))
        tn = time.perf_counter() - t0
    acc = accuracy_vs_oracle(acc_in, f) if acc_in is not None else None
    return {"value": threads * N / tn, "unit": UNIT, "cores": threads, "kind": "oracle",
            "single_thread_value": N / t1, "accuracy_vs_oracle": acc,
            "sample": "%d functions of the batch (N=2^24 each), one per thread, forward+weight+class sums+inverse "
                      "in FP64; K(C) tables replaced by constants (plan time excluded on both arms)" % threads}


def accuracy_vs_oracle(acc_in, f):
    """Relative L2 of the GPU results of function 0 of the timed workload against
    the FP64 oracle (Algorithm 1 of the oracle's own f), per path, and the int32
    path's bit-exactness on one function of the p = 2, m = 20 int32 workload."""
    import numpy as np

    import oracle
    import synthetic as S

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    ref = oracle.fwt(2, 24, f).real
    out = {"function": "0 of p2_m24_s32_b32 (N = 2^24), oracle FP64",
           "forward_f32_butterfly_rel_l2": rel(acc_in["fwd_f32"], ref),
           "forward_split_bf16_tc_rel_l2": rel(acc_in["fwd_tc"], ref),
           "round_trip_f32_rel_l2": rel(acc_in["round_trip_f32"], f),
           "tolerance_f32": 1e-5}
    w20 = S.workload_p2_m20()
    v = S.int_values(w20["int_seed"], 1, 1 << 20)[0].astype(np.int64)
    out["forward_i32_m20_bit_exact"] = bool(np.array_equal(acc_in["fwd_i32_m20"], oracle.fwt_i64(20, v)))
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# p = 2 interpolation kernels, read by ncu with --cache-control none on this
# workload's launches (one function per launch, as in every step), together
# with the SHA-256 of the kernel source they were taken from.  Any change to
# that source makes the figures stale: they are then reported as null.
MEASURED_TRAFFIC = {
    "source": "paper_0808_0487_gb300/csrc/dwt_p2i.cu",
    "sha256": "9f4acc73da8a8b9bcace41645fce869a7c34ae351e67f03c4ba7061996fe0bc8",
    # top pass: mean of two launches (81.5 and 100.9 MB); paired low pass: one launch
    "bytes_per_launch": {"interp_top": 91.2e6, "interp_inv_fwd": 138.5e6},
}


def _traffic(family):
    import hashlib
    try:
        src = open(os.path.join(ROOT, MEASURED_TRAFFIC["source"]), "rb").read()
    except OSError:
        return None
    if hashlib.sha256(src).hexdigest() != MEASURED_TRAFFIC["sha256"]:
        return None
    return MEASURED_TRAFFIC["bytes_per_launch"].get(family)


# Algorithmic bytes of one launch of each kernel family of dwt_interpolate at
# p = 2 (batch B, N points per function), from the per-point figures of the
# method: the whole interpolation moves f in and c out once (8 B per point) plus
# the weight and class tables once per batch (6 B per point / B).  The fused top
# pass carries one function's step (its share of the tables included); the
# paired low pass (interp_inv_fwd) reads one function's input and writes another
# function's result, 8 B per point; a lone low pass moves one of the two, 4 B.
def launch_bytes(family, N, B):
    per = {"interp_top": (8.0 + 6.0 / B) * N, "interp_inv_fwd": 8.0 * N, "interp_fwd": 4.0 * N,
           "interp_inv": 4.0 * N}
    return per.get(family)


# The launch's own loads and stores (what it touches, L2 included): the top pass
# reads and writes the intermediate and reads its 3-byte tables; a low pass
# reads and writes one function.
def launch_touched_bytes(family, N):
    per = {"interp_top": 11.0 * N, "interp_inv_fwd": 16.0 * N, "interp_fwd": 8.0 * N, "interp_inv": 8.0 * N}
    return per.get(family)


def roofline(dom, fams, N, B, peak, peak_kind):
    n, tot = fams[dom]
    avg_s = tot / n / 1e3
    alg = launch_bytes(dom, N, B)
    if alg is None:
        return None
    ach = alg / avg_s / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": _traffic(dom), "kernel": dom, "peak_kind": peak_kind, "avg_launch_us": avg_s * 1e6,
            "launches": n, "algorithmic_bytes_per_launch": alg,
            "touched_bytes_per_launch": launch_touched_bytes(dom, N),
            "touched_gbs": launch_touched_bytes(dom, N) / avg_s / 1e9}
    if roof["traffic"]:
        roof["dram_gbs"] = roof["traffic"] / avg_s / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / peak
        roof["dram_bytes_per_point"] = roof["traffic"] / N
    return roof


def memory_floor(f, c, B, N, stream, peak):
    """Time of the dwt_interpolate traffic pattern per function with no arithmetic:
    three torch copies per function (f_b into an L2-sized buffer, that buffer
    read and written in place, the buffer into c_b).  The step cannot be faster
    than its memory traffic; this shows where that floor lies on this GPU."""
    import torch
    buf = torch.empty(N, dtype=torch.float32, device=f.device)

    def one_pass():
        for b in range(B):
            buf.copy_(f[b])
            buf.mul_(1.0000001)
            c[b].copy_(buf)

    with torch.cuda.stream(torch.cuda.ExternalStream(stream.cuda_stream)):
        one_pass()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            one_pass()
        e1.record()
        torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / (3 * B)
    return {"us_per_function": us, "points_per_s": N / (us / 1e6),
            "step_hbm_frac_at_floor": N * (8.0 + 6.0 / B) / (us / 1e6) / 1e9 / peak,
            "how": "per function: copy f_b to a 64 MB buffer, buffer *= 1 in place, copy to c_b (torch kernels), "
                   "CUDA events over 3 passes of the batch"}


def run_other_configs(dwt, dev, stream, timed, steps):
    """Throughput of the transforms at the other workload shapes: p = 2, m = 20,
    s = 16 with 32 FP32 and 32 int32 functions (forward, inverse, round trip),
    mixed-size batches through the grouped call, and p = 3, m = 13, s = 8 (real
    FP32 in, complex FP32 out; forward and inverse)."""
    import numpy as np
    import torch

    import synthetic as S
    out = {}
    w = S.workload_p2_m20()
    p, m, s, B = w["p"], w["m"], w["s"], w["batch"]
    N = p ** m
    plan = dwt.dwt_plan_create(p, m, s, w["C"], dwt.DWT_PLAN_TRANSFORM_ONLY)
    for name, dt, tt in (("f32", torch.float32, dwt.DWT_F32), ("i32", torch.int32, dwt.DWT_I32)):
        x = torch.ones((B, N), dtype=dt, device=dev)
        y = torch.empty_like(x)

        def fw():
            dwt.dwt_forward(plan, x, y, B, N, N, tt, tt, stream=stream)

        def iv():
            dwt.dwt_inverse(plan, y, x, B, N, N, tt, tt, stream=stream)

        def rt():
            fw()
            iv()

        r = {}
        for k, fn in (("forward", fw), ("inverse", iv), ("round_trip", rt)):
            ms, _ = timed(fn, steps)
            r[k + "_points_per_s"] = B * N * steps / (ms / 1e3)
        out["p2_m20_s16_b32_" + name] = r
        del x, y
    # a mixed-size batch: several plans of different N in one grouped call
    # against one dwt_forward call per plan (same results, bit for bit)
    for gname, gp, gms, gin, gout in (("grouped_p2_m8_15_f32", 2, range(8, 16), dwt.DWT_F32, dwt.DWT_F32),
                                      ("grouped_p3_m5_9_c64", 3, range(5, 10), dwt.DWT_F32, dwt.DWT_C64)):
        gjobs, gpts = [], 0
        for i, gm in enumerate(gms):
            gN = gp ** gm
            gpl = dwt.dwt_plan_create(gp, gm, 1, S.small_net(gp, gm, 1, index=i), dwt.DWT_PLAN_TRANSFORM_ONLY)
            gx = torch.ones((4, gN), dtype=torch.float32, device=dev)
            gy = torch.empty((4, gN), dtype=torch.float32 if gp == 2 else torch.complex64, device=dev)
            gjobs.append((gpl, gx, gy, 4, gN, gN))
            gpts += 4 * gN

        def per_plan():
            for j in gjobs:
                dwt.dwt_forward(j[0], j[1], j[2], j[3], j[4], j[5], gin, gout, stream=stream)

        def grouped():
            dwt.dwt_forward_grouped(gjobs, gin, gout, stream=stream)

        ms_pp, l_pp = timed(per_plan, steps)
        ms_g, l_g = timed(grouped, steps)
        out[gname] = {"jobs": [[gp, gm, 4] for gm in gms], "points_per_step": gpts,
                      "per_plan_points_per_s": gpts * steps / (ms_pp / 1e3),
                      "grouped_points_per_s": gpts * steps / (ms_g / 1e3),
                      "per_plan_launches_per_step": l_pp / steps, "grouped_launches_per_step": l_g / steps}
        del gjobs
    # the kernel spline of Sec. 3.1 with its ANOVA variances (FP64) on the same
    # net: forward, weight 1 / (p^m K~), inverse and the 2s variance sums
    w2 = S.workload_p2_m20()
    plan2 = dwt.dwt_plan_create(2, 20, 16, w2["C"], dwt.DWT_PLAN_TRANSFORM_ONLY)
    N2 = 1 << 20
    dwt.dwt_spline_prepare(plan2, 2.0, [0.9 / (j + 1) ** 1.2 for j in range(16)])
    fs = torch.empty((32, N2), dtype=torch.float64, device=dev)
    dwt.dwt_eval_product(plan2, torch.tensor(w2["coef"], dtype=torch.float64, device=dev), fs, 32, N2, dwt.DWT_F64)
    cs = torch.empty_like(fs)
    vts = torch.empty((32, 17), dtype=torch.float64, device=dev)
    vss = torch.empty_like(vts)
    dims = torch.empty((32, 2), dtype=torch.int32, device=dev)

    def spl():
        dwt.dwt_spline(plan2, fs, cs, 32, N2, vts, vss, dims, stream=stream)

    ms_s, _ = timed(spl, steps)
    # the variance contraction reads |c~|^2 and the 2s tables once per function
    dwt.dwt_profile_reset()
    dwt.dwt_profile_enable(True)
    timed(spl, 1)
    dwt.dwt_profile_enable(False)
    nd, td = dwt.dwt_profile_query("spline_dots")
    dwt.dwt_profile_reset()
    dots_gbs = (2 * 16 + 1) * N2 * 8 * 32 / (td / max(nd, 1) / 1e3) / 1e9 if nd else None
    # values at the net shifted by one point of the finer net (the hold-out half
    # of a 2N-point net) and the squared error against the function there
    delta = [int(S.integers(S.stream_seed(2, S.P_SAMPLE, j), 1, 0, (1 << 21) - 1)[0]) | 1 for j in range(16)]
    vals = torch.empty_like(fs)
    sse = torch.empty(32, dtype=torch.float64, device=dev)

    def hold():
        dwt.dwt_spline_values_shifted(plan2, cs, delta, 21, vals, 32, N2, fs, sse, stream=stream)

    ms_h, _ = timed(hold, steps)
    # the spline at 256 arbitrary points (24 digits per coordinate), direct sums
    # over the net: s kernel factors and one multiply-add per function for every
    # (point, net point) pair, all FP64
    Qe = 256
    Xe = torch.from_numpy(S.integers(S.stream_seed(2, S.P_SAMPLE, 99), Qe * 16, 0, (1 << 24) - 1)
                          .astype(np.uint32).view(np.int32).reshape(Qe, 16)).to(dev)
    ve = torch.empty((32, Qe), dtype=torch.float64, device=dev)

    def ev():
        dwt.dwt_spline_eval(plan2, cs, 32, N2, Xe, Qe, 24, ve, stream=stream)

    ms_e, _ = timed(ev, max(1, steps // 10))
    ne = max(1, steps // 10)
    fp64_ops = (16 + 32) * Qe * N2 * ne / (ms_e / 1e3)
    out["spline_p2_m20_s16_b32"] = {"points_per_s": 32 * N2 * steps / (ms_s / 1e3), "dtype": "f64",
                                    "alpha": 2.0, "gamma": "0.9 / j^1.2",
                                    "holdout_points_per_s": 32 * N2 * steps / (ms_h / 1e3),
                                    "eval_at_points": {"points": Qe, "functions": 32, "digits": 24,
                                                       "ms": ms_e / ne,
                                                       "function_values_per_s": 32 * Qe * ne / (ms_e / 1e3),
                                                       "fp64_mul_per_s": fp64_ops},
                                    "dots_kernel": {"achieved_gbs": dots_gbs, "bytes_per_point": (2 * 16 + 1) * 8,
                                                    "frac": dots_gbs / _peaks()[0] if dots_gbs else None}}
    del fs, cs, vals, ve
    w = S.workload_p3_m13()
    p, m, s = w["p"], w["m"], w["s"]
    N = p ** m
    ld = (N + 3) // 4 * 4
    # the pass split measured on this GPU (DWT_PLAN_TUNE); plan time is not timed
    plan = dwt.dwt_plan_create(p, m, s, w["C"], dwt.DWT_PLAN_TRANSFORM_ONLY | dwt.DWT_PLAN_TUNE)
    x = torch.ones((1, ld), dtype=torch.float32, device=dev)
    y = torch.empty((1, ld), dtype=torch.complex64, device=dev)
    z = torch.empty_like(y)

    def fw3(st_=None):
        dwt.dwt_forward(plan, x, y, 1, ld, ld, dwt.DWT_F32, dwt.DWT_C64, stream=stream if st_ is None else st_)

    def iv3(st_=None):
        dwt.dwt_inverse(plan, y, z, 1, ld, ld, dwt.DWT_C64, dwt.DWT_C64, stream=stream if st_ is None else st_)

    # one transform is two launches of about 9 us: CUDA graphs of ten calls
    # (replayed), and the ordinary calls for comparison
    r = {}
    for k, fn in (("forward", fw3), ("inverse", iv3)):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(10):
                fn(torch.cuda.current_stream())
        torch.cuda.synchronize()
        reps = max(1, steps // 10)
        ms, _ = timed(g.replay, reps)
        r[k + "_points_per_s"] = N * 10 * reps / (ms / 1e3)
        ms, _ = timed(fn, steps)
        r[k + "_direct_calls_points_per_s"] = N * steps / (ms / 1e3)
    r["passes"] = dwt.dwt_plan_passes(plan, 8)
    r["tuned"] = dwt.dwt_plan_tuned(plan)
    # 32 such functions per call through the same tuned plan: one transform
    # fills less than one wave of the GPU, a batch fills several
    del x, y, z
    xb = torch.ones((32, ld), dtype=torch.float32, device=dev)
    yb = torch.empty((32, ld), dtype=torch.complex64, device=dev)

    def fwb():
        dwt.dwt_forward(plan, xb, yb, 32, ld, ld, dwt.DWT_F32, dwt.DWT_C64, stream=stream)

    ms, _ = timed(fwb, steps)
    r["forward_batch32_points_per_s"] = 32 * N * steps / (ms / 1e3)
    del xb, yb
    out["p3_m13_s8"] = r
    return out


def run_gpu(args):
    import numpy as np
    import torch

    import paper_0808_0487_gb300 as dwt
    import synthetic as S

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    dwt.lib()
    B = args.batch
    w = S.workload_p2_m24(batch=B)
    p, m, s = w["p"], w["m"], w["s"]
    N = p ** m
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    plan = dwt.dwt_plan_create(p, m, s, w["C"])
    plan_ms = (time.perf_counter() - t0) * 1e3

    f = torch.empty((B, N), dtype=torch.float32, device=dev)
    coef = torch.tensor(w["coef"], dtype=torch.float64, device=dev)
    dwt.dwt_eval_product(plan, coef, f, B, N, dwt.DWT_F32)
    c = torch.empty_like(f)
    var = torch.empty((B, 2, s + 1), dtype=torch.float64, device=dev)
    dim = torch.empty((B, 2), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    def step(st_=None):
        dwt.dwt_interpolate(plan, f, c, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER,
                            var=var, dim=dim, stream=stream if st_ is None else st_)

    region = {}

    def timed(fn, K):
        for _ in range(args.warmup):
            fn()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = dwt.dwt_launch_count()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        region["t"] = (t0, time.perf_counter())
        launches = dwt.dwt_launch_count() - l0
        if pg:
            pg.barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
        return ms, launches

    # The timed step replays a CUDA graph of one dwt_interpolate call: the call
    # only enqueues its launches (no host synchronisation, and no allocation
    # once an ordinary call has sized the plan's workspace), so it is captured
    # once and replayed; every replay runs all of its kernels.
    step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    l0 = dwt.dwt_launch_count()
    with torch.cuda.graph(graph):
        step(torch.cuda.current_stream())
    launches_per_step = dwt.dwt_launch_count() - l0
    torch.cuda.synchronize()

    def gstep():
        graph.replay()

    def pad(seconds):
        # untimed replays of the same step, so that the clock sampler also sees the
        # GPU under this load just before and after the (short) timed region
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            for _ in range(4):
                gstep()
            torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        pad(0.3)
        ms, _ = timed(gstep, args.steps)
        clk.mark(*region["t"])
        pad(0.3)
    launches = launches_per_step * args.steps
    clocks = clk.summary()
    value = whole_job_rate(B * N * args.steps, ws, ms)
    ms_direct, _ = timed(step, args.steps)   # the same step as ordinary calls

    # forward / inverse alone (extra context)
    def fwd():
        dwt.dwt_forward(plan, f, c, B, N, N, dwt.DWT_F32, dwt.DWT_F32, stream=stream)

    def inv():
        dwt.dwt_inverse(plan, c, c, B, N, N, dwt.DWT_F32, dwt.DWT_F32, stream=stream)

    ms_f, _ = timed(fwd, args.steps)
    ms_i, _ = timed(inv, args.steps)
    peak, peak_kind = _peaks()

    # the split-BF16 tensor-core forward (low 14 digits on tcgen05, the rest as
    # FP32 butterflies) against the FP32 butterfly forward: time and deviation
    c_tc = torch.empty_like(f)

    def fwd_tc():
        dwt.dwt_forward(plan, f, c_tc, B, N, N, dwt.DWT_F32, dwt.DWT_F32, algo=dwt.DWT_ALGO_TC_SPLIT_BF16,
                        stream=stream)

    ms_tc, _ = timed(fwd_tc, args.steps)

    def step_tc():
        dwt.dwt_interpolate(plan, f, c_tc, None, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER,
                            dwt.DWT_ALGO_TC_SPLIT_BF16, var=var, dim=dim, stream=stream)

    ms_tci, _ = timed(step_tc, args.steps)
    fwd()
    fwd_tc()
    torch.cuda.synchronize()
    tc_rel = float((torch.linalg.vector_norm((c_tc - c).double()) / torch.linalg.vector_norm(c.double())).item())
    tc_max = float(((c_tc - c).abs().max() / c.abs().max()).item())
    # outputs of function 0 of the timed workload for the comparison with the FP64
    # oracle in the CPU leg: FP32 forward, split-BF16 forward, FP32 round trip
    acc_in = {"fwd_f32": c[0].cpu().numpy().astype(np.float64), "fwd_tc": c_tc[0].cpu().numpy().astype(np.float64)}
    dwt.dwt_inverse(plan, c, c_tc, B, N, N, dwt.DWT_F32, dwt.DWT_F32, stream=stream)
    torch.cuda.synchronize()
    acc_in["round_trip_f32"] = c_tc[0].cpu().numpy().astype(np.float64)
    del c_tc
    # int32 forward (bit-exact path) of one p = 2, m = 20 function of the int32 workload
    w20 = S.workload_p2_m20()
    plan20 = dwt.dwt_plan_create(2, 20, w20["s"], w20["C"], dwt.DWT_PLAN_TRANSFORM_ONLY)
    vi = torch.from_numpy(S.int_values(w20["int_seed"], 1, 1 << 20)).to(dev)
    vo = torch.empty_like(vi)
    dwt.dwt_forward(plan20, vi, vo, 1, 1 << 20, 1 << 20, dwt.DWT_I32, dwt.DWT_I32, stream=stream)
    torch.cuda.synchronize()
    acc_in["fwd_i32_m20"] = vo[0].cpu().numpy().astype(np.int64)
    del vi, vo, plan20

    # per-kernel durations of the same step with events around every launch (on
    # the launching stream)
    dwt.dwt_profile_reset()
    dwt.dwt_profile_enable(True)
    ms_prof, _ = timed(step, args.steps)
    dwt.dwt_profile_enable(False)
    fams = {}
    for name in ("interp_fwd", "interp_top", "interp_inv", "interp_inv_fwd", "effdim_classes", "effdim_finalize"):
        n, tot = dwt.dwt_profile_query(name)
        if n:
            fams[name] = (n, tot)
    dom = max(fams, key=lambda k: fams[k][1]) if fams else None
    roof = roofline(dom, fams, N, B, peak, peak_kind) if dom else None
    dwt.dwt_profile_reset()

    # memory floor of the three-pass schedule on this GPU: the same traffic per
    # function with no arithmetic (torch copies: f_b -> an L2-sized buffer, the
    # buffer read and written in place, the buffer -> c_b), for comparison
    floor = memory_floor(f, c, B, N, stream, peak)

    # end to end: pinned host f -> device, the step, c and the variances back
    host_cpus = _bind_to_gpu_node(local)
    fh = torch.empty((B, N), dtype=torch.float32, pin_memory=True)
    fh.copy_(f)
    ch = torch.empty((B, N), dtype=torch.float32, pin_memory=True)
    vh = torch.empty((B, 2, s + 1), dtype=torch.float64, pin_memory=True)
    dh = torch.empty((B, 2), dtype=torch.int32, pin_memory=True)

    def e2e_step():
        # the public host-buffer call: chunked copies in and out overlapped with the transforms
        dwt.dwt_interpolate_host(plan, fh, ch, B, N, dwt.DWT_F32, dwt.DWT_WEIGHT_INV_SQ_WAVENUMBER, var=vh, dim=dh,
                                 stream=stream)

    K2 = max(1, min(args.steps, 5))
    ms_e2e, _ = timed(e2e_step, K2)
    e2e_value = B * N * K2 * ws / (ms_e2e / 1e3)

    others = run_other_configs(dwt, dev, stream, timed, args.steps) if not args.no_others else None

    # a bounded serving leg: the request mix of the serving workload (own nets,
    # plan build included), saturated and at 0.9 of the saturated rate
    serving = None
    if args.serve_requests > 0:
        del fh, ch
        torch.cuda.synchronize()
        runs = serve_runs(dwt, rank_requests(args.serve_requests, rank), args.slots, (0.9,))
        r9 = runs[-1]
        serving = {"requests": args.serve_requests, "slots": args.slots, "rate_req_s": r9["rate_req_s"],
                   "p50_ms": r9["p50_ms"], "p99_ms": r9["p99_ms"], "req_per_s": r9["req_per_s"],
                   "points_per_s": r9["points_per_s"], "plan_p50_ms": r9["plan_p50_ms"],
                   "plan_p99_ms": r9["plan_p99_ms"], "service_p99_ms": r9["service_p99_ms"],
                   "saturated": {k: runs[0][k] for k in ("req_per_s", "points_per_s", "plan_p50_ms", "plan_p99_ms")},
                   "latency": "submit to results on the host, queueing and plan build included"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_sample(acc_in)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "p2_m24_s32_b%d" % B, "p": p, "m": m, "s": s, "global_batch": B * ws,
                       "N": N, "weight": "prod_j (1+k_j)^-2", "l2": "inputs larger than L2 (2 GiB per rank)",
                       "parallelism": "replicas" if ws > 1 else "single", "host_cpus": host_cpus},
            "roofline": roof,
            "step_roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": peak_kind,
                              "bytes_per_point": 8 + 6.0 / B,
                              "achieved": B * N * (8 + 6.0 / B) * args.steps / (ms / 1e3) / 1e9,
                              "frac": B * N * (8 + 6.0 / B) * args.steps / (ms / 1e3) / 1e9 / peak},
            "memory_floor": floor,
            "accuracy_vs_oracle": cpu.get("accuracy_vs_oracle") if cpu else None,
            "serving": serving,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * N * 4,
                    "d2h_bytes_per_step": B * N * 4 + B * 2 * (s + 1) * 8 + B * 2 * 4},
            "gpu_launches": launches,
            "step_graph": {"launches_per_step": launches_per_step,
                           "direct_calls_ms_per_step": ms_direct / args.steps,
                           "direct_calls_points_per_s": whole_job_rate(B * N * args.steps, ws, ms_direct)},
            "clocks": clocks,
            "plan_build_ms": plan_ms,
            "forward_points_per_s": B * N * args.steps * ws / (ms_f / 1e3),
            "inverse_points_per_s": B * N * args.steps * ws / (ms_i / 1e3),
            "forward_hbm_frac": (B * N * args.steps * 8 / (ms_f / 1e3) / 1e9) / peak,
            "inverse_hbm_frac": (B * N * args.steps * 8 / (ms_i / 1e3) / 1e9) / peak,
            "forward_tc_points_per_s": B * N * args.steps * ws / (ms_tc / 1e3),
            "forward_tc_vs_butterfly": {"rel_l2": tc_rel, "max_abs_over_max": tc_max},
            "interpolate_tc_points_per_s": B * N * args.steps * ws / (ms_tci / 1e3),
            "step_hbm_frac_algorithmic": (B * N * args.steps * (8 + 6.0 / B) / (ms / 1e3) / 1e9) / peak,
            "kernel_ms": {k: v[1] / v[0] for k, v in fams.items()},
            "other_workloads": others,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()


def serve_runs(dwt, reqs, slots, fracs):
    """The serving mix: all arrivals at t = 0 (saturated rate R_sat), then Poisson
    arrivals at each fraction of R_sat.  Latency includes queueing and plan build."""
    import numpy as np

    import synthetic as S
    warm = S.serving_requests(16, first=10 ** 6)

    def run(rate, label):
        srv = dwt.dwt_server_create(0, slots=slots, max_queue=1 << 20)
        for r in warm:
            dwt.dwt_server_wait(srv, dwt.dwt_server_submit(srv, r["p"], r["m"], r["s"], r["C"], r["coef"]))
        t_arr = None if rate is None else S.poisson_arrivals(len(reqs), rate)
        t0 = time.perf_counter()
        tickets = []
        for i, r in enumerate(reqs):
            if t_arr is not None:
                dt = t0 + t_arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            tickets.append(dwt.dwt_server_submit(srv, r["p"], r["m"], r["s"], r["C"], r["coef"]))
        res = [dwt.dwt_server_wait(srv, t, 3600.0) for t in tickets]
        wall = time.perf_counter() - t0
        srv.close()
        bad = [(r["p"], r["m"], r["s"], x["status"], x["message"]) for r, x in zip(reqs, res) if x["status"]]
        assert not bad, bad[:8]
        lat = np.array([(x["t_done"] - x["t_submit"]) * 1e3 for x in res])
        svc = np.array([(x["t_done"] - x["t_admit"]) * 1e3 for x in res])
        plan = np.array([(x["t_plan"] - x["t_admit"]) * 1e3 for x in res])
        pts = float(sum(r["p"] ** r["m"] for r in reqs))
        # plan-build and service latency by net size (log2 N buckets)
        lg = np.array([r["m"] * np.log2(r["p"]) for r in reqs])
        by_size = []
        for lo, hi in ((10, 13), (13, 16), (16, 19), (19, 23)):
            sel = (lg >= lo - 0.01) & (lg < hi - 0.01)
            if sel.any():
                by_size.append({"log2N": [lo, hi], "requests": int(sel.sum()),
                                "plan_p50_ms": float(np.percentile(plan[sel], 50)),
                                "service_p50_ms": float(np.percentile(svc[sel], 50)),
                                "service_p99_ms": float(np.percentile(svc[sel], 99))})
        pr = np.array([r["p"] for r in reqs])
        by_p = [{"p": int(q), "requests": int((pr == q).sum()),
                 "plan_p50_ms": float(np.percentile(plan[pr == q], 50)),
                 "service_p50_ms": float(np.percentile(svc[pr == q], 50)),
                 "service_p99_ms": float(np.percentile(svc[pr == q], 99))} for q in sorted(set(pr.tolist()))]
        return {"label": label, "rate_req_s": rate, "wall_s": wall, "req_per_s": len(reqs) / wall, "by_size": by_size,
                "by_p": by_p,
                "points_per_s": pts / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "service_p50_ms": float(np.percentile(svc, 50)),
                "service_p99_ms": float(np.percentile(svc, 99)), "plan_p50_ms": float(np.percentile(plan, 50)),
                "plan_p99_ms": float(np.percentile(plan, 99))}

    sat = run(None, "saturated")
    runs = [sat]
    for frac in fracs:
        runs.append(run(frac * sat["req_per_s"], "poisson_%.1f" % frac))
    return runs


def run_serve(args):
    """The serving workload: requests with their own nets, Poisson arrivals, continuous batching."""
    import paper_0808_0487_gb300 as dwt

    ws, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    dwt.lib()
    reqs = rank_requests(args.requests, rank)
    runs = serve_runs(dwt, reqs, args.slots, (0.5, 0.9))
    if rank == 0:
        line = {"metric": "served p99 latency (ms), 10k-request mix p in {2,3,5}, N 2^10..2^22, s 2..64",
                "value": runs[-1]["p99_ms"], "unit": "ms", "n_gpus": ws, "higher_is_better": False,
                "requests": len(reqs), "slots": args.slots, "data": "synthetic", "dtype": "f32",
                "config": {"workload": "serving_mix", "requests": len(reqs)}, "runs": runs}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-others", action="store_true", help="skip the p = 2, m = 20 and p = 3, m = 13 lines")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the bounded serving leg of the default run (0: skip)")
    args = ap.parse_args()
    if args.serve:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
