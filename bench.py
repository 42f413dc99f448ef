"""Benchmark: exact Torontonians through libtor on GB300.

One step = one tor_eval_batch over a workload's matrices (intake, units,
reduce: every step of the hot path).  Workloads (seeded synthetic inputs):

  large_n30_34 (default)      lossy squeezed states n = 30 and 34 (r ~ U[0.3,0.8],
                              per-mode eta ~ U[0.3,0.7], Haar U); beside the timed
                              steps, one evaluation each of a lossy n = 38 state and
                              an n = 38 product state, the double-double factor on
                              the step's matrices, the error of every result against
                              the best available higher-precision reference, the
                              4096-matrix batch against the plain per-matrix path,
                              and the serving loop's p50/p99 against the plain path
  single_n16_20_24            lossy squeezed n = 16, 20, 24 plus a product state at n = 24
  single_n30 / single_n34 / single_n38   one lossy squeezed state of that size
  batch4096                   4096 click patterns k ~ U{4..24} of one 100-mode state
  serve                       chain-rule marginal requests on a 144-mode state (p50/p99)
  sample                      threshold-detector patterns drawn by tor_sample on a 40-mode state

Metric: subset terms per second (sum of 2^n over the step's matrices / time).
`value` times the device-resident path (inputs already on the GPU), `e2e` the
same call with host buffers (H2D of O and D2H of results inside the region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
       python bench.py --impl reference ...   (the CPU oracle, bounded sample)
"""
from __future__ import annotations

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

import numpy as np  # noqa: E402

from paper_2109_04528_gb300 import inputs  # noqa: E402

L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
FP64_PER_SM_CLK = 2  # GB300: FP64 thread instructions (add, mul, FMA) issued per SM per clock (ncu's peak)
MAX_SM_MHZ = 2070.0  # GB300 maximum SM clock, when the sampled clocks do not give it


DEFAULT_WORKLOAD = "large_n30_34"


def lossy(n: int, off: int = 0):
    """The lossy squeezed n-mode matrix of the single-matrix workloads.  Where the
    golden fixtures store the matrix of this recipe and seed (the input of a stored
    oracle sum), that stored matrix is used: the generator's linear algebra may
    round differently on another machine, and the stored sum is for these exact
    entries."""
    seed = inputs.SEED_BASE + 1000 + n + off
    try:
        with open(os.path.join(GOLDEN_DIR, f"lossy_n{n}.json")) as f:
            g = json.load(f)
        if g.get("seed") == seed and g.get("kind") == "lossy_squeezed" and g.get("n") == n:
            return np.array(g["O_re"]) + 1j * np.array(g["O_im"])
    except (OSError, ValueError):
        pass
    return inputs.config_single(n, seed=seed).O


def workload(name: str, rank: int = 0):
    """(list of O matrices, description)."""
    off = 7919 * rank
    if name == "large_n30_34":
        mats = [lossy(n, off) for n in (30, 34)]
        return mats, "lossy squeezed n=30,34 (r~U[0.3,0.8], eta_j~U[0.3,0.7], Haar U)"
    if name == "single_n16_20_24":
        mats = [lossy(n, off) for n in (16, 20, 24)]
        mats.append(inputs.product_state(24, inputs.SEED_BASE + 2024 + off).O)
        return mats, "lossy squeezed n=16,20,24 (r~U[0.3,0.8], eta_j~U[0.3,0.7]) + product state n=24"
    if name.startswith("single_n"):
        n = int(name[len("single_n"):])
        return [lossy(n, off)], f"lossy squeezed n={n} (r~U[0.3,0.8], eta_j~U[0.3,0.7])"
    if name == "batch4096":
        _, _, mats = inputs.click_pattern_batch(100, 4096, 4, 24, inputs.SEED_BASE + 3 + off, (0.5, 1.2), 0.4)
        return mats, "4096 submatrices of a 100-mode lossy squeezed state (r~U[0.5,1.2], eta=0.4), k~U{4..24}"
    raise SystemExit(f"unknown workload {name}")


KERNEL_SOURCES = ("tor_device.cuh", "tor_dd.cuh", "tor_internal.h", "tor_kernels.cu")


def kernel_hash() -> str:
    """Hash of the device code (the kernels and the structures they read); the
    host runtime and the allocation-free entry point are not part of it."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2109_04528_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_name: str, kernel: str = "k_units", prefix_depth=None):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, if it
    was taken of that kernel on this workload, on the kernel sources as they are
    now and with the same prefix depths (the launch's task decomposition)."""
    try:
        with open(os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("workload") != workload_name or t.get("kernel") != kernel or t.get("kernel_hash") != kernel_hash():
        return None
    if prefix_depth is not None and t.get("prefix_depth") != prefix_depth:
        return None
    return t.get("dram_bytes_per_launch")


def algorithmic_flops(n: int, path: int = 0) -> float:
    """FP64 flops of the rank-2 subset-tree walk over all 2^n subsets in the
    arithmetic the matrix took (tor_result.path).  FP64 complex path:
    F(n) = sum_j 2^j (32 m_j^2 + 40 m_j + 10) + 10 2^n, m_j = n-1-j (complex
    MAC = 8 flops, complex x real = 2, sqrt/rsqrt/div = 1); real (x, p) path
    F_real(n) = sum_j 2^j (8 m_j^2 + 12 m_j + 10) + 10 2^n; the double-double
    paths count every FP64 operation of the double-word algorithms
    (paper_2109_04528_gb300.flops.path_flops)."""
    from paper_2109_04528_gb300.flops import path_flops
    return path_flops(n, path)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        time.sleep(0.15)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def spread_sample(n: int, count: int):
    """(stride, count) of a sample of the 2^n subset masks, k * stride for k < count, spread over
    the whole range with an odd stride, so that it has the subset-size mix of the full sum (the
    first masks alone hold only the low modes: small, cheap determinants)."""
    count = max(1, min(int(count), 1 << n))
    if count >= (1 << n) or count == 1:
        return 1, count
    stride = ((1 << n) - 1) // (count - 1)
    stride -= 1 - stride % 2
    return max(stride, 1), count


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def timed_oracle(O, cores: int, count: int):
    import oracle
    n = O.shape[0] // 2
    stride, count = spread_sample(n, count)
    t0 = time.perf_counter()
    oracle.tor_brute(O, threads=cores, stride=stride, count=count)
    return time.perf_counter() - t0, stride, count


def cpu_baseline(mats, budget_s: float):
    """The oracle (binary128 brute force) on a bounded sample of the workload's
    largest matrix -- subsets spread over all 2^n masks -- on all host cores."""
    import oracle
    oracle.build()
    O = max(mats, key=lambda a: a.shape[0])
    n = O.shape[0] // 2
    cores = os.cpu_count() or 1
    count = 1 << min(n, 10)
    dt, _, count = timed_oracle(O, cores, count)
    while dt < 0.5 and count < (1 << n):  # calibrate
        dt, _, count = timed_oracle(O, cores, min(1 << n, count * 4))
    count = int(min(1 << n, max(count, count * budget_s / max(dt, 1e-3))))
    dt, stride, count = timed_oracle(O, cores, count)
    return {"value": count / dt, "unit": "subset terms/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
            "sample": f"{count} of the 2^{n} subsets of the n={n} matrix (masks k*{stride}, spread over all), "
                      f"binary128 LU per subset, {dt:.1f} s"}


def golden_for(O):
    """The stored binary128 oracle sum of exactly this matrix, if the golden
    fixtures hold one (written by the oracle alone): dict(hi, lo, abs_sum,
    method) or None."""
    n = O.shape[0] // 2
    try:
        with open(os.path.join(GOLDEN_DIR, f"lossy_n{n}.json")) as f:
            g = json.load(f)
    except (OSError, ValueError):
        return None
    G = np.array(g["O_re"]) + 1j * np.array(g["O_im"])
    if G.shape != O.shape or not np.array_equal(G, O):
        return None
    return {"hi": g["tor_hi"], "lo": g["tor_lo"], "abs_sum": g["abs_sum"],
            "method": g.get("method", "brute force")}


def product_closed_form(inst):
    """Tor and sum|term| of a product state in closed form (Eq. tor factorises
    over modes): prod_j (x_j - 1) and prod_j (x_j + 1), x_j = sqrt(det Sigma_j)
    of mode j's lossy squeezed vacuum (N = eta sinh^2 r, M = eta sinh r cosh r);
    x - 1 is formed as (2N + N^2 - M^2) / (x + 1), without cancellation."""
    import math
    sh, ch = np.sinh(inst.r), np.cosh(inst.r)
    N = inst.eta * sh * sh
    M = inst.eta * sh * ch
    x = np.sqrt((1 + N) ** 2 - M ** 2)
    xm1 = (2 * N + N * N - M * M) / (x + 1)
    return math.prod(float(v) for v in xm1), math.prod(float(v) for v in x + 1)


def error_entry(r, ref_hi: float, ref_lo: float):
    """|Tor - ref| of one result, against sum|term| and against |ref|."""
    d = abs((r.hi - ref_hi) + (r.lo - ref_lo))
    ref = ref_hi + ref_lo
    return {"abs_err": d, "err_over_abs_sum": d / r.abs_sum if r.abs_sum else None,
            "rel_err": d / abs(ref) if ref else None, "within_err_est": bool(d <= r.err_est)}


def result_record(name: str, n: int, r64, rx=None, ref=None):
    """One matrix's results and their errors.  ref = dict(hi, lo, name[, bound]):
    the binary128 oracle, a closed form, or the double-double GPU path (whose own
    a-priori bound is `bound`)."""
    rec = {"matrix": name, "n": n, "abs_sum": r64.abs_sum, "path": r64.path,
           "fp64": {"tor": r64.tor, "err_est": r64.err_est}}
    if rx is not None:
        rec["extended"] = {"tor": rx.tor, "err_est": rx.err_est}
    if ref is None:
        rec["ref"] = None
        return rec
    tref = ref["hi"] + ref["lo"]
    rec["ref"] = ref["name"]
    rec["tor_ref"] = tref
    if ref.get("bound") is not None:
        rec["ref_err_bound"] = ref["bound"]
    rec["kappa"] = r64.abs_sum / abs(tref) if tref else None
    rec["fp64"].update(error_entry(r64, ref["hi"], ref["lo"]))
    if rx is not None and ref["name"] != "double-double GPU path":
        rec["extended"].update(error_entry(rx, ref["hi"], ref["lo"]))
    return rec


def large_extras(local, stream, ctx_dev, mats, dmats, res64, ns, peak_ops: float):
    """Beside the timed steps of the n = 30/34 workload: the double-double factor
    on each step matrix, one evaluation each of a lossy and a product state at
    n = 38, sampled oracle units at n = 34, and the error of every result."""
    import torch

    import oracle
    from paper_2109_04528_gb300 import binding
    from paper_2109_04528_gb300.flops import path_ops
    device = torch.device("cuda", local)
    out = {"results": [], "extended": [], "n38": []}
    # double-double factor (TOR_EXTENDED) on the step's matrices, one timed evaluation each
    rxs = []
    with binding.Context(device=local, stream=stream.cuda_stream,
                         flags=binding.TOR_IN_DEVICE | binding.TOR_EXTENDED) as cx:
        binding.tor_eval(cx, torch.from_numpy(inputs.config_n8().O).to(device))  # module load, allocation
        for d, n in zip(dmats, ns):
            rx = binding.tor_eval(cx, d)
            ms = cx.last_times()["total_ms"]
            rxs.append(rx)
            out["extended"].append({"n": n, "ms": ms, "terms_per_s": 2.0 ** n / (ms * 1e-3), "path": rx.path,
                                    "status": rx.status, "prefix_depth": cx.plan_prefix_depth(n),
                                    "fp64_instructions_frac": path_ops(n, rx.path) / (ms * 1e-3) / peak_ops})
        # where no oracle sum exists, the double-double result is evaluated a second time on the
        # matrix with its modes in reverse order: Tor does not change under a relabelling of the
        # modes (Sec. 2), but every subset's factorisation pivots in another order, so its
        # rounding is independent of the first; the two agree to about the path's actual error
        second = {}
        for i, (O, n) in enumerate(zip(mats, ns)):
            if golden_for(O) is not None:
                continue
            rev = torch.from_numpy(inputs.permute_modes(O, list(range(n))[::-1])).to(device)
            r2 = binding.tor_eval(cx, rev)
            del rev
            d = abs((r2.hi - rxs[i].hi) + (r2.lo - rxs[i].lo))
            second[i] = {"modes": "reversed", "tor": r2.tor, "abs_diff": d, "diff_over_abs_sum": d / r2.abs_sum,
                         "rel_diff": d / abs(rxs[i].tor) if rxs[i].tor else None}
    for i, (O, n) in enumerate(zip(mats, ns)):
        g = golden_for(O)
        if g is not None:
            ref = {"hi": g["hi"], "lo": g["lo"], "name": f"binary128 oracle ({g['method']}), stored"}
        else:
            ref = {"hi": rxs[i].hi, "lo": rxs[i].lo, "name": "double-double GPU path", "bound": rxs[i].err_est}
        rec = result_record(f"lossy n={n} (timed step)", n, res64[i], rxs[i], ref)
        if i in second:
            rec["extended"]["second_evaluation"] = second[i]
        out["results"].append(rec)
    # a more strongly squeezed n = 30 state, whose terms cancel less: there the FP64 result keeps
    # digits, measured against the double-double path (not a benchmark configuration; a contrast)
    hs = inputs.lossy_squeezed(30, inputs.SEED_BASE + 3030, (1.0, 1.5), 0.7)
    d = torch.from_numpy(hs.O).to(device)
    r64 = binding.tor_eval(ctx_dev, d)
    with binding.Context(device=local, stream=stream.cuda_stream,
                         flags=binding.TOR_IN_DEVICE | binding.TOR_EXTENDED) as cx:
        rx = binding.tor_eval(cx, d)
    rec = result_record("lossy n=30, r~U[1.0,1.5], eta=0.7 (contrast)", 30, r64, rx,
                        {"hi": rx.hi, "lo": rx.lo, "name": "double-double GPU path", "bound": rx.err_est})
    out["results"].append(rec)
    del d
    # n = 38: a lossy squeezed state and a product state with a closed form, one evaluation each
    lossy38 = inputs.config_single(38, seed=inputs.SEED_BASE + 1038)
    prod38 = inputs.product_state(38, inputs.SEED_BASE + 2038)
    parts38 = None
    for name, inst in (("lossy n=38", lossy38), ("product state n=38", prod38)):
        d = torch.from_numpy(inst.O).to(device)
        if inst is lossy38:  # the same launch, with the unit partials copied back for the sampled check
            r, p38, parts38 = binding.tor_eval_units(ctx_dev, d)
        else:
            r = binding.tor_eval(ctx_dev, d)
        ms = ctx_dev.last_times()["total_ms"]
        out["n38"].append({"matrix": name, "ms": ms, "terms_per_s": 2.0 ** 38 / (ms * 1e-3), "status": r.status,
                           "path": r.path, "prefix_depth": ctx_dev.plan_prefix_depth(38)})
        ref = None
        if inst.kind == "product_state":
            t, a = product_closed_form(inst)
            ref = {"hi": t, "lo": 0.0, "name": "closed form prod_j (x_j - 1)"}
            out["n38"][-1]["abs_sum_closed_form"] = a
            out["n38"][-1]["abs_sum_rel_err"] = abs(r.abs_sum - a) / a
        rec = result_record(name, 38, r, None, ref)
        if ref is None:
            rec["note"] = ("no higher-precision reference within the bench's budget (the double-double path "
                           "would take ~150 s, the binary128 oracle years); second_evaluation: the same FP64 "
                           "walk on the matrix with its modes reversed (Tor is invariant, the rounding of every "
                           "term independent), whose difference shows the FP64 result's actual error")
            rev = torch.from_numpy(inputs.permute_modes(inst.O, list(range(38))[::-1])).to(device)
            r2 = binding.tor_eval(ctx_dev, rev)
            del rev
            dd = abs((r2.hi - r.hi) + (r2.lo - r.lo))
            rec["fp64"]["second_evaluation"] = {"modes": "reversed", "tor": r2.tor, "abs_diff": dd,
                                                "diff_over_abs_sum": dd / r2.abs_sum,
                                                "rel_diff": dd / abs(r.tor) if r.tor else None}
        out["results"].append(rec)
        del d
    # sampled prefix units of the n = 34 step matrix against the binary128 oracle (same launch plan)
    j = ns.index(34) if 34 in ns else len(ns) - 1
    res, p, parts = binding.tor_eval_units(ctx_dev, dmats[j])
    oracle.build()
    checks = []
    t0 = time.perf_counter()
    for u in (0, 0b1011, 0b1010010001):
        q = oracle.tor_unit(mats[j], p, u)
        d = abs((parts[u][0] - q.hi) + (parts[u][1] - q.lo))
        checks.append({"u": u, "abs_err": d, "err_over_abs_sum": d / q.abs_sum, "pass_1e-10": bool(d <= 1e-10 * q.abs_sum)})
    out["units_parity"] = {"n": ns[j], "p": p, "subsets_per_unit": 1 << (ns[j] - p), "units": checks,
                           "oracle_s": time.perf_counter() - t0,
                           "what": "GPU unit partials (tor_eval_units, the timed launch plan) against the "
                                   "binary128 brute force of the same units"}
    # the lossy n = 38 evaluation's own units: two with few prefix modes included (their subsets
    # are small, so the oracle's 2^18 determinants per unit take seconds)
    if parts38 is not None:
        checks = []
        t0 = time.perf_counter()
        for u in (0, (1 << 3) | (1 << 17)):
            q = oracle.tor_unit(lossy38.O, p38, u)
            d = abs((parts38[u][0] - q.hi) + (parts38[u][1] - q.lo))
            checks.append({"u": u, "abs_err": d, "err_over_abs_sum": d / q.abs_sum,
                           "pass_1e-10": bool(d <= 1e-10 * q.abs_sum)})
        out["units_parity_n38"] = {"n": 38, "p": p38, "subsets_per_unit": 1 << (38 - p38), "units": checks,
                                   "oracle_s": time.perf_counter() - t0,
                                   "what": "unit partials of the timed lossy n = 38 evaluation against the "
                                           "binary128 brute force of the same units"}
    return out


def small_batch(local, stream, count: int = 65536, k: int = 8, steps: int = 5):
    """Many small Torontonians (the small-n regime of the paper's benchmark, where
    calls, not terms, bound the rate): count k-click patterns of the 100-mode
    state of the batch workload, as one stacked device tensor with record results
    (tor_eval_batch_arrays), beside the same matrices as a list of tensors."""
    import torch

    from paper_2109_04528_gb300 import binding
    device = torch.device("cuda", local)
    base = inputs.lossy_squeezed(100, inputs.SEED_BASE + 4, (0.5, 1.2), 0.4).O
    rng = inputs.rng_for(inputs.SEED_BASE + 45)
    idx = np.sort(np.argsort(rng.random((count, 100)), axis=1)[:, :k], axis=1)
    rows = np.concatenate([idx, idx + 100], axis=1)  # block layout: a_j and a_j^dag of each mode
    stack = torch.from_numpy(base[rows[:, :, None], rows[:, None, :]]).to(device)
    out = {"count": count, "k": k, "terms_per_call": float(count) * 2.0 ** k,
           "desc": f"{count} random {k}-mode submatrices of the 100-mode state (r~U[0.5,1.2], eta=0.4)"}
    with binding.Context(device=local, stream=stream.cuda_stream, flags=binding.TOR_IN_DEVICE) as c:
        for name, src, fn in (("stacked_records", stack, binding.tor_eval_batch_arrays),
                              ("list_of_tensors", [stack[i] for i in range(count)], binding.tor_eval_batch)):
            fn(c, src)
            torch.cuda.synchronize()
            ts = []
            for _ in range(steps):
                t0 = time.perf_counter()
                fn(c, src)
                ts.append(time.perf_counter() - t0)
            wall = statistics.median(ts)
            out[name] = {"wall_ms": 1e3 * wall, "tor_per_s": count / wall, "device_ms": c.last_times()["total_ms"]}
        # the plan tuned for this batch (small matrices alone fill the GPU with larger units)
        p0 = c.plan_prefix_depth(k)
        binding.tor_autotune_batch(c, stack, 3.0)
        binding.tor_eval_batch_arrays(c, stack)
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            binding.tor_eval_batch_arrays(c, stack)
            ts.append(time.perf_counter() - t0)
        wall = statistics.median(ts)
        out["stacked_records_autotuned"] = {"wall_ms": 1e3 * wall, "tor_per_s": count / wall,
                                            "device_ms": c.last_times()["total_ms"],
                                            "prefix_depth": [p0, c.plan_prefix_depth(k)]}
    out["what"] = "host wall time of the call (marshalling, launches, device, results), median of 5"
    return out


def batch_compare(local, stream, steps: int, tune_s: float = 15.0):
    """The 4096-matrix batch (k ~ U{4..24} click patterns of a 100-mode state):
    one batched launch, its CUDA-graph replay, and the plain path (one tor_eval
    per matrix, looped in C by tor_eval_seq), all device-resident."""
    import torch

    from paper_2109_04528_gb300 import binding
    device = torch.device("cuda", local)
    mats, desc = workload("batch4096")
    dmats = [torch.from_numpy(m).to(device) for m in mats]
    terms = float(sum(2.0 ** (m.shape[0] // 2) for m in mats))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def run(ctx, k):
        ms = []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = binding.tor_eval_batch(ctx, dmats)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if any(r.status != 0 for r in res):
                raise SystemExit("batch evaluation failed")
        return ms, res

    out = {"workload": "batch4096", "desc": desc, "matrices": len(mats), "terms_per_batch": terms}
    with binding.Context(device=local, stream=stream.cuda_stream, flags=binding.TOR_IN_DEVICE) as c:
        run(c, 2)
        ms, res_b = run(c, steps)
        out["batched"] = {"ms_per_batch": statistics.median(ms), "value": terms / (statistics.median(ms) * 1e-3),
                          "unit": "subset terms/s", "steps": steps, "tor_per_s": len(mats) / (statistics.median(ms) * 1e-3)}
    with binding.Context(device=local, stream=stream.cuda_stream,
                         flags=binding.TOR_IN_DEVICE | binding.TOR_GRAPHS) as c:
        run(c, 2)
        ms, res_g = run(c, steps)
        out["graph_replay"] = {"ms_per_batch": statistics.median(ms), "value": terms / (statistics.median(ms) * 1e-3),
                               "unit": "subset terms/s", "steps": steps}
    # the batch autotuner: prefix depths tuned for this batch's throughput (a bounded budget)
    with binding.Context(device=local, stream=stream.cuda_stream, flags=binding.TOR_IN_DEVICE) as c:
        t0 = time.perf_counter()
        plan = binding.tor_autotune_batch(c, dmats, tune_s)
        tune_took = time.perf_counter() - t0
        run(c, 1)
        ms, _ = run(c, steps)
        builtin = {}
        with binding.Context(device=local, flags=binding.TOR_IN_DEVICE) as c0:
            builtin = {n: c0.plan_prefix_depth(n) for n in sorted(plan)}
        out["batched_autotuned"] = {"ms_per_batch": statistics.median(ms), "value": terms / (statistics.median(ms) * 1e-3),
                                    "unit": "subset terms/s", "steps": steps, "tune_s": tune_took,
                                    "changed_depths": {str(n): [builtin[n], p] for n, p in sorted(plan.items())
                                                       if p != builtin[n]},
                                    "what": "tor_autotune_batch (coordinate descent over the sizes' prefix depths, "
                                            "timing the whole batch), then the same timed batch"}
    with binding.Context(device=local, stream=stream.cuda_stream, flags=binding.TOR_IN_DEVICE) as c:
        binding.tor_eval_seq(c, dmats[:64])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_p, lat = binding.tor_eval_seq(c, dmats)
        plain_s = time.perf_counter() - t0
    lat = np.sort(lat)
    out["plain_per_matrix"] = {"s_per_batch": plain_s, "value": terms / plain_s, "unit": "subset terms/s",
                               "tor_per_s": len(mats) / plain_s, "per_matrix_ms_p50": float(lat[len(lat) // 2]),
                               "per_matrix_ms_p99": float(lat[min(len(lat) - 1, int(0.99 * len(lat)))]),
                               "what": "tor_eval_seq: one tor_eval per matrix (descriptors H2D, 3 kernels, results "
                                       "D2H, one sync) looped in C, host wall time"}
    same = all((a.hi, a.lo, a.abs_sum) == (b.hi, b.lo, b.abs_sum) == (g.hi, g.lo, g.abs_sum)
               for a, b, g in zip(res_b, res_p, res_g))
    out["bitwise_equal_batched_graph_plain"] = bool(same)
    out["batched_over_plain"] = out["batched"]["value"] / out["plain_per_matrix"]["value"]
    out["graph_over_plain"] = out["graph_replay"]["value"] / out["plain_per_matrix"]["value"]
    out["autotuned_over_builtin"] = out["batched_autotuned"]["value"] / out["batched"]["value"]
    return out


def sharded_step(binding, ctx, batch, ns, world: int, rank: int):
    """One step split over the ranks (paper Sec. 4): this rank evaluates its
    aligned leaf range of every matrix in one launch (tor_eval_range_batch), the
    ranks gather three doubles per matrix, and every rank merges them with the
    fixed tree, which reproduces one GPU's result bitwise.  Returns (merged
    results, this rank's units-kernel ms)."""
    from paper_2109_04528_gb300 import shard
    ranges = [shard.shard_range(binding.tor_plan_leaves(ctx, n), world, rank) for n in ns]
    res = binding.tor_eval_range_batch(ctx, batch, ranges)
    units = ctx.last_times()["units_ms"]
    got = shard._gather_checked(lambda: [(r.hi, r.lo, r.abs_sum) for r in res])
    merged = [shard.tree_merge([g[i] for g in got]) for i in range(len(batch))]
    for r, m in zip(res, merged):
        r.hi, r.lo, r.abs_sum = m
    return res, units


def sharded_depths(ctx, ns, world: int):
    """Prefix depth per size for a matrix split over `world` ranks: the context's
    plan deepened by log2(world) - 1 levels (none for two ranks), so that each
    rank's share of a matrix keeps about as many warp tasks per SM as one GPU's
    whole matrix, up to the limit of 30 and n - 1.  Every rank and the one-GPU
    check use the same depths, so the merge stays bitwise equal to one GPU."""
    deeper = max(0, world.bit_length() - 2)
    return {n: min(30, n - 1, ctx.plan_prefix_depth(n) + deeper) for n in sorted(set(ns))}


def launches_per_step(ctx, ns) -> int:
    """Kernels one tor_eval_batch launches: k_intake, k_units, k_reduce, and
    k_reduce_chunks when a matrix has more than 256 reduction leaves (2^(p-5)
    task partials for p >= 5, 2^p unit partials below)."""
    big = any((p - 5 if p >= 5 else p) > 8 for p in (ctx.plan_prefix_depth(n) for n in ns))
    return 3 + (1 if big else 0)


def cpu_alg2(mats, budget_s: float):
    """The paper's own method on the host cores: Algorithm 2 in FP64 with a
    thread pool over subtrees (oracle/tor_alg2_cpu.c), on the workload's
    largest matrix -- the whole sum if it fits the budget, else its largest
    subtrees first."""
    from oracle import alg2_cpu
    alg2_cpu.build()
    O = max(mats, key=lambda a: a.shape[0])
    n = O.shape[0] // 2
    cores = os.cpu_count() or 1
    k = cores
    while True:
        t0 = time.perf_counter()
        r = alg2_cpu.tor_alg2(O, threads=cores, max_tasks=k)
        dt = time.perf_counter() - t0
        if r.terms >= (1 << n) or dt >= 0.25 * budget_s:
            break
        k *= 4
    if r.terms < (1 << n) and (1 << n) / (r.terms / max(dt, 1e-6)) <= budget_s:
        t0 = time.perf_counter()
        r = alg2_cpu.tor_alg2(O, threads=cores)
        dt = time.perf_counter() - t0
    what = "all" if r.terms >= (1 << n) else f"{r.terms} (largest subtrees first)"
    return {"value": r.terms / dt, "unit": "subset terms/s", "cores": cores, "cpu": cpu_model(),
            "kind": "paper Algorithm 2 (remove-mode recursion, Cholesky block reuse), FP64, threads over subtrees",
            "sample": f"{what} of the 2^{n} terms of the n={n} matrix, {dt:.2f} s"}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    mats, desc = workload(args.workload)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    O = max(mats, key=lambda a: a.shape[0])
    n = O.shape[0] // 2
    # size one step to ~2 s of CPU work, subsets spread over all 2^n masks
    dt, _, count = timed_oracle(O, cores, 1 << min(n, 8))
    count = int(min(1 << n, max(count, count * 2.0 / max(dt, 1e-3))))
    for _ in range(args.warmup):
        timed_oracle(O, cores, count)
    times = []
    for _ in range(args.steps):
        dt, stride, count = timed_oracle(O, cores, count)
        times.append(dt)
    tot = sum(times)
    value = count * args.steps / tot
    line = {"impl": "reference", "metric": "subset terms/s", "value": value, "unit": "subset terms/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f128",
            "data": "synthetic", "config": {"workload": args.workload, "desc": desc},
            "cpu_baseline": {"value": value, "unit": "subset terms/s", "cores": cores, "cpu": cpu_model(),
                             "kind": "oracle",
                             "sample": f"each step: {count} of the 2^{n} subsets of the n={n} matrix "
                                       f"(masks k*{stride}, spread over all)"},
            "e2e": {"value": value, "unit": "subset terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serve_requests(rate: float, window: float, seed: int, N: int = 144):
    """Seeded Poisson arrivals of chain-rule marginal requests on an N-mode state:
    k ~ U{2..30}, j ~ U{max(k,1)..N}, S = a k-subset of modes 0..j-1 that
    contains mode j-1 (the mode the chain rule is adding)."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > window:
            break
        k = int(rng.integers(2, 31))
        j = int(rng.integers(max(k, 1), N + 1))
        rest = rng.choice(j - 1, size=k - 1, replace=False) if k > 1 else np.zeros(0, dtype=int)
        S = sorted([j - 1] + [int(x) for x in rest])
        reqs.append((t, j, S))
    return reqs


def replay(ctx, sess, reqs, mode: str, drain_s: float):
    """Submits reqs at their scheduled times; returns latencies (s) of the
    requests completed by window end + drain_s, and counts.  mode 'served' =
    tor_submit_marginal, completions collected as they happen (tor_poll_any);
    'plain' = one blocking tor_eval_marginal at a time in arrival order."""
    from paper_2109_04528_gb300 import binding
    window = reqs[-1][0] if reqs else 0.0
    deadline = window + drain_s
    lat, terms_done = [], 0.0
    t0 = time.perf_counter()
    if mode == "plain":
        for (ta, j, S) in reqs:
            now = time.perf_counter() - t0
            if now > deadline:
                break
            if now < ta:
                time.sleep(ta - now)
            binding.tor_eval_marginal(ctx, sess, j, S)
            lat.append(time.perf_counter() - t0 - ta)
            terms_done += 2.0 ** len(S)
        return lat, len(lat), terms_done
    tickets, meta = [], []
    i = 0
    while True:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            ta, j, S = reqs[i]
            tickets.append(binding.tor_submit_marginal(ctx, sess, j, S))
            meta.append((ta, len(S)))
            i += 1
        if (i >= len(reqs) and not tickets) or now > deadline:
            break
        wait = (reqs[i][0] - now) if i < len(reqs) else deadline - now
        wait = max(0.0, min(wait, 0.05))
        if not tickets:
            time.sleep(wait)
            continue
        # poll without sleeping (the plain path's blocking call spins in cudaStreamSynchronize too)
        st, k, r = binding.tor_poll_any(ctx, tickets, 0.0)
        if k < 0:
            continue
        done_at = time.perf_counter() - t0
        ta, kk = meta[k]
        tickets.pop(k)
        meta.pop(k)
        if st == 0:
            lat.append(done_at - ta)
            terms_done += 2.0 ** kk
    return lat, len(lat), terms_done


def _pct(x, q):
    if not x:
        return None
    x = sorted(x)
    return x[min(len(x) - 1, int(q * len(x)))]


def serve_runs(local, loads, seed: int):
    """Replays seeded Poisson streams of chain-rule marginal requests on the
    144-mode state (r ~ U[0.5,1.2], eta = 0.3) through the serving loop and
    through the plain blocking path.  loads: list of (name, rate or callable of
    the runs so far, window_s, modes, drain_s)."""
    from paper_2109_04528_gb300 import binding
    inst = inputs.lossy_squeezed(144, inputs.SEED_BASE + 5, (0.5, 1.2), 0.3)
    runs = {}
    for name, rate, window, modes, drain in loads:
        if callable(rate):
            rate = rate(runs)
        reqs = serve_requests(rate, window, seed)
        for mode in modes:
            ctx = binding.Context(device=local)
            sess = binding.Session(ctx, inst.sigma)
            binding.tor_eval_marginal(ctx, sess, 10, [0, 3, 9])  # warm-up
            t0 = time.perf_counter()
            lat, done, terms = replay(ctx, sess, reqs, mode, drain_s=drain)
            el = time.perf_counter() - t0
            stats = ctx.serving_stats()
            ctx.close()  # drops the backlog, stops running jobs, waits for the GPU
            sess.close()
            runs[f"{name}_{mode}"] = {
                "offered_rate": rate, "window_s": window, "offered": len(reqs), "completed": done,
                "requests_per_s": done / el, "terms_per_s": terms / el,
                "p50_ms": None if not lat else 1e3 * _pct(lat, 0.5), "p99_ms": None if not lat else 1e3 * _pct(lat, 0.99),
                "backlog_at_end": len(reqs) - done, "batches": stats["batches"]}
    return runs


def capacity_rate(runs, frac: float = 0.8):
    """Requests/s at `frac` of the capacity measured under overload.  Under
    overload small requests pass large ones and the backlog is dropped, so the
    completion rate overstates capacity; capacity is the subset terms/s the GPU
    sustained there over the mean request, E[2^k] = (2^31 - 4) / 29."""
    mean_terms = (2.0 ** 31 - 4.0) / 29.0
    return round(frac * runs["overload_served"]["terms_per_s"] / mean_terms, 1)


def run_serve(args, world, rank, local):
    """Serving benchmark on a 144-mode lossy squeezed state (r ~ U[0.5,1.2], eta = 0.3)."""
    if rank != 0:
        return 0
    from paper_2109_04528_gb300 import build
    build.build()
    high = args.serve_high_rate if args.serve_high_rate > 0 else capacity_rate
    runs = serve_runs(local, [("overload", args.serve_rate, args.serve_window, ("served", "plain"), 2.0),
                              ("sustained", args.serve_sustain_rate, args.serve_sustain_window, ("served", "plain"), 30.0),
                              ("high", high, args.serve_high_window, ("served", "plain"), 30.0)],
                      inputs.SEED_BASE + 17)
    out = {"metric": "requests/s", "unit": "requests/s", "n_gpus": 1, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "serve", "state": "144-mode lossy squeezed, r~U[0.5,1.2], eta=0.3",
                      "request": "k~U{2..30}, j~U{max(k,1)..144}, S a k-subset of [j] containing j-1",
                      "latency": "completion minus scheduled arrival"}}
    out["runs"] = runs
    s = runs["high_served"]
    out["value"] = s["requests_per_s"]
    out["p50_ms"], out["p99_ms"] = s["p50_ms"], s["p99_ms"]
    out["plain_p50_ms"], out["plain_p99_ms"] = runs["high_plain"]["p50_ms"], runs["high_plain"]["p99_ms"]
    out["config"]["high_rate"] = runs["high_served"]["offered_rate"]
    print(json.dumps(out), flush=True)
    return 0


def serve_summary(local, window: float, light_rate: float):
    """The serving loop against the plain path at ~80 % of capacity and at a
    light load, for the headline line."""
    runs = serve_runs(local, [("overload", 2000.0, 2.0, ("served",), 2.0),
                              ("high", capacity_rate, window, ("served", "plain"), 30.0),
                              ("light", light_rate, window, ("served", "plain"), 30.0)],
                      inputs.SEED_BASE + 17)
    out = {"state": "144-mode lossy squeezed, r~U[0.5,1.2], eta=0.3",
           "request": "chain-rule marginal Tor(O^(j)_S), k=|S|~U{2..30}, Poisson arrivals",
           "latency": "completion minus scheduled arrival", "runs": runs}
    for load in ("high", "light"):
        a, b = runs[f"{load}_served"], runs[f"{load}_plain"]
        out[load] = {"rate": a["offered_rate"], "served_p50_ms": a["p50_ms"], "served_p99_ms": a["p99_ms"],
                     "plain_p50_ms": b["p50_ms"], "plain_p99_ms": b["p99_ms"],
                     "served_requests_per_s": a["requests_per_s"], "plain_requests_per_s": b["requests_per_s"]}
    return out


def sample_work(pat):
    """(subset terms, Torontonians) that tor_sample evaluates for the drawn patterns:
    at step j, the two continuations of every distinct click set S among the
    samples' first j modes, 2^|S| + 2^(|S|+1) terms."""
    count, n = pat.shape
    terms, evals = 0.0, 0
    for j in range(n):
        distinct = {tuple(np.flatnonzero(row[:j])) for row in pat}
        evals += 2 * len(distinct)
        terms += sum(3.0 * 2.0 ** len(S) for S in distinct)
    return terms, evals


def run_sample(args, world, rank, local):
    """Chain-rule threshold-detector sampling (tor_sample) on a 40-mode lossy
    squeezed state (r ~ U[0.5,1.2], eta = 0.5; ~14 clicks per pattern on average)."""
    if rank != 0:
        return 0
    from paper_2109_04528_gb300 import binding, build
    build.build()
    n = 40
    inst = inputs.lossy_squeezed(n, inputs.SEED_BASE + 9, (0.5, 1.2), 0.5)
    u = inputs.rng_for(inputs.SEED_BASE + 21).uniform(0.0, 1.0, size=(args.sample_count, n))
    flags = binding.TOR_EXTENDED if args.extended else 0
    ctx = binding.Context(device=local, flags=flags)
    sess = binding.Session(ctx, inst.sigma)
    binding.tor_sample(ctx, sess, u[:16])  # warm-up
    t0 = time.perf_counter()
    pat, prob, dev = binding.tor_sample(ctx, sess, u)
    el = time.perf_counter() - t0
    # the evaluations of each step: Tor(O^(j+1)_S) and Tor(O^(j+1)_{S u {j}}) for every distinct
    # S (the clicks before the step) among the samples, 2^|S| + 2^(|S|+1) subset terms
    terms, evals = sample_work(pat)
    before = np.cumsum(pat, axis=1) - pat
    k = pat.sum(axis=1)
    out = {"metric": "samples/s", "value": len(u) / el, "unit": "samples/s", "n_gpus": 1,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64x2" if args.extended else "f64", "data": "synthetic",
           "config": {"workload": "sample", "state": f"{n}-mode lossy squeezed, r~U[0.5,1.2], eta=0.5",
                      "samples": len(u), "modes": n,
                      "per_step": "Tor(O^(j+1)_S) and Tor(O^(j+1)_{S u {j}}) of the step's distinct S, "
                                  "in batched launches"},
           "seconds": el, "terms_per_s": terms / el, "tor_per_s": evals / el,
           "conditionals_per_s": 2.0 * len(u) * n / el,
           "requested_terms_per_s": float((3.0 * np.exp2(before)).sum()) / el,
           "mean_clicks": float(k.mean()), "max_clicks": int(k.max()),
           "min_log10_prob": float(np.log10(prob.min())), "chain_rule_max_dev": dev}
    # the plan tuned for the sampler's own batches: tor_autotune_batch on one step's batch (the
    # distinct marginals of the last step of the patterns just drawn), then the same sampling
    j = n - 1
    Oj = sess.marginal_matrix(j + 1)
    pmats = []
    for S in sorted({tuple(np.flatnonzero(row[:j])) for row in pat}):
        pmats += [inputs.submatrix(Oj, S), inputs.submatrix(Oj, S + (j,))]
    before_plan = {m: ctx.plan_prefix_depth(m) for m in range(1, n + 1)}
    t0 = time.perf_counter()
    binding.tor_autotune_batch(ctx, pmats, 10.0)
    tune_s = time.perf_counter() - t0
    binding.tor_sample(ctx, sess, u[:16])
    t0 = time.perf_counter()
    pat2, prob2, dev2 = binding.tor_sample(ctx, sess, u)
    el2 = time.perf_counter() - t0
    out["autotuned"] = {"value": len(u) / el2, "unit": "samples/s", "seconds": el2, "tune_s": tune_s,
                        "pilot_marginals": len(pmats), "same_patterns": bool(np.array_equal(pat, pat2)),
                        "max_prob_rel_diff": float(np.max(np.abs(prob2 - prob) / prob)),
                        "chain_rule_max_dev": dev2,
                        "changed_depths": {str(m): [before_plan[m], ctx.plan_prefix_depth(m)]
                                           for m in range(1, n + 1) if ctx.plan_prefix_depth(m) != before_plan[m]},
                        "what": "tor_autotune_batch (10 s) on the batch of the last chain-rule step of the "
                                "samples drawn above, then the same samples again"}
    out["autotuned_over_builtin"] = out["autotuned"]["value"] / out["value"]
    ctx.close()
    sess.close()
    print(json.dumps(out), flush=True)
    return 0


def run_sweep_n(args, world, rank, local):
    """Subset terms/s against the mode count n, one lossy squeezed state per n
    (r ~ U[0.3,0.8], eta_j ~ U[0.3,0.7]): the GPU (one device-resident tor_eval,
    CUDA events, best of a few), the paper's Algorithm 2 in FP64 on all host
    cores, and the binary128 oracle on all cores and on one.  The CPU rows stop
    where one evaluation would take longer than a few seconds."""
    if rank != 0:
        return 0
    import torch

    import oracle
    from oracle import alg2_cpu
    from paper_2109_04528_gb300 import binding, build
    build.build()
    oracle.build()
    alg2_cpu.build()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    cores = os.cpu_count() or 1
    rows = []
    with binding.Context(device=local, flags=binding.TOR_IN_DEVICE) as ctx:
        for n in range(8, 35, 2):
            O = inputs.config_single(n, seed=inputs.SEED_BASE + 1000 + n).O
            d = torch.from_numpy(O).to(device)
            binding.tor_eval(ctx, d)
            reps = 5 if n <= 28 else 2
            best = min((binding.tor_eval(ctx, d), ctx.last_times()["total_ms"])[1] for _ in range(reps))
            row = {"n": n, "gpu": 2.0 ** n / (best * 1e-3), "gpu_ms": best, "p": ctx.plan_prefix_depth(n)}
            if n <= 28:
                t0 = time.perf_counter()
                r = alg2_cpu.tor_alg2(O, threads=cores)
                row["cpu_alg2"] = r.terms / (time.perf_counter() - t0)
            if n <= 18:
                t0 = time.perf_counter()
                oracle.tor_brute(O, threads=cores)
                row["oracle"] = 2.0 ** n / (time.perf_counter() - t0)
            if n <= 14:
                t0 = time.perf_counter()
                oracle.tor_brute(O, threads=1)
                row["oracle_1core"] = 2.0 ** n / (time.perf_counter() - t0)
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "subset terms/s", "unit": "subset terms/s", "n_gpus": 1, "higher_is_better": True,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "sweep_n", "desc": "lossy squeezed, r~U[0.3,0.8], eta_j~U[0.3,0.7], one matrix per n",
                      "gpu": "one tor_eval per matrix, device-resident input, CUDA events (intake, units, reduce), best of 5 (2 for n > 28)",
                      "cpu_alg2": f"paper Algorithm 2 in FP64, {cores} threads, the whole sum",
                      "oracle": f"binary128 brute force, {cores} threads and 1 thread, the whole sum", "cpu": cpu_model()},
           "rows": rows}
    print(json.dumps(out), flush=True)
    return 0


ACCURACY_S = (0.2, 0.35, 0.5, 0.75, 1.0, 1.5)
ACCURACY_N = (12, 16, 20, 24, 28, 32)
ACCURACY_ORACLE_MAX_N = 16


def accuracy_row(n, S, r64, rx, oracle_ref=None, rx_rev=None):
    """One cell of the error-against-squeezing table: kappa = sum|term| / |Tor| and
    the relative error of the FP64 and double-double results against the binary128
    oracle where it runs (n <= ACCURACY_ORACLE_MAX_N), else the FP64 error against
    the double-double result and the double-double result's own error estimated
    from a second evaluation on the mode-reversed matrix."""
    if oracle_ref is not None:
        ref_hi, ref_lo, ref_name = oracle_ref.hi, oracle_ref.lo, "binary128 oracle"
    else:
        ref_hi, ref_lo, ref_name = rx.hi, rx.lo, "double-double GPU path"
    tref = ref_hi + ref_lo
    row = {"n": n, "S": S, "ref": ref_name, "tor": tref, "abs_sum": r64.abs_sum,
           "kappa": r64.abs_sum / abs(tref) if tref else None,
           "fp64_rel_err": abs((r64.hi - ref_hi) + (r64.lo - ref_lo)) / abs(tref) if tref else None,
           "fp64_rel_bound": r64.err_est / abs(tref) if tref else None,
           "ext_rel_bound": rx.err_est / abs(tref) if tref else None}
    if oracle_ref is not None:
        row["ext_rel_err"] = abs((rx.hi - ref_hi) + (rx.lo - ref_lo)) / abs(tref) if tref else None
    elif rx_rev is not None:
        row["ext_rel_diff_reversed"] = abs((rx.hi - rx_rev.hi) + (rx.lo - rx_rev.lo)) / abs(tref) if tref else None
    return row


def run_accuracy(args, world, rank, local):
    """The error of the FP64 and double-double paths against the squeezing S of the
    state (the question of Sec. 5, Fig. 6): lossy squeezed states with r_j ~
    U[0.8 S, 1.2 S], eta = 0.5 and a Haar unitary, one matrix per (n, S); the
    binary128 oracle is the reference up to n = 16, the double-double path beyond
    (its own error estimated by a second evaluation on the mode-reversed matrix)."""
    if rank != 0:
        return 0
    import torch

    import oracle
    from paper_2109_04528_gb300 import binding, build
    build.build()
    oracle.build()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    rows = []
    with binding.Context(device=local, flags=binding.TOR_IN_DEVICE) as c64, \
            binding.Context(device=local, flags=binding.TOR_IN_DEVICE | binding.TOR_EXTENDED) as cx:
        for n in ACCURACY_N:
            for k, S in enumerate(ACCURACY_S):
                inst = inputs.lossy_squeezed(n, inputs.SEED_BASE + 5000 + 10 * n + k, (0.8 * S, 1.2 * S), 0.5)
                d = torch.from_numpy(inst.O).to(device)
                r64 = binding.tor_eval(c64, d)
                rx = binding.tor_eval(cx, d)
                ref = rev = None
                if n <= ACCURACY_ORACLE_MAX_N:
                    ref = oracle.tor_brute(inst.O)
                else:
                    dr = torch.from_numpy(inputs.permute_modes(inst.O, list(range(n))[::-1])).to(device)
                    rev = binding.tor_eval(cx, dr)
                row = accuracy_row(n, S, r64, rx, ref, rev)
                rows.append(row)
                print(json.dumps(row), file=sys.stderr, flush=True)
    out = {"metric": "relative error of Tor", "unit": "|Tor - Tor_ref| / |Tor_ref|", "n_gpus": 1,
           "higher_is_better": False, "dtype": "f64 and f64x2", "data": "synthetic",
           "config": {"workload": "accuracy",
                      "desc": "lossy squeezed, r_j ~ U[0.8 S, 1.2 S], eta = 0.5, Haar U; one matrix per (n, S)",
                      "S": list(ACCURACY_S), "n": list(ACCURACY_N),
                      "reference": f"binary128 brute force for n <= {ACCURACY_ORACLE_MAX_N}; the double-double "
                                   "GPU path beyond, with its second evaluation on the mode-reversed matrix"},
           "rows": rows}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--weak", action="store_true",
                    help="several ranks: every rank evaluates its own copy of large_n30_34 (default there: the "
                         "ranks split each matrix's leaves, strong scaling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="large_n30_34: skip the nested results (n = 38, double-double, batch, serving)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end (host buffer) timing; 0 = --steps, at most 5 for n >= 30")
    ap.add_argument("--impl", default="libtor", choices=["libtor", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of host time for each CPU baseline (the oracle; Algorithm 2 in FP64)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--complex-path", action="store_true",
                    help="evaluate every matrix in complex arithmetic (TOR_COMPLEX_PATH)")
    ap.add_argument("--extended", action="store_true",
                    help="double-double factor arithmetic (TOR_EXTENDED)")
    ap.add_argument("--autotune", type=float, default=0.0,
                    help="seconds for the prefix-depth autotuner before timing (0 = built-in plan)")
    ap.add_argument("--sample-count", type=int, default=1000, help="sample: patterns to draw")
    ap.add_argument("--serve-window", type=float, default=2.0, help="serve: seconds of the overload window")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serve: offered requests/s")
    ap.add_argument("--serve-sustain-rate", type=float, default=40.0, help="serve: sustainable requests/s")
    ap.add_argument("--serve-sustain-window", type=float, default=8.0)
    ap.add_argument("--serve-high-rate", type=float, default=0.0,
                    help="serve: requests/s of the loaded run (0: 80%% of the capacity measured under overload)")
    ap.add_argument("--serve-high-window", type=float, default=8.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "serve":
        return run_serve(args, world, rank, local)
    if args.workload == "sample":
        return run_sample(args, world, rank, local)
    if args.workload == "sweep_n":
        return run_sweep_n(args, world, rank, local)
    if args.workload == "accuracy":
        return run_accuracy(args, world, rank, local)

    import torch

    from paper_2109_04528_gb300 import binding, build
    build.build()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    # Several ranks on one large-matrix workload split each matrix's leaves (strong scaling,
    # one host-level gather of three doubles per matrix and rank); otherwise every rank
    # evaluates its own copy of the workload (weak scaling, no data-path exchange).
    sharded = world > 1 and args.workload == "large_n30_34" and not args.weak
    mats, desc = workload(args.workload, 0 if sharded else rank)
    ns = [m.shape[0] // 2 for m in mats]
    terms = float(sum(2.0 ** n for n in ns))
    stream = torch.cuda.Stream(device=device)
    dmats = [torch.from_numpy(m).to(device) for m in mats]
    # device-resident inputs, plain launches (per-kernel CUDA-event times for the roofline)
    xf = (binding.TOR_COMPLEX_PATH if args.complex_path else 0) | (binding.TOR_EXTENDED if args.extended else 0)
    ctx_dev = binding.Context(device=local, stream=stream.cuda_stream, flags=binding.TOR_IN_DEVICE | xf)
    # host inputs through the C ABI, replayed as a CUDA graph
    ctx_host = binding.Context(device=local, stream=stream.cuda_stream, flags=binding.TOR_GRAPHS | xf)
    tuned = None
    if args.autotune > 0:
        sizes = sorted(set(ns))
        import tempfile
        plan_file = os.path.join(tempfile.mkdtemp(prefix="torplan_"), f"plan_{args.workload}.txt")
        tuned = {}
        for n in sizes:
            tuned.update(ctx_host.autotune(n, n, args.autotune / len(sizes)))
        ctx_host.save_plan(plan_file)
        ctx_dev.load_plan(plan_file)
    if sharded and not tuned:
        for n, p in sharded_depths(ctx_dev, ns, world).items():
            ctx_dev.set_prefix_depth(n, p)
            ctx_host.set_prefix_depth(n, p)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    dfma, fp64_tflops = binding.tor_probe_fp64(local, 0.5)

    paths = {}
    last_res = []

    def sharded_batch(ctx, batch):
        return sharded_step(binding, ctx, batch, ns, world, rank)

    def timed(ctx, batch, k):
        ms, units_ms = [], []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if sharded:
                res, u = sharded_batch(ctx, batch)
            else:
                res = binding.tor_eval_batch(ctx, batch)
                u = ctx.last_times()["units_ms"]
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            units_ms.append(u)
            for i, r in enumerate(res):
                if r.status != 0:
                    raise SystemExit(f"evaluation failed: status {r.status}")
                paths[i] = r.path
            last_res[:] = res
        return ms, units_ms

    timed(ctx_dev, dmats, args.warmup)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, units_ms = timed(ctx_dev, dmats, args.steps)
    torch.cuda.synchronize()
    barrier(world)
    tot_ms = max_over_ranks(world, sum(ms), device)
    # end to end: host buffers, H2D + kernels + D2H per step
    large = max(ns) >= 30
    e2e_steps = args.e2e_steps or (min(args.steps, 5) if large else args.steps)
    timed(ctx_host, mats, 1 if large else 2)
    barrier(world)
    e2e_ms, _ = timed(ctx_host, mats, e2e_steps)
    barrier(world)
    e2e_tot = max_over_ranks(world, sum(e2e_ms), device)
    copies = 1 if sharded else world  # sharded: the ranks split one copy of the workload
    value = terms * copies * args.steps / (tot_ms * 1e-3)
    e2e_value = terms * copies * e2e_steps / (e2e_tot * 1e-3)
    # the same device-resident step replayed as a CUDA graph (launch-bound steps only)
    graph_ms = None
    if not large:
        with binding.Context(device=local, stream=stream.cuda_stream,
                             flags=binding.TOR_IN_DEVICE | binding.TOR_GRAPHS | xf) as ctx_g:
            if tuned:
                ctx_g.load_plan(plan_file)
            timed(ctx_g, dmats, 2)
            gms, _ = timed(ctx_g, dmats, args.steps)
            graph_ms = sum(gms) / len(gms)
    plain = None
    if len(mats) > 8:
        # the plain GPU path: one tor_eval per matrix (launches + sync each), looped in C, same plan
        with binding.Context(device=local, stream=stream.cuda_stream,
                             flags=binding.TOR_IN_DEVICE | xf) as ctx_plain:
            if tuned:
                ctx_plain.load_plan(plan_file)
            binding.tor_eval_seq(ctx_plain, dmats[:64])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, lat = binding.tor_eval_seq(ctx_plain, dmats)
            plain_s = time.perf_counter() - t0
        lat = np.sort(lat)
        plain = {"value": terms / plain_s, "unit": "subset terms/s", "tor_per_s": len(mats) / plain_s,
                 "ms_per_batch": 1e3 * plain_s, "per_matrix_ms_p50": float(lat[len(lat) // 2]),
                 "per_matrix_ms_p99": float(lat[min(len(lat) - 1, int(0.99 * len(lat)))]),
                 "what": "tor_eval_seq: one tor_eval per matrix (descriptors H2D, 3 kernels, D2H, sync), "
                         "looped in C, host wall time"}
    units_avg = sum(units_ms) / len(units_ms)
    # algorithmic flops of the arithmetic each matrix actually took
    flops = float(sum(algorithmic_flops(n, paths.get(i, 0)) for i, n in enumerate(ns))) / (world if sharded else 1)
    n_real = sum(1 for i in range(len(ns)) if paths.get(i, 0) & 1)
    ext = any(paths.get(i, 0) & 2 for i in range(len(ns)))
    achieved = flops / (units_avg * 1e-3) / 1e12
    # Peak from unit counts and clocks: each SM issues FP64_PER_SM_CLK FP64 thread instructions
    # (add, mul or FMA) per cycle at the maximum SM clock.  The in-run DFMA-chain probe reaches
    # about 0.84 of it and is reported beside it.
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    clocks = clk.summary()
    sm_max_mhz = clocks.get("sm_max_mhz") or MAX_SM_MHZ
    peak_ops = sms * FP64_PER_SM_CLK * sm_max_mhz * 1e6
    peak_tflops = 2.0 * peak_ops / 1e12
    # The FP64 pipe issues one add, mul or FMA per slot alike, while the flop count weighs an FMA
    # twice; so also report the pipe's busy fraction in algorithmic FP64 instructions (flops.path_ops)
    from paper_2109_04528_gb300.flops import path_ops
    ops = float(sum(path_ops(n, paths.get(i, 0)) for i, n in enumerate(ns))) / (world if sharded else 1)
    inst = {"ops_per_launch": ops, "achieved_gops": ops / (units_avg * 1e-3) / 1e9,
            "peak_gops": peak_ops / 1e9, "frac": ops / (units_avg * 1e-3) / peak_ops,
            "probe_gops": dfma / 1e9,
            "what": "algorithmic FP64-pipe instructions (add, mul, FMA: 1 each; not the rcp/rsqrt estimates) per second "
                    "over the nominal FP64 issue rate (SMs x 2 per clock x max SM clock)"}
    line = {
        "metric": "subset terms/s", "value": value, "unit": "subset terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "ms_per_step_median": statistics.median(ms),
        "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f64x2" if ext else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "n": ns, "terms_per_step": terms,
                   "l2": "flushed between steps (512 MB write)",
                   "prefix_depth": {str(n): ctx_dev.plan_prefix_depth(n) for n in sorted(set(ns))}},
        "tor_per_s": len(mats) * copies * args.steps / (tot_ms * 1e-3),
        "e2e": {"value": e2e_value, "unit": "subset terms/s",
                "h2d_bytes_per_step": int(sum(m.size * 16 for m in mats)),
                "d2h_bytes_per_step": int(32 * len(mats)), "steps": e2e_steps},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops,
                     "traffic": profiled_traffic(args.workload, "k_units_ext" if ext else "k_units",
                                                 {str(n): ctx_dev.plan_prefix_depth(n) for n in sorted(set(ns))}),
                     "kernel": "k_units_ext" if ext else "k_units",
                     "peak_source": f"nominal FP64 rate from unit counts and clocks: {sms} SMs x "
                                    f"{FP64_PER_SM_CLK} FP64 FMA per clock x 2 flop x {sm_max_mhz:.0f} MHz",
                     "probe_tflops": fp64_tflops,
                     "flops_per_launch": flops, "units_ms_avg": units_avg,
                     "path": f"{n_real} of {len(ns)} matrices in the real (x,p) basis, rest complex"
                             + ("; double-double factor (every FP64 operation counted)" if ext else "")},
        "gpu_launches": launches_per_step(ctx_dev, ns) * args.steps,
        "clocks": clocks,
    }
    line["roofline"]["fp64_instructions"] = inst
    if graph_ms:
        line["graph_replay"] = {"ms_per_step": graph_ms, "value": terms / (graph_ms * 1e-3), "unit": "subset terms/s"}
    if tuned:
        line["config"]["autotuned"] = True
    if plain:
        line["plain_per_matrix"] = plain
        line["batched_over_plain"] = value / plain["value"]
    if sharded:
        one = [binding.tor_eval(ctx_dev, d) for d in dmats]  # the whole of every matrix on this GPU alone
        line["config"]["parallelism"] = f"leaf ranges of each matrix split over {world} ranks, host gather + fixed-tree merge"
        line["sharded_equals_one_gpu"] = all((a.hi, a.lo, a.abs_sum) == (b.hi, b.lo, b.abs_sum)
                                             for a, b in zip(last_res, one))
    if args.workload == "large_n30_34" and not args.no_extras and world == 1 and not xf:
        # nested results beside the timed steps; a failure in one of them is recorded in the
        # line instead of costing the headline
        def nested(key, fn):
            try:
                got = fn()
                if key is None:
                    line.update(got)
                else:
                    line[key] = got
            except Exception as e:  # noqa: BLE001 -- reported in the JSON line
                line.setdefault("nested_errors", {})[key or "errors_and_extended"] = f"{type(e).__name__}: {e}"
        res64 = list(binding.tor_eval_batch(ctx_dev, dmats))  # the timed step's own results
        nested(None, lambda: large_extras(local, stream, ctx_dev, mats, dmats, res64, ns, peak_ops))
        nested("batch4096", lambda: batch_compare(local, stream, steps=5))
        nested("small_batch", lambda: small_batch(local, stream))
        nested("serve", lambda: serve_summary(local, args.serve_high_window, args.serve_sustain_rate))
    elif last_res:
        line["results"] = [result_record(f"n={n}", n, r, None,
                                         ({"hi": g["hi"], "lo": g["lo"], "name": f"binary128 oracle ({g['method']}), stored"}
                                          if (g := golden_for(O)) is not None else None))
                           for n, r, O in zip(ns, last_res, mats)][:16]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mats, args.cpu_budget)
        line["cpu_alg2"] = cpu_alg2(mats, args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx_dev.close()
    ctx_host.close()
    torch.cuda.synchronize()  # surface any late device error in this process
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
