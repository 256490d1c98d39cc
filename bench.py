"""Benchmark of the B300 progressive refactor / retrieve path (one JSON line).

Workload (default): the 512^3 FP32 turbulence-like field (spectral Gaussian
random field, |u_hat| ~ k^-11/6, rescaled to [-1, 1], seed 2), refactored with
per-level cubic interpolation plus coefficient decomposition (slices normal to
the fastest axis) and generic bitplanes, then retrieved at a relative error
bound of 1e-4 (the tolerance of the paper's transfer use case).  One step =
refactor + plan + retrieve of that field.  value = field bytes processed per
second (refactor input + retrieve output) over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pcr|reference]

Multi-GPU (torchrun): every rank refactors and retrieves its own independent
field (the paper's block-parallel scaling: no data-path collective), so the
run is weak scaling; the max over ranks of the timed region defines the time.
--impl reference times the CPU oracle (test infrastructure) on a bounded
block of the same workload, on the host cores.
"""
import argparse
import collections
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FIELD_SHAPE = (512, 512, 512)
SEED = 2
TARGET = ("rel", 1e-4)
WORKLOAD = "grf_k-5/3_512^3_f32"
METRIC = "refactor & retrieve GB/s (fraction of HBM roofline) at stated eb/PSNR vs CPU oracle"

# DRAM traffic per launch of the dominant kernel, from a committed ncu
# summary under profiles/ (scaled by the level-0 value count when captured on
# a smaller field); absent when the kernel changed after that capture or the
# run's size differs.
TRAFFIC_PER_LAUNCH = {("encode_float", 512): 844.4e6}   # k_encode_f32 at 384^3: 356.3 MB x 2.370


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pcr", choices=["pcr", "reference"])
    ap.add_argument("--size", type=int, default=512, help="cube edge (default 512)")
    ap.add_argument("--mode", default="headline", choices=["headline", "batch", "serve", "shard"],
                    help="headline (default): the 512^3 step; batch: 96 uneven fields, one "
                         "batched refactor vs sequential calls; serve: continuous-batching server; "
                         "shard: one 1024x512x512 field as 256x512x512 blocks planned together")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the batch/serve workload")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """SM clock and throttle reasons sampled during the timed region.

    NVML (the driver's library, through ctypes) is read in-process from a
    background thread (one clock and one reason query per sample, no
    subprocess), on the device this process computes on (matched by UUID, so
    the NVML index is right under CUDA_VISIBLE_DEVICES).  __enter__ returns only after the first
    sample has been taken; __exit__ takes one more after the region.  Without
    NVML the nvidia-smi loop is the fallback."""

    PERIOD_S = 0.02
    NAMES = ["sw_power_cap", "hw_slowdown", "sw_thermal_slowdown", "hw_thermal_slowdown"]

    def __init__(self, device_index):
        self.device_index = device_index
        self.samples = []          # (sm_mhz, sm_max_mhz, [reason names])
        self.source = None
        self.nvml_error = None
        self._stop = threading.Event()
        self._thread = None
        self._nv = None
        self._h = None
        self.proc = None

    # NVML clock-event reason bits (nvml.h): sw power cap, hw slowdown, sw
    # thermal, hw thermal
    MASKS = [0x4, 0x8, 0x20, 0x40]
    NVML_CLOCK_SM = 1

    def _nvml_handle(self):
        """NVML through ctypes (libnvidia-ml ships with the driver)."""
        import ctypes as C
        import torch
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        props = torch.cuda.get_device_properties(self.device_index)
        h = C.c_void_p()
        uuid = ("GPU-" + str(props.uuid)).encode()
        if lib.nvmlDeviceGetHandleByUUID(C.c_char_p(uuid), C.byref(h)) != 0:
            bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0".encode()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) != 0:
                raise RuntimeError("no NVML handle for this device")
        return lib, h

    def _sample_nvml(self):
        import ctypes as C
        lib, h = self._nv, self._h
        sm, mx, bits = C.c_uint(), C.c_uint(), C.c_ulonglong()
        if (lib.nvmlDeviceGetClockInfo(h, self.NVML_CLOCK_SM, C.byref(sm)) or
                lib.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, C.byref(mx)) or
                lib.nvmlDeviceGetCurrentClocksEventReasons(h, C.byref(bits))):
            raise RuntimeError("NVML query failed")
        self.samples.append((float(sm.value), float(mx.value),
                             [n for n, m in zip(self.NAMES, self.MASKS) if bits.value & m]))

    def _loop(self):
        while not self._stop.wait(self.PERIOD_S):
            try:
                self._sample_nvml()
            except Exception:
                return

    def __enter__(self):
        try:
            self._nv, self._h = self._nvml_handle()
            self._sample_nvml()
            self.source = "nvml"
            self._thread = threading.Thread(target=self._loop, daemon=True)
            self._thread.start()
            return self
        except Exception as e:
            self._nv = None
            self.nvml_error = f"{type(e).__name__}: {e}"
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.sw_power_cap,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.hw_thermal_slowdown")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._thread = threading.Thread(target=self._read_smi, daemon=True)
            self._thread.start()
            self.source = "nvidia-smi"
            t0 = time.time()
            while not self.samples and time.time() - t0 < 10:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read_smi(self):
        for line in self.proc.stdout:
            s = [x.strip() for x in line.split(",")]
            try:
                self.samples.append((float(s[0]), float(s[1]),
                                     [n for n, v in zip(self.NAMES, s[2:6]) if v.lower() == "active"]))
            except (ValueError, IndexError):
                pass

    def __exit__(self, *exc):
        if self._nv is not None:
            self._stop.set()
            self._thread.join(timeout=2)
            try:
                self._sample_nvml()
            except Exception:
                pass
        elif self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = sorted({r for s in self.samples for r in s[2]})
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples), "reasons": reasons,
                "samples": len(self.samples), "source": self.source,
                **({"nvml_error": self.nvml_error} if self.nvml_error else {})}


def max_over_ranks(ms, world, device):
    """The timed region's milliseconds, the maximum over the ranks of the
    process group (every rank refactors and retrieves its own field, so the
    job ends when the slowest rank does)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(nbytes_per_rank, world, ms):
    """Whole-job throughput: every rank's field refactored and retrieved
    (2 x its bytes) within the slowest rank's time."""
    return world * 2 * nbytes_per_rank / (ms * 1e-3) / 1e9


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6400.0, "fallback": True}


def make_field(shape, device):
    import numpy as np
    import torch
    from synth import grf
    X = grf(shape, SEED, np.float32)
    return torch.from_numpy(X).to(device), X


def run_pcr(args):
    import numpy as np
    import torch
    import paper_2609_04573_b300 as pcr

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    shape = (args.size,) * 3
    x, X = make_field(shape, dev)
    nbytes = x.numel() * x.element_size()
    scheme = pcr.Scheme(mode="eb", interp="level", degree="cubic", decomp_axis=2)
    target = pcr.Target(*TARGET)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def step():
        h = pcr.refactor(x, scheme)
        pl = h.plan(target)
        h.retrieve(pl, out=out)
        return h, pl

    for _ in range(args.warmup):
        h, pl = step()
    torch.cuda.synchronize()
    # correctness of the timed configuration: bound respected at full size
    err = (out.double() - x.double()).abs().max().item()
    xmin, xmax, _ = h.field_stats()
    bound_ok = err <= TARGET[1] * (xmax - xmin)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    rstream = torch.cuda.Stream()

    def run_pipelined(k, sch=None, tgt=None):
        """k steps, step i+1's refactor enqueued before step i's tables are
        finished, planned and retrieved: the host work of one step overlaps
        the GPU work of the next.  Refactors run on `stream`, retrievals on
        `rstream`, so the small coarse-level kernels of one overlap the other.
        A handle is released only once its retrieval has run (its buffers
        belong to the refactor stream's allocator pool).  Exactly k
        refactors and k retrievals; `stream` waits for `rstream` at the end."""
        sch = sch or scheme
        tgt = tgt or target
        pending = collections.deque()
        job = pcr.refactor_async(x, sch, stream=stream)
        hk = plk = None
        for i in range(k):
            nxt = pcr.refactor_async(x, sch, stream=stream) if i + 1 < k else None
            hk = job.result()
            plk = hk.plan(tgt)
            hk.retrieve(plk, out=out, stream=rstream)
            done = torch.cuda.Event()
            done.record(rstream)
            pending.append((hk, done))
            while len(pending) > 2:
                pending.popleft()[1].synchronize()
            job = nxt
        stream.wait_stream(rstream)
        return hk, plk

    h, pl = run_pipelined(args.warmup)
    torch.cuda.synchronize()
    launches0 = pcr.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        h, pl = run_pipelined(args.steps)
        ev1.record(stream)
        barrier()
    launches = pcr.launch_count() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    pipe_err = (out.double() - x.double()).abs().max().item()
    bound_ok = bound_ok and pipe_err <= TARGET[1] * (xmax - xmin)
    # the same steps one after another (each refactor waits for its tables
    # before the next step starts), for comparison
    nser = min(args.steps, 50)
    es0, es1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    es0.record(stream)
    for _ in range(nser):
        step()
    es1.record(stream)
    torch.cuda.synchronize()
    serial_ms = es0.elapsed_time(es1) / nser
    # per-stage CUDA-event timing in a separate traced pass (tracing stays out
    # of the timed region above)
    psteps = min(args.steps, 5)
    pcr.profile_enable(True)
    pcr.profile_read(reset=True)
    for _ in range(psteps):
        h, pl = step()
    torch.cuda.synchronize()
    prof = pcr.profile_read(reset=True)
    pcr.profile_enable(False)
    ms = max_over_ranks(ms, world, dev)

    # the configuration's scheme (B): per-region cubic with the same
    # decomposition, negabinary + XOR planes, PSNR mode, retrieved at
    # 80 dB, pipelined the same way on fewer steps
    sch_b = pcr.Scheme(mode="psnr", interp="region", degree="cubic", decomp_axis=2)
    tgt_b = pcr.Target("psnr", 80.0)
    run_pipelined(args.warmup, sch_b, tgt_b)
    torch.cuda.synchronize()
    nr = max(10, args.steps // 4)
    er0, er1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    er0.record(stream)
    hb, plb = run_pipelined(nr, sch_b, tgt_b)
    er1.record(stream)
    torch.cuda.synchronize()
    R = xmax - xmin
    mse_b = ((out.double() - x.double()) ** 2).mean().item()
    ms_r = er0.elapsed_time(er1) / nr
    per_region = {"scheme": "(B) per-region cubic, order (0,1,2), decomposition (axis 2), negabinary + XOR, "
                            "PSNR mode, B=32", "target": "psnr 80",
                  "ms_per_step": ms_r, "value": whole_job_gbs(nbytes, 1, ms_r), "unit": "GB/s",
                  "psnr_db": 20 * math.log10(R / math.sqrt(mse_b)) if mse_b > 0 else None,
                  "bound_respected_full_size": bool(mse_b == 0 or 20 * math.log10(R / math.sqrt(mse_b)) >= 80.0),
                  "retrievals": sweep(pcr, hb, x, out, stream, R)}
    # progressive retrieval across the configuration's targets (plan +
    # retrieve of the per-level handle, event-timed, 5 repetitions each)
    retrievals = sweep(pcr, h, x, out, stream, R)
    progressive = progressive_leg(pcr, h, x, out, R)

    # e2e through the public API with host buffers (pinned), every step's
    # copies inside the timed region: the field in from pinned host memory,
    # the retrieved field out to it.  Pipelined as a streaming application
    # would run it: two device buffers each way and two copy streams, so step
    # i+1's upload and step i-1's download overlap step i's compute (the copy
    # engines run both directions and beside the kernels).
    xh = torch.from_numpy(X).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    xd = [torch.empty_like(x) for _ in range(2)]
    od = [torch.empty_like(x) for _ in range(2)]
    cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_run(n):
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_free = [torch.cuda.Event() for _ in range(2)]
        for e in ev_free:
            e.record(cout)
        with torch.cuda.stream(cin):
            xd[0].copy_(xh, non_blocking=True)
            ev_in[0].record(cin)
        for i in range(n):
            k = i % 2
            if i + 1 < n:   # step i-1's refactor has returned: its input buffer is free
                with torch.cuda.stream(cin):
                    xd[1 - k].copy_(xh, non_blocking=True)
                    ev_in[1 - k].record(cin)
            stream.wait_event(ev_in[k])
            h2 = pcr.refactor(xd[k], scheme, stream=stream)
            pl2 = h2.plan(target)
            stream.wait_event(ev_free[k])   # step i-2's download of od[k] is done
            h2.retrieve(pl2, out=od[k], stream=stream)
            ev_done[k].record(stream)
            with torch.cuda.stream(cout):
                cout.wait_event(ev_done[k])
                oh.copy_(od[k], non_blocking=True)
                ev_free[k].record(cout)
        stream.wait_stream(cout)

    e2e_run(3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps

    precision = precision_leg(pcr, dev) if rank == 0 else None
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6400.0)
    value = whole_job_gbs(nbytes, world, ms)
    # per-stage shares and the dominant stage's roofline
    total_prof = sum(v[0] for v in prof.values()) or 1.0
    stages = {k: {"ms_per_step": v[0] / psteps, "launches_per_step": v[1] / psteps,
                  "share": v[0] / total_prof} for k, v in prof.items()}
    dom = max(prof, key=lambda k: prof[k][0])
    n = x.numel()
    algo = algorithmic_bytes(dom, shape, x.element_size(), pl)
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)         # per launch
    achieved = algo["per_launch"] / (dom_ms * 1e-3) / 1e9 if algo["per_launch"] else None
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": TRAFFIC_PER_LAUNCH.get((dom, args.size)),
            "algorithmic_bytes_per_launch": algo["per_launch"], "ms_per_launch": dom_ms,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if not pk.get("fallback") else "fallback"}
    refactor_ms = sum(v[0] for k, v in prof.items() if k in REFACTOR_STAGES) / psteps
    retrieve_ms = sum(v[0] for k, v in prof.items() if k in RETRIEVE_STAGES) / psteps
    strict = 8.1 * n / 1e9 / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if shape == FIELD_SHAPE else f"grf_k-5/3_{'x'.join(map(str, shape))}_f32",
                   "shape": list(shape), "scheme": "per-level cubic + "
                   "coefficient decomposition (axis 2) + generic bitplanes, B=32",
                   "target": f"{TARGET[0]} {TARGET[1]}", "l2": f"inputs larger than L2 ({nbytes >> 20} MB field)",
                   "parallelism": f"replicas x{world}",
                   "pipelined": "step i+1's refactor enqueued before step i's tables are finished, "
                                "planned and retrieved; refactors and retrievals on two streams; "
                                "K refactors + K retrievals timed"},
        "serial": {"ms_per_step": serial_ms, "value": whole_job_gbs(nbytes, world, serial_ms), "steps": nser},
        "refactor_gbs": nbytes / (refactor_ms * 1e-3) / 1e9 if refactor_ms else None,
        "retrieve_gbs": nbytes / (retrieve_ms * 1e-3) / 1e9 if retrieve_ms else None,
        "strict_roofline_frac": {"refactor": (8.1 * n / (refactor_ms * 1e-3) / 1e9) / hbm if refactor_ms else None,
                                 "retrieve": ((pl.bytes + 4 * n) / (retrieve_ms * 1e-3) / 1e9) / hbm
                                 if retrieve_ms else None},
        "retrieve_bytes_per_elem": pl.bytes / n, "bound_respected_full_size": bool(bound_ok),
        "max_err": err, "roofline": roof, "stages": stages, "progressive": progressive,
        "e2e": {"value": world * 2 * nbytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms,
                "pipelined": "upload of step i+1 and download of step i-1 overlap step i (two copy streams)"},
        "per_region": per_region, "retrievals": retrievals, "precision": precision,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "cpu_baseline": cpu_baseline(),
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SWEEP = [("rel", 10.0 ** -k) for k in range(1, 8)] + [("psnr", float(d)) for d in range(40, 121, 20)]


def sweep(pcr, h, x, out, stream, R, targets=SWEEP, reps=5):
    """Plan + retrieve of one handle at each target (event-timed, `reps`
    repetitions); bytes read, whether the bound meets the target and
    whether the retrieved field does."""
    import torch
    res = []
    ptab = h.packed_tables()
    for kind, v in targets:
        tg = pcr.Target(kind, v)
        plr = h.plan(tg, allow_unsat=True)
        h.retrieve(plr, out=out)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(reps):
            h.retrieve(h.plan(tg, allow_unsat=True), out=out)
        eb.record(stream)
        torch.cuda.synchronize()
        d = out.double() - x.double()
        e = d.abs().max().item()
        mse = (d ** 2).mean().item()
        ok = (e <= v * R) if kind == "rel" else (mse == 0 or 20 * math.log10(R / math.sqrt(mse)) >= v)
        coded = sum(ptab[i][b] for i, b in enumerate(plr.planes))
        row = {"target": f"{kind} {v:g}", "ms": ea.elapsed_time(eb) / reps, "bytes": plr.bytes,
               "bytes_per_value": plr.bytes / x.numel(), "coded_bytes_per_value": coded / x.numel(),
               "satisfied": bool(plr.satisfied),
               "within_target": bool(ok) if plr.satisfied else None, "max_err": e}
        if plr.satisfied:
            # the best-first search interpreter on the same target: its plan
            # retrieved once and checked the same way
            pls, info = h.plan_search(tg)
            h.retrieve(pls, out=out)
            torch.cuda.synchronize()
            d = out.double() - x.double()
            es, mses = d.abs().max().item(), (d ** 2).mean().item()
            oks = (es <= v * R) if kind == "rel" else (mses == 0 or 20 * math.log10(R / math.sqrt(mses)) >= v)
            row["search"] = {"bytes": pls.bytes, "bytes_per_value": pls.bytes / x.numel(),
                             "vs_greedy": pls.bytes / plr.bytes, "expanded": info["expanded"],
                             "optimal": info["optimal"], "plan_ms": info["plan_ms"], "within_target": bool(oks)}
        res.append(row)
    return res


def progressive_leg(pcr, h, x, out, R, values=(1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)):
    """A progressive session over the headline handle (Progressive.refine:
    each tighter relative target planned from the planes already fetched):
    per refinement the bytes it adds, the retrieval time and the error; and
    the one-shot plan of the last target for comparison."""
    import torch
    sess = pcr.Progressive(h)
    rows = []
    for v in values:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o, pl, added = sess.refine(pcr.Target("rel", v), out=out)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e = (o.double() - x.double()).abs().max().item()
        rows.append({"target": f"rel {v:g}", "added_bytes": added, "plan_bytes": pl.bytes,
                     "satisfied": bool(pl.satisfied), "ms": dt * 1e3,
                     "within_target": (e <= v * R) if pl.satisfied else None})
    one = h.plan(pcr.Target("rel", values[-1]), allow_unsat=True)
    return {"refinements": rows, "session_bytes": sess.fetched, "one_shot_bytes_last_target": one.bytes}


def precision_leg(pcr, dev):
    """The FP64 climate-like 256x384x384 field refactored in FP64 (B = 64,
    FP64 tables) and its FP32 cast refactored in FP32 (B = 32): per-level
    cubic + decomposition (axis 2), retrievals at relative bounds 1e-3 ..
    1e-9 and with every plane; each retrieval's error measured against the
    FP64 field."""
    import numpy as np
    import torch
    from synth import climate
    X64 = climate((256, 384, 384), 3)
    x64 = torch.from_numpy(X64).to(dev)
    R = float(X64.max() - X64.min())
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    out = {}
    stream = torch.cuda.current_stream()
    for name, xin in (("f64", x64), ("f32_cast", x64.float())):
        pcr.refactor(xin, sch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            h = pcr.refactor(xin, sch)
        e1.record(stream)
        torch.cuda.synchronize()
        ref_ms = e0.elapsed_time(e1) / 3
        rows = []
        o = torch.empty_like(xin)
        B = h.stream_info(0)["nplanes"]
        plans = [("rel", 10.0 ** -k) for k in range(3, 10)]
        for kind, v in plans + [("all planes", None)]:
            pl = h.plan(pcr.Target(kind, v), allow_unsat=True) if v else h.plan_from_planes([B] * h.nstreams)
            h.retrieve(pl, out=o)
            torch.cuda.synchronize()
            err = (o.double() - x64).abs().max().item()
            rows.append({"target": f"{kind} {v:g}" if v else kind, "bytes_per_value": pl.bytes / xin.numel()
                         if v else None, "satisfied": bool(pl.satisfied) if v else None,
                         "max_err_vs_f64": err, "rel_err_vs_f64": err / R,
                         "within_target": (err <= v * R) if v and pl.satisfied else None})
        out[name] = {"refactor_ms": ref_ms, "refactor_gbs": xin.numel() * xin.element_size() / ref_ms / 1e6,
                     "retrievals": rows}
    return {"workload": "climate-like 256x384x384 (zonal bands x lognormal noise, seed 3)",
            "scheme": "per-level cubic + decomposition (axis 2), generic", "range": R, **out}


REFACTOR_STAGES = {"stats", "to_fixed", "coarsest", "interp_level0", "interp_fixed_levels", "zero_pads",
                   "absmax", "decompose", "encode_float", "encode_fixed"}
RETRIEVE_STAGES = {"decode_float", "decode_fixed", "recompose", "recon_coarsest", "recon_fixed_levels",
                   "coarse_out", "recon_level0", "copy_raw"}


def algorithmic_bytes(stage, shape, w, pl):
    """Algorithmic DRAM bytes of one launch of a stage:
    interp_level0 (refactor): read the field, write level-0 coefficients;
    recon_level0: read level-0 coefficients and the coarse points' fixed-point
      values (8 bytes each), write field;
    decompose / recompose: read and write the decomposed region values;
    encode_float: read level-0 stream values, write B planes + signs;
    decode_float: read the planned planes + signs, write stream values."""
    n = math.prod(shape)
    n0 = n - math.prod((s + 1) // 2 for s in shape)  # level-0 points (odd somewhere)
    table = {
        "interp_level0": (n * w + n0 * w) / 1,
        "recon_level0": n0 * w + (n - n0) * 8 + n * w,
        "decompose": 2 * n0 * w / 3,          # three launches (regions) per step
        "recompose": 2 * n0 * w / 3,
        "encode_float": n0 * w + n0 * 4 + n0 / 8,
        "decode_float": pl.bytes + n0 * w,
    }
    return {"per_launch": table.get(stage)}


def _oracle_block(job):
    """One block of the headline recipe through the oracle (refactor +
    retrieve at the headline target); runs in a spawned worker process."""
    edge, seed = job
    import numpy as np
    import oracle
    from synth import grf
    X = grf((edge,) * 3, seed, np.float32)
    t0 = time.perf_counter()
    h = oracle.refactor(X, oracle.Scheme(mode="eb", interp="level", degree="cubic", decomp_axis=2))
    oracle.retrieve(h, oracle.Target(*TARGET))
    return 2 * X.nbytes, time.perf_counter() - t0


MAX_ORACLE_WORKERS = 32


def _one_thread():
    os.environ["OMP_NUM_THREADS"] = "1"


def oracle_all_cores(edge, rounds, warm=True):
    """The oracle on every usable host core (capped at MAX_ORACLE_WORKERS
    processes, one block each per round, spawned: the parent already holds a
    CUDA context).  Returns (GB/s over the wall time of the rounds, workers,
    seconds)."""
    import multiprocessing as mp
    try:
        ncpu = len(os.sched_getaffinity(0))
    except AttributeError:
        ncpu = os.cpu_count() or 1
    workers = max(1, min(ncpu, MAX_ORACLE_WORKERS))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_one_thread) as pool:
        if warm:
            pool.map(_oracle_block, [(16, 1)] * workers)          # import and start every worker
        t0 = time.perf_counter()
        done = 0
        for r in range(rounds):
            res = pool.map(_oracle_block, [(edge, SEED + 100 * r + k) for k in range(workers)])
            done += sum(b for b, _ in res)
        wall = time.perf_counter() - t0
    return done / wall / 1e9, workers, wall


def cpu_baseline():
    """The oracle on the host: every usable core (the reported figure) and
    one core, on bounded blocks of the same workload."""
    gbs, workers, wall = oracle_all_cores(128, 2)
    nb, dt = _oracle_block((128, SEED))
    return {"value": gbs, "unit": "GB/s", "cores": workers, "kind": "oracle",
            "single_core_value": nb / dt / 1e9,
            "sample": f"{2 * workers} blocks of 128^3 of the same recipe (refactor + retrieve at rel 1e-4), "
                      f"{workers} single-threaded numpy processes, {wall:.1f} s wall; single core: one "
                      f"128^3 block, {dt:.1f} s"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    edge = 128
    gbs, workers, wall = oracle_all_cores(edge, args.warmup, warm=True) if args.warmup else (0, 0, 0)
    gbs, workers, wall = oracle_all_cores(edge, args.steps, warm=False)
    dt = wall / args.steps
    sample = (f"per step {workers} blocks of 128^3 of the same recipe (refactor + retrieve at rel 1e-4), "
              f"one per single-threaded numpy process")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "shape": list(FIELD_SHAPE), "sample_shape": [edge] * 3},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args):
    """96 independent fields of uneven shapes (32 x 100x500x500, 32 x
    64x256x1024, 32 x 2-D 1800x3600): the batch captured in one CUDA graph
    (autotuned level schedule), and one batched refactor (one work list per
    stage, one synchronisation), against the same fields refactored one call
    at a time."""
    import torch
    import paper_2609_04573_b300 as pcr
    from synth.device import grf_torch
    torch.cuda.set_device(0)
    per = max(1, int(round(32 * args.scale)))
    shapes = [(100, 500, 500)] * per + [(64, 256, 1024)] * per + [(1800, 3600)] * per
    xs = [grf_torch(s, 1000 + i) for i, s in enumerate(shapes)]
    nbytes = sum(x.numel() * 4 for x in xs)
    schemes = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if x.dim() == 3 else -1) for x in xs]
    torch.cuda.synchronize()
    hb = pcr.refactor_batch(xs, schemes)          # warm-up
    del hb
    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r
    tb, hb = timed(lambda: pcr.refactor_batch(xs, schemes))
    ts, hs = timed(lambda: [pcr.refactor(x, s) for x, s in zip(xs, schemes)])
    # the same batch captured in one CUDA graph (creation autotunes the level
    # schedule and refactors once); the timed runs are graph launches
    tc0 = time.perf_counter()
    g = pcr.RefactorGraph(xs, schemes)
    torch.cuda.synchronize()
    tcreate = time.perf_counter() - tc0
    g.run()
    runs = sorted(((timed(g.run)[0], g.times()) for _ in range(5)), key=lambda t: t[0])
    tg, gt = runs[len(runs) // 2]
    same = all(a.stream_copy(i)[0].tobytes() == b.stream_copy(i)[0].tobytes() == c.stream_copy(i)[0].tobytes()
               for a, b, c in zip(hb[:3], hs[:3], g.handles[:3]) for i in range(a.nstreams))
    print(json.dumps({"mode": "batch", "fields": len(xs), "bytes": nbytes,
                      "graph_gbs": nbytes / tg / 1e9, "batched_gbs": nbytes / tb / 1e9,
                      "sequential_gbs": nbytes / ts / 1e9, "graph_s": tg, "batched_s": tb, "sequential_s": ts,
                      "graph_create_s": tcreate, "graph": {**g.info(), **gt},
                      "graph_device_gbs": nbytes / gt["gpu_ms"] / 1e6,
                      "speedup_graph_vs_sequential": ts / tg, "speedup_batched_vs_sequential": ts / tb,
                      "autotuned": {str(k): v for k, v in pcr.autotune_table().items()},
                      "first_fields_identical": same}))


def run_shard(args):
    """Block sharding (the paper's per-block scaling setup: 256x512x512
    blocks): one 1024x512x512 FP32 GRF refactored as four axis-0 blocks on
    this GPU (ShardedField), planned together for whole-field targets and
    retrieved into one output; the same field refactored whole for
    comparison.  Under torchrun every rank holds its blocks of a field of
    world x 4 blocks and plans through distributed_plans (states exchanged
    over a gloo group)."""
    import torch
    import torch.distributed as dist
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.shard import ShardedField, distributed_plans
    from synth.device import grf_torch
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nb = 4
    shape = (256 * nb, 512, 512)
    x = grf_torch(shape, 7)
    nbytes = x.numel() * 4
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    targets = [("rel", 1e-4), ("psnr", 80.0)]

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps, r

    t_ref, sf = timed(lambda: ShardedField(x, nb, sch))
    t_whole, hw = timed(lambda: pcr.refactor(x, sch))
    out = torch.empty_like(x)
    rows = []
    for kind, v in targets:
        tg = pcr.Target(kind, v)
        t0 = time.perf_counter()
        pls, bound, ok = sf.plan(tg)
        t_plan = time.perf_counter() - t0
        t_ret, _ = timed(lambda: sf.retrieve(pls, out=out))
        d = out.double() - x.double()
        R = (x.max() - x.min()).item()
        err = d.abs().max().item()
        mse = (d ** 2).mean().item()
        pw = hw.plan(tg, allow_unsat=True)
        rows.append({"target": f"{kind} {v:g}", "satisfied": ok, "bytes": sum(p.bytes for p in pls),
                     "bytes_whole_field_plan": pw.bytes, "plan_ms": t_plan * 1e3,
                     "retrieve_gbs": nbytes / t_ret / 1e9, "max_err_rel": err / R,
                     "psnr_db": 20 * math.log10(R / math.sqrt(mse)) if mse > 0 else None})
    res = {"mode": "shard", "field": list(shape), "blocks": nb, "block": [256, 512, 512],
           "refactor_blocks_gbs": nbytes / t_ref / 1e9, "refactor_whole_gbs": nbytes / t_whole / 1e9,
           "targets": rows}
    if world > 1:
        if not dist.is_initialized():
            dist.init_process_group("gloo")
        local_blocks = [(rank * nb + i, h) for i, h in enumerate(sf.handles)]
        t0 = time.perf_counter()
        plans, bound, ok = distributed_plans(local_blocks, pcr.Target("psnr", 80.0))
        res["distributed"] = {"world": world, "blocks": world * nb, "plan_ms": (time.perf_counter() - t0) * 1e3,
                              "satisfied": ok}
    if rank == 0:
        print(json.dumps(res))


def run_serve(args):
    """Resident refactored fields, Poisson arrivals of mixed-tolerance
    requests (half whole-field, half 128^3 boxes), continuous batching with
    memory admission, against a one-at-a-time server."""
    import random
    import torch
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.serve import Server, percentile
    from synth.device import grf_torch
    torch.cuda.set_device(0)
    n512 = max(1, int(round(48 * args.scale)))
    n256 = max(1, int(round(192 * args.scale)))
    shapes = [(512,) * 3] * n512 + [(256,) * 3] * n256
    handles = []
    for i, s in enumerate(shapes):
        x = grf_torch(s, 2000 + i)
        handles.append(pcr.refactor(x, pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)))
        del x
    torch.cuda.synchronize()
    resident = sum(sum(h.stream_info(i)["words"] * 4 * h.stream_info(i)["nplanes"] for i in range(h.nstreams))
                   for h in handles)
    rng = random.Random(7)
    nreq = max(50, int(400 * min(1.0, args.scale * 4)))
    reqs, t = [], 0.0
    for _ in range(nreq):
        t += rng.expovariate(2000.0)
        f = rng.randrange(len(handles))
        if rng.random() < 0.5:
            tg = pcr.Target("rel", 10.0 ** -rng.randint(2, 6))
        else:
            tg = pcr.Target("psnr", float(rng.choice(range(50, 111, 10))))
        box = None
        if rng.random() < 0.5:
            box = tuple((lo, lo + 128) for lo in (rng.randrange(0, s - 127) for s in shapes[f]))
        reqs.append((t, f, tg, box))

    def serve(batch, streams, budget):
        srv = Server(handles, mem_budget=budget, max_batch=batch, streams=streams)
        t0 = time.perf_counter()
        live = []
        for ta, f, tg, box in reqs:
            while time.perf_counter() - t0 < ta:
                time.sleep(0.00005)
            live.append(srv.submit(f, tg, box))
        for r in live:
            r.future.result(timeout=600)
        wall = time.perf_counter() - t0
        srv.close()
        lat = [r.latency * 1e3 for r in live]
        # bytes delivered: the field, or the box of a box request
        out_bytes = sum(handles[r.field_id].out_bytes if r.box is None else
                        math.prod(b - a for a, b in r.box) * 4 for r in live)
        return {"p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "wall_s": wall,
                "field_gbs": out_bytes / wall / 1e9, "read_gbs": sum(r.bytes_read for r in live) / wall / 1e9,
                "batches": srv.batches}
    cont = serve(16, 2, 24 << 30)
    seq = serve(1, 1, 24 << 30)
    print(json.dumps({"mode": "serve", "fields": len(handles), "resident_plane_bytes": resident,
                      "requests": nreq, "arrival_rate_per_s": 2000, "continuous": cont, "sequential": seq}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "batch":
        run_batch(a)
    elif a.mode == "shard":
        run_shard(a)
    elif a.mode == "serve":
        run_serve(a)
    else:
        run_pcr(a)
