"""Benchmark: coded A.B with e erasures (array BP-XOR code), one JSON line.

Workload (``sysmoj_8192``): systematic Mojette array code n = 11 (k = 8 data
columns of an 8 x 8 source grid, e = 3 parity projections), h = 128-row
source blocks, A and B 8192 x 8192 FP32 iid N(0,1); step i erases 3 columns
drawn from seed 2000 + (i mod 100) (100 trials).  One step = the whole hot
path: symbolic peel, encode + coded products, numeric peel.

value = useful 2MNK FLOP / step time of the headline precision (split-BF16x3
on tcgen05 when the build has it, else plain FP32), with inputs resident in
HBM (A, B = 256 MB each, larger than L2).  The FP32 CUDA-core path is timed
beside it.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import ctypes as ct
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "useful TFLOP/s of coded A·B w/ e erasures, BF16x3 vs FP32; rel. error"
WORKLOAD = "sysmoj_8192"

CODE_TEXT = {
    "sysmoj_8192": "systematic Mojette array n=11 (k=8 data columns, 8x8 grid, e=3 parities q=1, slopes 0,+1,-1)",
    "mojA_16384": "Mojette Construction A n=32 (k=24 x b=683 grid, q=1, p=-15..16), e=8",
    "sysmoj_8192_2d": "systematic Mojette array n=11 (k=8 data columns, 8x8 grid, e=3 parities q=1, slopes 0,+1,-1) "
                      "in the two-dimensional scheme (source (z, l) = A_z B_l, 1024 x 1024 blocks)",
    "sysmoj_8192_straggler": "systematic Mojette array n=11 (k=8 data columns, 8x8 grid, e=3 parities q=1, "
                             "slopes 0,+1,-1); processor-level stragglers, task times sigma_c X_c, X_c ~ Exp(1)",
    "mojA_16384_straggler": "Mojette Construction A n=32 (k=24 x b=683 grid, q=1, p=-15..16); processor-level "
                            "stragglers, task times sigma_c X_c, X_c ~ Exp(1)",
    "mojA_bsweep": "Mojette Construction A n=32 (k=24 x b grid, q=1, p=-15..16), e=8, b in {16, 32, 64, 683}",
    "batch512": "512 jobs: half array codes (Table I, Table III, systematic Mojette n=6..32, e=2..3), "
                "half Construction A (n=6..32, e=n//4); each job its own seeded mask",
}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the coded GEMM at full size, from a one-pass ncu capture of this benchmark's
# own launch (default tile config, first timed step), keyed by workload,
# precision, config and the SHA-256 of the GEMM sources it was taken with: a
# changed kernel reports null until it is captured again.
TRAFFIC = {
    ("sysmoj_8192", "bf16x3", 0): ("b653608ba7325866b23c715fd20a2f60acb16d7b16b30ed9f30d539d646aa41b",
                                   2741324288 + 301022720),
}


def _traffic(wl_name, prec, cfg):
    import hashlib
    ent = TRAFFIC.get((wl_name, prec, cfg))
    if ent is None:
        return None
    h = hashlib.sha256()
    for name in ("gemm_tc.cu", "tc_common.cuh"):  # the kernel's sources
        with open(os.path.join(ROOT, "paper_1904_11563_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return ent[1] if h.hexdigest() == ent[0] else None


def _lib_code(bpx, wl):
    kind, *args = wl["code"]
    return {"systematic": lambda: bpx.Code.systematic(*args),
            "mojette_a": lambda: bpx.Code.mojette_a(*args),
            "table1": bpx.Code.table1, "table3": bpx.Code.table3}[kind]()


def _oracle_code(o, wl):
    kind, *args = wl["code"]
    return {"systematic": lambda: o.systematic_mojette(*args),
            "mojette_a": lambda: o.construction_a(*args),
            "table1": o.table1, "table3": o.table3}[kind]()


def _n_cols(wl):
    kind, *args = wl["code"]
    return {"systematic": lambda: args[0] + args[1], "mojette_a": lambda: args[0]}.get(kind, lambda: 5)()


def _mask(W, wl, t):
    return W.erasure_mask(_n_cols(wl), wl["e"], wl["mask_seed_base"] + (t % wl.get("trials", 100)))


def _parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "bf16x3", "bf16", "mxfp8", "fp32", "exact", "fp16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-inflight", type=int, default=3,
                    help="end-to-end steps in flight (each on its own stream with its own device buffers)")
    ap.add_argument("--inflight", type=int, default=2,
                    help="steps in flight in the timed region of `value` (each on its own stream with its own "
                         "workspace, C and info words); 1 = one step at a time")
    ap.add_argument("--compensate-depth", type=int, default=-1,
                    help="peel the sources deeper than this with compensated subtraction (-1: off)")
    ap.add_argument("--gemm-config", type=int, default=0,
                    help="tensor-core GEMM tile config; 0 = the library default, -1 = run the library's "
                         "autotuner first")
    ap.add_argument("--precisions", default="",
                    help="comma list overriding the timed precisions (e.g. 'bf16x3' for profiling)")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(CODE_TEXT))
    ap.add_argument("--shape", default="",
                    help="M,N,K override of the workload (profiling of reduced cases only)")
    ap.add_argument("--jobs", type=int, default=512,
                    help="jobs of the batch512 workload (fewer: profiling of reduced cases only)")
    ap.add_argument("--oracle-sample-seconds", type=float, default=0.0,
                    help=argparse.SUPPRESS)  # internal: time the oracle alone for about this long, print JSON
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def _config(wl):
    mb = 4 * wl["M"] * wl["K"] / 1e6
    return {"workload": wl["name"], "code": CODE_TEXT[wl["name"]],
            "M": wl["M"], "N": wl["N"], "K": wl["K"], "h": wl["h"], "erasures": wl["e"],
            "trials": wl.get("trials", 100),
            "mask_seeds": f"{wl['mask_seed_base']}+t, t=step mod {wl.get('trials', 100)}",
            "inputs": f"A, B iid {'N(0,1)' if wl['dist'] == 'normal' else 'U(-1,1)'} FP32, seeded",
            "l2": f"inputs larger than L2 (A {mb:.0f} MB; no flush)"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling (every 25 ms) while the timed
    region runs.  Each sample is stamped with the host time it arrived;
    begin() / end() bracket the timed loops, and the record keeps the samples
    inside that window (all samples only when none fell inside)."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.window = [None, None]

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def begin(self):
        if self.window[0] is None:
            self.window[0] = time.time()

    def end(self):
        self.window[1] = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)  # the sample that covers the window's end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

        def parse(rows):
            sm, smax, reasons = [], [], set()
            for _t, ln in rows:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) != len(self.FIELDS):
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[3:]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            return sm, smax, reasons

        t0, t1 = self.window
        inside = [r for r in self.lines if t0 is not None and t1 is not None and t0 <= r[0] <= t1 + 0.03]
        sm, smax, reasons = parse(inside)
        in_window = bool(sm)
        if not sm:
            sm, smax, reasons = parse(self.lines)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "in_timed_region": in_window,
                "period_ms": 25}


class StageEvents:
    """CUDA events the library records around each kernel of a step."""

    def __init__(self, bpx, steps):
        self.rt = ct.CDLL("libcudart.so.13")
        self.rt.cudaEventCreate.argtypes = [ct.POINTER(ct.c_void_p)]
        self.rt.cudaEventElapsedTime.argtypes = [ct.POINTER(ct.c_float), ct.c_void_p, ct.c_void_p]
        self.rt.cudaEventDestroy.argtypes = [ct.c_void_p]
        self.n = 2 * bpx.NUM_STAGES
        self.arrays = []
        for _ in range(steps):
            arr = (ct.c_void_p * self.n)()
            for i in range(self.n):
                ev = ct.c_void_p()
                assert self.rt.cudaEventCreate(ct.byref(ev)) == 0
                arr[i] = ev
            self.arrays.append(arr)

    def ptr(self, i):
        return ct.cast(self.arrays[i], ct.POINTER(ct.c_void_p))

    def stage_ms(self, i, stage):
        """Milliseconds between the stage's two events, or None when the path
        did not record them (the error is cleared so that it does not
        surface in a later CUDA call)."""
        a = self.arrays[i]
        ms = ct.c_float()
        rc = self.rt.cudaEventElapsedTime(ct.byref(ms), a[2 * stage], a[2 * stage + 1])
        if rc != 0:
            self.rt.cudaGetLastError()
            return None
        return ms.value


# ------------------------------------------------------------------ CPU oracle legs

TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "fp16x3": 1e-5, "bf16": 2e-2, "mxfp8": 6e-2, "exact": 1e-5,
       "bf16x3-fused": 1e-5}
# MMA flops executed per useful coded flop by each tensor-core precision
MMA_MULT = {"bf16x3": 3, "bf16x3-fused": 3, "fp16x3": 3, "bf16": 1, "mxfp8": 1}


def _propagation(code, order, Ah, Bh, h, sources, ncols=256, kappa=None):
    """nu_s = sqrt(sum_c coef_{s,c}^2 ||P_c||^2) / ||C_s|| for the sampled
    sources: coef from the peel recurrence over the library's plan (each
    recovered source = its resolver's product minus the resolver's other
    sources), norms of FP64 products on the first `ncols` columns of B.
    With a dict `kappa`, also kappa_s = sum_c |coef_{s,c}| ||P_c|| / ||C_s||
    (the worst case) into it."""
    res = {int(s_): int(r_) for s_, r_, _d in order if s_ >= 0}
    seq = [int(s_) for s_, _r, _d in order if s_ >= 0]
    coef = {}
    for s_ in seq:
        r_ = res[s_]
        e_ = {r_: 1}
        for t_ in code.cell_src[code.cell_ptr[r_]:code.cell_ptr[r_ + 1]]:
            t_ = int(t_)
            if t_ != s_:
                for c_, v_ in coef[t_].items():
                    e_[c_] = e_.get(c_, 0) - v_
        coef[s_] = {c_: v_ for c_, v_ in e_.items() if v_}
    Bs = Bh[:, :ncols]
    M = Ah.shape[0]

    def blk(s_):
        lo, hi = s_ * h, min((s_ + 1) * h, M)
        out = np.zeros((h, Ah.shape[1]))
        if lo < hi:
            out[:hi - lo] = Ah[lo:hi]
        return out

    pn = {}
    nu = {}
    for s_ in sources:
        for c_ in coef[s_]:
            if c_ not in pn:
                Ac = sum(blk(int(t_)) for t_ in code.cell_src[code.cell_ptr[c_]:code.cell_ptr[c_ + 1]])
                pn[c_] = float(np.linalg.norm(Ac @ Bs))
        num = np.sqrt(sum(float(v_) ** 2 * pn[c_] ** 2 for c_, v_ in coef[s_].items()))
        den = np.linalg.norm(blk(s_) @ Bs)
        nu[s_] = float(num / den)
        if kappa is not None:
            kappa[s_] = float(sum(abs(float(v_)) * pn[c_] for c_, v_ in coef[s_].items()) / den)
    return nu


def _oracle_sample(A, B, h, mask, ncols, wl):
    """Runs the FP64 oracle's whole coded path on the first ncols columns of
    B (the path is columnwise separable); returns seconds."""
    from oracle import bpx_oracle as o
    code = _oracle_code(o, wl)
    t0 = time.perf_counter()
    C, sch = o.coded_matmul(code, A, B[:, :ncols], h, list(np.nonzero(mask)[0]))
    dt = time.perf_counter() - t0
    assert sch.ok
    return dt


def _cores():
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count()


def _oracle_timed(A, B, wl, budget_s, cols):
    """Times the oracle's coded path on column samples of `cols` columns until
    about budget_s seconds have passed; returns (seconds, columns)."""
    from paper_1904_11563_gb300 import workloads as W
    mask = _mask(W, wl, 0)
    total_t, total_cols = 0.0, 0
    while total_cols == 0 or (total_t < budget_s and total_cols + cols <= wl["N"]):
        total_t += _oracle_sample(A, B, wl["h"], mask, cols, wl)
        total_cols += cols
    return total_t, total_cols


def oracle_single_thread(wl, budget_s=10.0, cols=128):
    """The oracle on one host thread: a child process with every BLAS / OpenMP
    pool limited to one thread (set before numpy loads), inputs of the same
    shapes and distribution from the host generator."""
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", wl["name"],
           "--oracle-sample-seconds", str(budget_s)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout).strip().splitlines()[-1:]}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    useful = 2.0 * wl["M"] * wl["K"] * out["cols"]
    return {"value": useful / out["seconds"] / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle FP64 coded path (numpy BLAS on one thread) on {out['cols']} of {wl['N']} columns "
                      f"of B, same shapes and distribution (host generator), trial mask seed "
                      f"{wl['mask_seed_base']}, {out['seconds']:.1f} s"}


def cpu_baseline(A, B, wl, budget_s=12.0):
    """The oracle as it stands on a bounded column sample of the workload."""
    M, K, N = wl["M"], wl["K"], wl["N"]
    total_t, total_cols = _oracle_timed(A, B, wl, budget_s, 256)
    useful = 2.0 * M * K * total_cols
    return {"value": useful / total_t / 1e12, "unit": "TFLOP/s", "cores": _cores(), "kind": "oracle",
            "sample": f"oracle FP64 coded path (numpy BLAS, all host cores) on {total_cols} of {N} columns of B, "
                      f"trial mask seed {wl['mask_seed_base']}, {total_t:.1f} s",
            "single_thread": oracle_single_thread(wl)}


# ------------------------------------------------------------ replicas (N > 1)
# One process per GPU under torchrun, each an independent replica of the
# whole path (no data-path collective): the ranks meet only at the barriers
# around the timed region, and rank 0 reports the slowest rank's time.

def _world():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))


def _dist_init(backend):
    """Joins the replicas' process group (rendezvous from the MASTER_* env)."""
    world, _rank = _world()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world


def _barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def _max_over_ranks(values, device="cpu"):
    """The element-wise maximum of `values` over all ranks (identity for one
    process): the timed region ends when the slowest replica does."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1904_11563_gb300 import workloads as W
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    A = W.matrix((M, K), wl["dist"], wl["seed"])
    B = W.matrix((K, N), wl["dist"], wl["seed"] + 1)
    cols = 128
    warm = max(args.warmup, 3)
    times = []
    for i in range(warm + args.steps):
        mask = _mask(W, wl, i)
        dt = _oracle_sample(A, B, h, mask, cols, wl)
        if i >= warm:
            times.append(dt)
    tot = sum(times)
    val = 2.0 * M * K * cols * len(times) / tot / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": warm, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(wl),
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"each step: oracle FP64 coded path on {cols} of {N} columns of B"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def run_ours(args, wl):
    import torch
    from paper_1904_11563_gb300 import build as B_
    B_.build()
    from paper_1904_11563_gb300 import bpx
    from paper_1904_11563_gb300 import workloads as W

    world, rank = _world()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    _dist_init("nccl")
    dev = torch.device("cuda", local)
    M, K, N, h = wl["M"], wl["K"], wl["N"], wl["h"]
    code = _lib_code(bpx, wl)
    A, Bm = W.device_inputs(M, K, N, wl["dist"], wl["seed"], device=dev)
    trials = wl.get("trials", 100)
    wl["trials"] = trials
    masks = torch.from_numpy(np.stack([_mask(W, wl, t) for t in range(trials)])).to(dev)
    warm = max(args.warmup, 3)
    steps = args.steps

    # the headline precision
    precs = []
    if args.precisions:
        precs = [x for x in args.precisions.split(",") if x]
    elif args.precision == "auto":
        precs = ["bf16x3", "fp32", "bf16", "mxfp8", "exact", "fp16x3", "bf16x3-fused"]
    else:
        precs = [args.precision] + (["fp32"] if args.precision != "fp32" else [])
    results = {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    gpu_index = local
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if cvd and cvd.split(",")[0].strip().isdigit():
        gpu_index = int(cvd.split(",")[local].strip())

    tuned = {}
    surv_rows = []
    col_cells = np.diff(code.col_ptr)
    for t in range(trials):
        m = _mask(W, wl, t)
        surv_rows.append(int(sum(int(col_cells[j]) for j in range(code.n) if not m[j])) * h)

    for prec in precs:
        # "<precision>-fused": the same precision with the encode fused into the GEMM's operand load
        fused = int(prec.endswith("-fused"))
        P = bpx.PRECISIONS[prec.replace("-fused", "")]
        try:
            ws = bpx.Workspace(code, M, N, K, h, P, device=dev)
        except bpx.BpxError:
            continue
        C = bpx.alloc_C(code, h, N, dev)
        info = torch.zeros(bpx.INFO_LEN, dtype=torch.int32, device=dev)
        cfg = args.gemm_config
        if cfg < 0:
            cfg = 0
            if prec in ("bf16x3", "bf16", "exact", "fp16x3"):
                cfg, _tuned_ms = bpx.autotune(code, A, Bm, h, P, masks[0], ws, C=C)
        tuned[prec] = cfg
        opts = bpx.default_opts(gemm_config=cfg, compensate_depth=args.compensate_depth, fused_encode=fused)
        try:
            for i in range(warm):
                bpx.coded_matmul(code, A, Bm, h, P, masks[i % wl["trials"]], ws, C=C, opts=opts, info=info)
            torch.cuda.synchronize()
        except bpx.BpxError as e:
            if e.code == bpx.ERR_UNSUPPORTED:
                continue
            raise
        sev = StageEvents(bpx, steps)
        clocks = ClockSampler(gpu_index)
        clocks.start()
        time.sleep(0.3)
        _barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        clocks.begin()
        t0.record()
        for i in range(steps):
            o = bpx.default_opts(gemm_config=cfg, compensate_depth=args.compensate_depth, fused_encode=fused)
            o.stage_events = sev.ptr(i)
            bpx.coded_matmul(code, A, Bm, h, P, masks[(warm + i) % wl["trials"]], ws, C=C, opts=o, info=info)
        t1.record()
        torch.cuda.synchronize()
        _barrier()
        ms_serial = t0.elapsed_time(t1)
        inf = info.cpu().numpy()
        assert inf[bpx.INFO_STATUS] == bpx.OK, inf
        # The same number of steps with `inflight` of them in flight: step i
        # runs on stream i % inflight with that stream's own workspace, C and
        # info words, so one step's HBM-bound stages (schedule, B split,
        # encode, peel) run beside another step's tensor-core GEMM.  Every
        # step does all of its work; only the order in time changes.
        ms = ms_serial
        C_last = C
        nf = max(1, args.inflight)
        if nf > 1:
            slots = [dict(ws=ws, C=C, info=info, stream=torch.cuda.Stream(device=dev))]
            for _ in range(nf - 1):
                slots.append(dict(ws=bpx.Workspace(code, M, N, K, h, P, device=dev), C=bpx.alloc_C(code, h, N, dev),
                                  info=torch.zeros(bpx.INFO_LEN, dtype=torch.int32, device=dev),
                                  stream=torch.cuda.Stream(device=dev)))
            cur = torch.cuda.current_stream()

            def _pipelined(first, count):
                for sl in slots:
                    sl["stream"].wait_stream(cur)
                for i in range(count):
                    sl = slots[i % nf]
                    with torch.cuda.stream(sl["stream"]):
                        bpx.coded_matmul(code, A, Bm, h, P, masks[(first + i) % wl["trials"]], sl["ws"], C=sl["C"],
                                         opts=opts, info=sl["info"])
                for sl in slots:
                    cur.wait_stream(sl["stream"])

            _pipelined(0, max(warm, nf))
            torch.cuda.synchronize()
            _barrier()
            torch.cuda.synchronize()
            t0.record()
            _pipelined(warm, steps)
            t1.record()
            torch.cuda.synchronize()
            _barrier()
            ms = t0.elapsed_time(t1)
            for sl in slots:
                si = sl["info"].cpu().numpy()
                assert si[bpx.INFO_STATUS] == bpx.OK and si[bpx.INFO_DEVICE_ERR] == 0, si
            C_last = slots[(steps - 1) % nf]["C"]  # the last timed step's output (error report)
            del slots
        clocks.end()
        ms, ms_serial = _max_over_ranks([ms, ms_serial], device=dev)
        stage = {}
        recorded = ["schedule", "a_prep", "gemm", "peel"] + (["b_prep"] if prec != "fp32" else [])
        # (the autotuner covers the bf16 tensor-core kernels only)
        for si, nm in enumerate(bpx.STAGE_NAMES):
            if nm not in recorded:
                continue
            vals = [sev.stage_ms(i, si) for i in range(steps)]
            vals = [v for v in vals if v is not None and v > 0]
            stage[nm] = sum(vals) / len(vals) if vals else 0.0
        rows_t = [surv_rows[(warm + i) % wl["trials"]] for i in range(steps)]
        ck = clocks.stop()
        results[prec] = dict(ms=ms / steps, ms_serial=ms_serial / steps, stage=stage, clocks=ck, ws=ws, C=C_last,
                             rows=rows_t)

    if not results:
        raise RuntimeError("no precision could run")
    head = "bf16x3" if "bf16x3" in results else list(results)[0]
    useful = 2.0 * M * N * K
    R = results[head]
    value = world * useful / (R["ms"] * 1e-3) / 1e12

    # relative error per block on sampled sources vs FP64 A_s B (numpy), the
    # depths taken from the library's own plan for the last timed mask
    rel = {}
    last_mask = torch.from_numpy(_mask(W, wl, warm + steps - 1)).to(dev)
    ws_s = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32, device=dev)
    order, _rec, _inf = bpx.schedule(code, last_mask, ws_s)
    order = order.cpu().numpy()
    depth = {int(s_): int(d_) for s_, _r, d_ in order if s_ >= 0}
    if rank == 0:
        Ah = A.cpu().numpy()
        Bh = Bm.cpu().numpy().astype(np.float64)
        deep = sorted(depth, key=lambda s_: -depth[s_])[:3]
        direct = [s_ for s_ in sorted(depth) if depth[s_] == 1][:1]
        samples = [s_ for s_ in sorted(set(deep + direct)) if (s_ + 1) * h <= M]
        refs = {s_: Ah[s_ * h:(s_ + 1) * h].astype(np.float64) @ Bh for s_ in samples}
        nu = _propagation(code, order, Ah, Bh, h, samples)
        for prec, r in results.items():
            Cn = r["C"]
            errs = []
            for s_ in samples:
                blk = Cn[s_ * h:(s_ + 1) * h].double().cpu().numpy()
                errs.append(float(np.linalg.norm(blk - refs[s_]) / np.linalg.norm(refs[s_])))
            direct_err = [e_ for e_, s_ in zip(errs, samples) if depth[s_] == 1]
            scaled = [e_ / max(1.0, nu[s_]) for e_, s_ in zip(errs, samples)]
            rel[prec] = {"max": max(errs), "max_direct": max(direct_err) if direct_err else None,
                         "max_nu_scaled": max(scaled), "tol": TOL.get(prec),
                         "sources": samples, "depths": [depth[s_] for s_ in samples], "errs": errs,
                         "nu": [nu[s_] for s_ in samples],
                         "reference": "FP64 A_s B (numpy) for the deepest and one direct source; nu_s from "
                                      "the plan's integer expansion and FP64 product norms on 256 columns"}

    # decode GB/s: per non-direct source, read the resolver's product and the
    # other blocks it subtracts, write C_s: (deg(resolver) + 1) h N 4 bytes
    peel_bytes = []
    deg = np.diff(code.cell_ptr)
    for i in range(steps):
        mk = torch.from_numpy(_mask(W, wl, warm + i)).to(dev)
        od, _r2, _i2 = bpx.schedule(code, mk, ws_s)
        od = od.cpu().numpy()
        peel_bytes.append(sum(int(deg[r_] + 1) * h * N * 4 for s_, r_, d_ in od if s_ >= 0 and d_ >= 2))
    peel_b = float(np.mean(peel_bytes))

    # roofline of the dominant kernel (the coded GEMM)
    import json as _j
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _j.load(open(pk))
    gemm_ms = R["stage"]["gemm"]
    rows_mean = sum(R["rows"]) / len(R["rows"])
    clk = R["clocks"].get("sm_mhz") or 0
    if head != "fp32":
        # tensor-core paths: MMA flops executed per launch (split terms, or
        # the exact path's digit-pair products) against the measured bf16
        # peak (FP8: times the nominal fp8 / bf16 ratio of 2)
        if head == "exact":
            S_ex = bpx.exact_params(code, K)["S"]
            mult = S_ex * (S_ex + 1) // 2
        else:
            mult = MMA_MULT[head]
        flops = 2.0 * rows_mean * N * K * mult
        achieved = flops / (gemm_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops", 1900.0) * (2.0 if head == "mxfp8" else 1.0)
        src = "measured bf16 burst (MEASURED_PEAKS.json)" if peaks else "fallback"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": _traffic(wl["name"], head, tuned.get(head)),
                "peak_source": src + (" x 2 (nominal fp8/bf16)" if head == "mxfp8" else ""),
                "kernel": "coded tcgen05 GEMM" + (" (block-scaled MXFP8)" if head == "mxfp8" else ""),
                "work_per_launch": "2 x coded rows x N x K x %d MMA flops" % mult}
    else:
        flops = 2.0 * rows_mean * N * K
        achieved = flops / (gemm_ms * 1e-3) / 1e12
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": f"FFMA: {sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz",
                "kernel": "coded FP32 SIMT GEMM", "work_per_launch": "2 x coded rows x N x K"}
    # decode GB/s: compulsory bytes of the peel (read each non-direct
    # resolver's product and every other block it subtracts, write C_s)
    peel_ms = R["stage"]["peel"]

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": steps,
            "warmup": warm, "ms_per_step": R["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": head, "data": "synthetic", "config": _config(wl)}
    line["ms_per_step_serial"] = R["ms_serial"]
    line["serial_tflops"] = world * useful / (R["ms_serial"] * 1e-3) / 1e12
    line["config"]["launch"] = (
        "%d steps in flight on %d streams (each its own workspace, C and info words); stage times and "
        "the roofline from the same steps run one at a time" % (max(1, args.inflight), max(1, args.inflight))
        if args.inflight > 1 else "one step at a time")
    if args.compensate_depth >= 0:
        line["config"]["compensate_depth"] = args.compensate_depth
    line["stages_ms"] = R["stage"]
    line["stages_ms_by_precision"] = {p_: r_["stage"] for p_, r_ in results.items()}
    line["gemm_config"] = tuned
    for prec, r in results.items():
        line[f"{prec}_tflops"] = world * useful / (r["ms"] * 1e-3) / 1e12
        line[f"{prec}_ms_per_step"] = r["ms"]
        line[f"{prec}_ms_per_step_serial"] = r["ms_serial"]
    if "bf16x3" in results and "fp32" in results:
        line["speedup_bf16x3_vs_fp32"] = results["fp32"]["ms"] / results["bf16x3"]["ms"]
    line["rel_err"] = rel
    # each precision's largest sampled block error, flat and divided by the
    # block's propagation factor, against its stated tolerance
    line["block_err"] = {p_: {"flat_max": r_["max"], "nu_scaled_max": r_["max_nu_scaled"], "tol": r_["tol"],
                              "flat_within_tol": (r_["max"] <= r_["tol"]) if r_["tol"] else None}
                         for p_, r_ in rel.items()}
    # the accuracy target: >= 4x the plain FP32 coded path at <= 1e-5 on
    # every block, flat; which split path meets it
    if "fp32" in results and rel:
        tgt = {}
        for p_ in ("bf16x3", "fp16x3"):
            if p_ in results and p_ in rel:
                tgt[p_] = {"tflops": line[f"{p_}_tflops"], "x_fp32": results["fp32"]["ms"] / results[p_]["ms"],
                           "flat_max_rel_err": rel[p_]["max"],
                           "meets": bool(rel[p_]["max"] <= 1e-5 and results["fp32"]["ms"] / results[p_]["ms"] >= 4.0)}
        line["accuracy_target"] = tgt
    line["roofline"] = roof
    # every precision's GEMM against its own peak (FP8: the measured bf16 peak
    # times the nominal fp8 / bf16 ratio of 2)
    gr = {}
    for prec, r in results.items():
        gm = r["stage"].get("gemm", 0.0)
        rows_m = sum(r["rows"]) / len(r["rows"])
        if gm <= 0:
            continue
        if prec == "fp32":
            mhz = peaks.get("sm_max_mhz", 2070.0)
            pk, unit = sms * 128 * 2 * mhz * 1e6 / 1e12, "FFMA"
            work = 2.0 * rows_m * N * K
        else:
            if prec == "exact":
                S_ex = bpx.exact_params(code, K)["S"]
                mult = S_ex * (S_ex + 1) // 2     # digit pairs (i, l) with i + l < S
            else:
                mult = MMA_MULT[prec]
            pk = peaks.get("bf16_tflops", 1900.0) * (2.0 if prec == "mxfp8" else 1.0)
            unit = "measured bf16 burst" + (" x 2 (nominal fp8/bf16)" if prec == "mxfp8" else "")
            work = 2.0 * rows_m * N * K * mult
        ach = work / (gm * 1e-3) / 1e12
        gr[prec] = {"achieved_tflops": ach, "peak_tflops": pk, "frac": ach / pk, "peak": unit, "gemm_ms": gm}
    line["gemm_roofline"] = gr
    line["peel_ms"] = peel_ms
    hbm = peaks.get("hbm_gbs", 6800.0)
    line["decode"] = {"bytes_per_step": peel_b, "ms": peel_ms,
                      "gbs": peel_b / (peel_ms * 1e-3) / 1e9 if peel_ms > 0 else None,
                      "frac_hbm": (peel_b / (peel_ms * 1e-3) / 1e9) / hbm if peel_ms > 0 else None,
                      "bytes_def": "sum over non-direct sources of (deg(resolver)+1) h N 4"}
    # the HBM-bound staging stages against their compulsory bytes: the
    # encode reads A once and writes the coded rows (bf16 hi + lo: 4 B per
    # element, or FP32: 4 B), the B split reads B and writes B^T hi + lo
    def _hbm(nbytes, ms, what):
        gbs = nbytes / (ms * 1e-3) / 1e9 if ms and ms > 0 else None
        return {"bytes_per_step": nbytes, "ms": ms, "gbs": gbs, "frac_hbm": gbs / hbm if gbs else None,
                "bytes_def": what}
    st_ = R["stage"]
    if head in ("bf16x3", "bf16", "fp32"):
        out_b = 4 if head in ("bf16x3", "fp32") else 2
        line["encode"] = _hbm(4.0 * M * K + out_b * rows_mean * K, st_.get("a_prep", 0.0),
                              "read A once (4 M K) + write the coded rows (%d B per element)" % out_b)
    if head in ("bf16x3", "bf16"):
        line["b_split"] = _hbm(4.0 * K * N + (4 if head == "bf16x3" else 2) * K * N, st_.get("b_prep", 0.0),
                               "read B (4 K N) + write B^T hi (+ lo) bf16")
    line["clocks"] = R["clocks"]
    per_step = {"bf16x3": 5, "bf16": 5, "mxfp8": 5, "fp32": 4, "exact": 7, "fp16x3": 7, "bf16x3-fused": 4}[head]
    if head == "fp16x3" and len(code.cell_src) >= 4 * code.num_cells:
        per_step += 2  # the K-chunked encode of high-degree codes: three kernels instead of one
    line["gpu_launches"] = per_step * steps

    # end to end through the host entry points (pinned host buffers): every
    # step copies its A, B and mask in and its C and info words out inside the
    # timed region.  "e2e": bpx_coded_matmul_host_async with three steps in
    # flight (three streams, each with its own device buffers and workspace),
    # so one step's copies overlap the others' kernels; "e2e_sync": one
    # synchronous bpx_coded_matmul_host call per step.
    if not args.no_e2e and rank == 0:
        P = bpx.PRECISIONS[head]
        o_e2e = bpx.default_opts(gemm_config=tuned.get(head, 0), compensate_depth=args.compensate_depth)
        hA = A.cpu().pin_memory()
        hB = Bm.cpu().pin_memory()
        hmasks = [torch.from_numpy(_mask(W, wl, t)).pin_memory() for t in range(wl["trials"])]
        ws0, dC0 = R["ws"], R["C"]
        for p_, r_ in list(results.items()):
            if p_ != head:      # free the other precisions' buffers
                r_["ws"] = r_["C"] = None
        torch.cuda.empty_cache()
        e2e_steps = max(10, steps)
        nflight = max(1, args.e2e_inflight)
        sets = []
        for j in range(nflight):
            sets.append(dict(
                dA=torch.empty_like(A), dB=torch.empty_like(Bm),
                dmask=torch.empty(code.n, dtype=torch.uint8, device=dev),
                dC=dC0 if j == 0 else bpx.alloc_C(code, h, N, dev),
                ws=ws0 if j == 0 else bpx.Workspace(code, M, N, K, h, P, device=dev),
                hC=torch.empty((M, N), dtype=torch.float32).pin_memory(),
                hinfo=torch.zeros(bpx.INFO_LEN, dtype=torch.int32).pin_memory(),
                dinfo=torch.zeros(bpx.INFO_LEN, dtype=torch.int32, device=dev),
                stream=torch.cuda.Stream(device=dev)))

        def _enqueue(i):
            S_ = sets[i % nflight]
            bpx.coded_matmul_host_async(code, hA, hB, h, P, hmasks[i % wl["trials"]], S_["hC"], S_["dA"], S_["dB"],
                                        S_["dmask"], S_["dC"], S_["ws"], S_["hinfo"], opts=o_e2e,
                                        stream=S_["stream"])

        def _drain():
            for S_ in sets:
                S_["stream"].synchronize()
                assert int(S_["hinfo"][bpx.INFO_STATUS]) == bpx.OK and int(S_["hinfo"][bpx.INFO_DEVICE_ERR]) == 0

        torch.cuda.synchronize()
        for i in range(2 * nflight):
            _enqueue(i)
        _drain()
        t_s = time.perf_counter()
        for i in range(e2e_steps):
            _enqueue(i)
        _drain()
        dt = (time.perf_counter() - t_s) / e2e_steps
        h2d = 4 * (M * K + K * N) + code.n
        d2h = 4 * M * N + 4 * bpx.INFO_LEN
        line["e2e"] = {"value": useful / dt / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3,
                       "api": "bpx_coded_matmul_host_async, %d steps in flight (separate streams, buffers, "
                              "workspaces)" % nflight, "steps": e2e_steps}
        # The same host-link traffic without the computation -- the floor the
        # link puts under "e2e": every step's copies in (A, B, the mask) on one
        # stream and out (C, the info words) on another, so that both
        # directions stay busy as they do between the pipelined steps.
        s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

        def _copies(i):
            S_ = sets[i % nflight]
            with torch.cuda.stream(s_in):
                S_["dA"].copy_(hA, non_blocking=True)
                S_["dB"].copy_(hB, non_blocking=True)
                S_["dmask"].copy_(hmasks[i % wl["trials"]], non_blocking=True)
            with torch.cuda.stream(s_out):
                S_["hC"].copy_(S_["dC"][:M], non_blocking=True)
                S_["hinfo"].copy_(S_["dinfo"], non_blocking=True)

        for i in range(nflight):
            _copies(i)
        torch.cuda.synchronize()
        t_s = time.perf_counter()
        for i in range(e2e_steps):
            _copies(i)
        torch.cuda.synchronize()
        dtc = (time.perf_counter() - t_s) / e2e_steps
        line["e2e"]["link_only_ms_per_step"] = dtc * 1e3
        line["e2e"]["link_only_note"] = ("the same copies without the computation, host-to-device on one stream and "
                                         "device-to-host on another (both directions busy): the host link's floor "
                                         "under the end-to-end step")
        S0 = sets[0]
        with torch.cuda.stream(S0["stream"]):
            for i in range(2):
                bpx.coded_matmul_host(code, hA, hB, h, P, hmasks[i], S0["hC"], S0["dA"], S0["dB"], S0["dmask"],
                                      S0["dC"], S0["ws"], opts=o_e2e)
            t_s = time.perf_counter()
            for i in range(e2e_steps):
                rc, _ = bpx.coded_matmul_host(code, hA, hB, h, P, hmasks[i % wl["trials"]], S0["hC"], S0["dA"],
                                              S0["dB"], S0["dmask"], S0["dC"], S0["ws"], opts=o_e2e)
                assert rc == bpx.OK
            dts = (time.perf_counter() - t_s) / e2e_steps
        line["e2e_sync"] = {"value": useful / dts / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                            "d2h_bytes_per_step": d2h, "ms_per_step": dts * 1e3, "api": "bpx_coded_matmul_host"}
        del sets
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        Ah = A.cpu().numpy()
        Bh = Bm.cpu().numpy()
        line["cpu_baseline"] = cpu_baseline(Ah, Bh, wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """512 independent coded multiplications (M, N, K log-uniform on
    256..4096, multiples of 128): one grouped split-BF16x3 run per step,
    replayed from a CUDA graph, against per-job plain FP32 launches."""
    import torch
    from paper_1904_11563_gb300 import build as B_
    B_.build()
    from paper_1904_11563_gb300 import bpx
    from paper_1904_11563_gb300 import workloads as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    specs = W.batch_specs(args.jobs, 5)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    jobs = []
    for sp in specs:
        kind, *a = sp["code"]
        code = {"table1": bpx.Code.table1, "table3": bpx.Code.table3,
                "systematic": lambda: bpx.Code.systematic(*a), "mojette_a": lambda: bpx.Code.mojette_a(*a)}[kind]()
        A = torch.rand((sp["M"], sp["K"]), generator=g, device=dev).mul_(2).sub_(1)
        Bm = torch.rand((sp["K"], sp["N"]), generator=g, device=dev).mul_(2).sub_(1)
        m = torch.from_numpy(W.erasure_mask(code.n, sp["e"], sp["mask_seed"])).to(dev)
        jobs.append(dict(code=code, A=A, B=Bm, C=bpx.alloc_C(code, sp["h"], sp["N"], dev), mask=m,
                         info=torch.zeros(16, dtype=torch.int32, device=dev), h=sp["h"]))
    useful = sum(2.0 * sp["M"] * sp["N"] * sp["K"] for sp in specs)
    G = bpx.Group(jobs, bpx.BF16X3, device=dev)
    best, best_ms = G.autotune()
    peel_target, peel_tuned_ms = G.autotune_peel()
    stream = torch.cuda.Stream(device=dev)
    warm = max(args.warmup, 3)
    steps = args.steps
    with torch.cuda.stream(stream):
        for _ in range(warm):
            G.graph_launch()
        stream.synchronize()
        clocks = ClockSampler(dev.index)
        clocks.start()
        time.sleep(0.3)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        clocks.begin()
        t0.record(stream)
        for _ in range(steps):
            G.graph_launch()
        t1.record(stream)
        stream.synchronize()
        clocks.end()
        ck = clocks.stop()
    ms = t0.elapsed_time(t1) / steps
    ok = all(int(j["info"][bpx.INFO_STATUS].item()) == bpx.OK for j in jobs)
    # stage breakdown of one non-graph run
    sev = StageEvents(bpx, 1)
    o = bpx.default_opts()
    o.stage_events = sev.ptr(0)
    G.run(opts=o)
    torch.cuda.synchronize()
    stage = {nm: sev.stage_ms(0, si) for si, nm in enumerate(bpx.STAGE_NAMES)}
    # baselines: per-job launches, plain FP32 and split-BF16x3 (not grouped)
    base = {}
    for prec in ("fp32", "bf16x3"):
        P = bpx.PRECISIONS[prec]
        wss = [bpx.Workspace(j["code"], j["A"].shape[0], j["B"].shape[1], j["A"].shape[1], j["h"], P, device=dev)
               for j in jobs]
        for j, ws in zip(jobs, wss):
            bpx.coded_matmul(j["code"], j["A"], j["B"], j["h"], P, j["mask"], ws, C=j["C"], info=j["info"])
        torch.cuda.synchronize()
        t0.record()
        reps = 1 if prec == "fp32" else 3
        for _ in range(reps):
            for j, ws in zip(jobs, wss):
                bpx.coded_matmul(j["code"], j["A"], j["B"], j["h"], P, j["mask"], ws, C=j["C"], info=j["info"])
        t1.record()
        torch.cuda.synchronize()
        base[prec] = t0.elapsed_time(t1) / reps
        del wss
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    rows = 0
    for j in jobs:
        col_cells = np.diff(j["code"].col_ptr)
        mk = j["mask"].cpu().numpy()
        rows += sum(int(col_cells[c]) for c in range(j["code"].n) if not mk[c]) * j["h"] * j["B"].shape[1] * j["A"].shape[1]
    mma = 2.0 * rows * 3
    gemm_ms = stage["gemm"]
    line = {"metric": METRIC, "value": useful / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": "batch512", "code": CODE_TEXT["batch512"], "jobs": args.jobs,
                       "dims": "M, N, K = 128 * round(x / 128), x log-uniform on [256, 4096], seeded",
                       "inputs": "A, B iid U(-1,1) FP32, seeded", "useful_tflop_per_batch": useful / 1e12,
                       "launch": "one grouped run per step replayed from a CUDA graph",
                       "peel_ctas_per_job": peel_target,
                       "gemm_config": best, "l2": "inputs larger than L2"},
            "all_ok": ok, "stages_ms": stage,
            "per_job_fp32_ms": base["fp32"], "per_job_bf16x3_ms": base["bf16x3"],
            "speedup_vs_per_job_fp32": base["fp32"] / ms, "speedup_vs_per_job_bf16x3": base["bf16x3"] / ms,
            "roofline": {"bound": "tensor", "achieved": mma / (gemm_ms * 1e-3) / 1e12,
                         "peak": peaks.get("bf16_tflops", 1900.0), "unit": "TFLOP/s",
                         "frac": mma / (gemm_ms * 1e-3) / 1e12 / peaks.get("bf16_tflops", 1900.0),
                         "traffic": None, "kernel": "grouped tcgen05 GEMM (one non-graph run)"},
            "clocks": ck, "gpu_launches": 5 * steps}
    print(json.dumps(line), flush=True)


def run_2d(args, wl):
    """The paper's two-dimensional scheme on the benchmark code: C's 8 x 8
    blocks of 1024 x 1024 are the sources, cells sum block products; one
    step = schedule, operand staging, coded products, peel."""
    import torch
    from paper_1904_11563_gb300 import build as B_
    B_.build()
    from paper_1904_11563_gb300 import bpx
    from paper_1904_11563_gb300 import workloads as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    code = _lib_code(bpx, wl)
    M, N, K, h = wl["M"], wl["N"], wl["K"], wl["h"]
    w = N // code.k
    A, Bm = W.device_inputs(M, K, N, wl["dist"], wl["seed"], device=str(dev))
    masks = torch.from_numpy(np.stack([_mask(W, wl, t) for t in range(wl["trials"])])).to(dev)
    prec = args.precision if args.precision in ("bf16", "bf16x3") else "bf16x3"
    P = bpx.PRECISIONS[prec]
    ws = bpx.Workspace2D(code, M, N, K, h, P, device=dev)
    C = torch.zeros((code.b * h, N), dtype=torch.float32, device=dev)
    info = torch.zeros(bpx.INFO_LEN, dtype=torch.int32, device=dev)
    opts = bpx.default_opts(gemm_config=args.gemm_config)
    warm, steps = max(args.warmup, 3), args.steps
    for i in range(warm):
        bpx.coded_matmul_2d(code, A, Bm, h, P, masks[i % wl["trials"]], ws, C=C, opts=opts, info=info)
    torch.cuda.synchronize()
    sev = StageEvents(bpx, steps)
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks.begin()
    t0.record()
    for i in range(steps):
        o_ = bpx.default_opts(gemm_config=args.gemm_config)
        o_.stage_events = sev.ptr(i)
        bpx.coded_matmul_2d(code, A, Bm, h, P, masks[(warm + i) % wl["trials"]], ws, C=C, opts=o_, info=info)
    t1.record()
    torch.cuda.synchronize()
    clocks.end()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1) / steps
    assert int(info[bpx.INFO_STATUS].item()) == bpx.OK
    stage = {}
    for si, nm in enumerate(bpx.STAGE_NAMES):
        vals = [v for v in (sev.stage_ms(i, si) for i in range(steps)) if v]
        if vals:
            stage[nm] = sum(vals) / len(vals)
    # executed MMA work: every surviving cell's products (T_c of them) of
    # h x w x K, times 3 for split-BF16x3
    per, summ = bpx.terms_2d(code)
    col_of = np.repeat(np.arange(code.n), np.diff(code.col_ptr))
    mult = 3 if prec == "bf16x3" else 1
    mma = []
    for i in range(steps):
        mk = masks[(warm + i) % wl["trials"]].cpu().numpy()
        mma.append(sum(int(per[c]) for c in range(code.num_cells) if not mk[col_of[c]]) * 2.0 * h * w * K * mult)
    mma_mean = float(np.mean(mma))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = mma_mean / (stage["gemm"] * 1e-3) / 1e12
    useful = 2.0 * M * N * K
    # relative error of the deepest blocks and a direct one vs FP64 A_z B_l
    last = masks[(warm + steps - 1) % wl["trials"]]
    order, _r, _i = bpx.schedule(code, last, bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32, device=dev))
    order = order.cpu().numpy()
    depth = {int(s_): int(d_) for s_, _r2, d_ in order if s_ >= 0}
    samples = sorted(depth, key=lambda s_: -depth[s_])[:2] + [s_ for s_ in sorted(depth) if depth[s_] == 1][:1]
    Ah, Bh = A.cpu().numpy(), Bm.cpu().numpy()
    errs = []
    for s_ in samples:
        z, l = divmod(s_, code.k)
        r = Ah[z * h:(z + 1) * h].astype(np.float64) @ Bh[:, l * w:(l + 1) * w].astype(np.float64)
        c = C[z * h:(z + 1) * h, l * w:(l + 1) * w].double().cpu().numpy()
        errs.append(float(np.linalg.norm(c - r) / np.linalg.norm(r)))
    line = {"metric": METRIC, "value": useful / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": wl["name"], "code": CODE_TEXT[wl["name"]], "M": M, "N": N, "K": K, "h": h, "w": w,
                       "erasures": wl["e"], "trials": wl["trials"], "inputs": "A, B iid N(0,1) FP32, seeded",
                       "l2": "inputs larger than L2 (A 268 MB; no flush)"},
            "stages_ms": stage, "terms_2d": summ, "executed_over_useful": mma_mean / mult / useful,
            "rel_err": {"sources": samples, "depths": [depth[s_] for s_ in samples], "errs": errs},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "tcgen05 GEMM over each cell's products (two-dimensional scheme)",
                         "work_per_launch": "sum over surviving cells of T_c x 2 h w K x %d MMA flops" % mult},
            "clocks": ck, "gpu_launches": 5 * steps}
    print(json.dumps(line), flush=True)


def run_straggler(args, wl):
    """Processor-level stragglers (Section IV): every step draws the cells'
    task times, finds the first decodable arrival set (online peel on the
    host) and runs the whole GPU path on exactly those cells (cell-level
    mask).  value = useful 2MNK / GPU step time; the model's parallel task
    time T_par = min over decodable sets of the latest arrival is reported
    beside it (units of 1 / mu)."""
    import torch
    from paper_1904_11563_gb300 import build as B_
    B_.build()
    from paper_1904_11563_gb300 import bpx
    from paper_1904_11563_gb300 import straggler as st
    from paper_1904_11563_gb300 import workloads as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    code = _lib_code(bpx, wl)
    M, N, K, h = wl["M"], wl["N"], wl["K"], wl["h"]
    A, Bm = W.device_inputs(M, K, N, wl["dist"], wl["seed"], device=str(dev))
    prec = args.precision if args.precision in ("bf16", "bf16x3", "fp16x3", "fp32", "exact") else "bf16x3"
    P = bpx.PRECISIONS[prec]
    ws = bpx.Workspace(code, M, N, K, h, P, device=dev)
    C = bpx.alloc_C(code, h, N, dev)
    info = torch.zeros(bpx.INFO_LEN, dtype=torch.int32, device=dev)
    warm, steps = max(args.warmup, 3), args.steps
    plans = []
    for i in range(warm + steps):
        X = W.exponential_draws(code.num_cells, wl["mu"], wl["mask_seed_base"] + i)
        T = st.task_times(code, X)
        order, first, t_par, _rec = st.arrivals(code, T)
        mask = np.ones(code.num_cells, dtype=np.uint8)
        mask[order[:first]] = 0
        plans.append(dict(mask=torch.from_numpy(mask).to(dev), first=first, t_par=t_par, order=order))
    col_of = np.repeat(np.arange(code.n), np.diff(code.col_ptr))
    o_ = bpx.default_opts(mask_cells=1)
    for i in range(warm):
        bpx.coded_matmul(code, A, Bm, h, P, plans[i]["mask"], ws, C=C, opts=o_, info=info)
    torch.cuda.synchronize()
    sev = StageEvents(bpx, steps)
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks.begin()
    t0.record()
    for i in range(steps):
        oi = bpx.default_opts(mask_cells=1)
        oi.stage_events = sev.ptr(i)
        bpx.coded_matmul(code, A, Bm, h, P, plans[warm + i]["mask"], ws, C=C, opts=oi, info=info)
    t1.record()
    torch.cuda.synchronize()
    clocks.end()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1) / steps
    assert int(info[bpx.INFO_STATUS].item()) == bpx.OK
    stage = {}
    for si, nm in enumerate(bpx.STAGE_NAMES):
        vals = [v for v in (sev.stage_ms(i, si) for i in range(steps)) if v]
        if vals:
            stage[nm] = sum(vals) / len(vals)
    timed = plans[warm:]
    useful = 2.0 * M * N * K
    rows = [int((p_["mask"] == 0).sum().item()) * h for p_ in timed]
    if prec == "exact":
        S_ex = bpx.exact_params(code, K)["S"]
        mult = S_ex * (S_ex + 1) // 2     # digit pairs (i, l) with i + l < S
    else:
        mult = {"bf16x3": 3, "fp16x3": 3, "bf16": 1, "fp32": 1}[prec]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    ach = 2.0 * float(np.mean(rows)) * N * K * mult / (stage["gemm"] * 1e-3) / 1e12
    if prec != "fp32":
        pk = peaks.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": None, "kernel": "coded tcgen05 GEMM",
                "work_per_launch": "2 x coded rows x N x K x %d MMA flops" % mult}
    else:
        mhz = peaks.get("sm_max_mhz", 2070.0)
        pk = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": None, "kernel": "coded FP32 SIMT GEMM", "work_per_launch": "2 x coded rows x N x K"}
    H = sum(1.0 / j for j in range(1, code.num_cells + 1))
    # How much of the peel could have overlapped the products (outside the
    # timed region, on the first timed steps): the decodable set's arrivals in
    # eight runs; per run, the peel positions the plan could run once it is
    # in, and the sources an arrival-ordered peel would recover with it.
    nch = 8
    ws_s = bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32, device=dev)
    ready, online = np.zeros(nch), np.zeros(nch)
    sample = timed[:min(3, len(timed))]
    for p_ in sample:
        po, _r, _i = bpx.schedule(code, p_["mask"], ws_s, cells=True)
        ready += st.overlap_bound(code, p_["order"], p_["first"], po.cpu().numpy(), nch)
        online += st.online_recovery(code, p_["order"], p_["first"], ws_s, nch, device=dev)
    ready, online = ready / len(sample), online / len(sample)
    before = float(ready[:-1].sum() / max(1.0, ready.sum()))
    overlap = {"chunks": nch, "steps_sampled": len(sample),
               "peel_positions_ready_by_chunk": [round(float(x), 1) for x in ready],
               "peel_positions_ready_before_last_chunk": before,
               "online_sources_recovered_by_chunk": [round(float(x), 1) for x in online],
               "online_recovered_before_last_chunk": float(online[:-1].sum() / max(1.0, online.sum())),
               "peel_ms": stage.get("peel", 0.0),
               "peel_ms_overlappable_bound": stage.get("peel", 0.0) * before,
               "note": "peel positions (non-direct) by the arrival run after which the plan could run them "
                       "(their resolver's product and every block they subtract are in); the GPU runs all "
                       "arrived products in one launch and the peel after them"}
    line = {"metric": METRIC, "value": useful / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": wl["name"], "code": CODE_TEXT[wl["name"]], "M": M, "N": N, "K": K, "h": h,
                       "mu": wl["mu"], "task_time_seeds": "%d + step" % wl["mask_seed_base"],
                       "inputs": "A, B iid %s FP32, seeded" % {"normal": "N(0,1)", "uniform": "U(-1,1)"}.get(
                           wl["dist"], wl["dist"]), "l2": "inputs larger than L2"},
            "stages_ms": stage, "overlap": overlap,
            "model": {"t_par_mean": float(np.mean([p_["t_par"] for p_ in timed])),
                      "arrivals_to_decode_mean": float(np.mean([p_["first"] for p_ in timed])),
                      "cells": code.num_cells,
                      "t_all_cells_expected_unscaled": H / wl["mu"],
                      "units": "1 / mu; T_c = sigma_c X_c"},
            "computed_cells_mean": float(np.mean(rows)) / h,
            "roofline": roof, "clocks": ck,
            "gpu_launches": ({"bf16x3": 5, "bf16": 5, "fp16x3": 7, "fp32": 4, "exact": 7}[prec]
                             + (2 if prec == "fp16x3" and len(code.cell_src) >= 4 * code.num_cells else 0)) * steps}
    print(json.dumps(line), flush=True)


def run_bsweep(args, wl):
    """Construction A n = 32, k = 24, e = 8 at every grid height b of the
    sweep: the worst-case overhead eps against the conditioning of the peel
    (depth, nu_s, kappa_s), and every precision's relative error per depth
    against FP64 A_s B, with its useful TFLOP/s (one seeded mask per b)."""
    import torch
    from paper_1904_11563_gb300 import build as B_
    B_.build()
    from paper_1904_11563_gb300 import bpx
    from paper_1904_11563_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    K, N, h = wl["K"], wl["N"], 1
    precs = [p_ for p_ in (args.precisions.split(",") if args.precisions else
                           ["fp32", "bf16x3", "fp16x3", "mxfp8", "exact"]) if p_]
    sweep = []
    head_tflops = None
    for b in wl["bs"]:
        code = bpx.Code.mojette_a(32, 24, b)
        S = code.num_sources
        M = S
        A, Bm = W.device_inputs(M, K, N, wl["dist"], wl["seed"], device=dev)
        mask = torch.from_numpy(W.erasure_mask(32, wl["e"], wl["mask_seed_base"])).to(dev)
        order, _rec, info = bpx.schedule(code, mask, bpx.Workspace(code, 0, 0, 0, 1, bpx.FP32, device=dev))
        order = order.cpu().numpy()
        assert int(info.cpu()[bpx.INFO_STATUS]) == bpx.OK
        depth = {int(s_): int(d_) for s_, _r, d_ in order if s_ >= 0}
        nsurv = int(info.cpu()[bpx.INFO_SURVIVING])
        # up to three sources per depth bucket [2^i, 2^(i+1))
        buckets = {}
        for s_ in sorted(depth, key=lambda x: (-depth[x], x)):
            bi = int(np.floor(np.log2(depth[s_])))
            if len(buckets.setdefault(bi, [])) < 3:
                buckets[bi].append(s_)
        samples = sorted(s_ for v_ in buckets.values() for s_ in v_)
        Ah = A.cpu().numpy()
        Bh = Bm.cpu().numpy().astype(np.float64)
        refs = {s_: Ah[s_:s_ + 1].astype(np.float64) @ Bh for s_ in samples}
        nu, kap = {}, {}
        if b <= 64:   # the integer expansion of the deep codes is too large to walk here
            nu = _propagation(code, order, Ah, Bh, h, samples, ncols=N, kappa=kap)
        errs, tflops = {}, {}
        for prec in precs:
            P = bpx.PRECISIONS[prec]
            ws = bpx.Workspace(code, M, N, K, h, P, device=dev)
            C = bpx.alloc_C(code, h, N, dev)
            bpx.coded_matmul(code, A, Bm, h, P, mask, ws, C=C)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(3):
                _C, inf = bpx.coded_matmul(code, A, Bm, h, P, mask, ws, C=C)
            t1.record()
            torch.cuda.synchronize()
            assert int(inf.cpu()[bpx.INFO_STATUS]) == bpx.OK
            tflops[prec] = 2.0 * M * N * K / (t0.elapsed_time(t1) / 3 * 1e-3) / 1e12
            Cn = C.double().cpu().numpy()
            errs[prec] = {s_: float(np.linalg.norm(Cn[s_] - refs[s_]) / np.linalg.norm(refs[s_])) for s_ in samples}
            del ws, C
        by_depth = []
        for bi in sorted(buckets):
            ss = buckets[bi]
            row = {"depths": [2 ** bi, 2 ** (bi + 1) - 1], "sources": ss,
                   "err_max": {p_: max(errs[p_][s_] for s_ in ss) for p_ in precs}}
            if nu:
                row["nu_max"] = max(nu[s_] for s_ in ss)
                row["kappa_max"] = max(kap[s_] for s_ in ss)
            by_depth.append(row)
        ent = {"b": b, "sources": S, "cells": code.num_cells, "surviving_cells": nsurv,
               "eps": code.eps, "coded_rows_over_sources": nsurv / S, "max_depth": max(depth.values()),
               "useful_tflops": tflops, "by_depth": by_depth}
        if not nu:
            ent["nu_kappa"] = "not computed (integer expansion over hundreds of waves; its coefficients reach ~1e26)"
        sweep.append(ent)
        if b == max(wl["bs"]):
            head_tflops = tflops.get("bf16x3")
        del A, Bm
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": head_tflops, "unit": "TFLOP/s", "n_gpus": 1, "steps": 3, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3",
            "data": "synthetic",
            "config": {"workload": "mojA_bsweep", "code": CODE_TEXT["mojA_bsweep"], "K": K, "N": N, "h": 1,
                       "inputs": "U(-1,1) FP32, seed 4; mask seed 4000", "value": "bf16x3 at b = 683",
                       "reference": "FP64 A_s B (numpy) per sampled source"},
            "b_sweep": sweep}
    print(json.dumps(line), flush=True)


def main():
    args = _parse()
    from paper_1904_11563_gb300 import workloads as W
    wl = dict(W.WORKLOADS.get(args.workload, W.WORKLOADS[WORKLOAD]))
    wl["name"] = args.workload
    if args.shape:
        wl["M"], wl["N"], wl["K"] = (int(x) for x in args.shape.split(","))
    if args.oracle_sample_seconds > 0:
        A = W.matrix((wl["M"], wl["K"]), wl["dist"], wl["seed"])
        B = W.matrix((wl["K"], wl["N"]), wl["dist"], wl["seed"] + 1)
        secs, cols = _oracle_timed(A, B, wl, args.oracle_sample_seconds, 128)
        print(json.dumps({"seconds": secs, "cols": cols}), flush=True)
        return
    if args.workload == "batch512":
        run_batch(args)
    elif wl.get("bsweep"):
        if args.impl == "reference":
            raise SystemExit("mojA_bsweep is an error report of this library's paths; no reference arm")
        run_bsweep(args, wl)
    elif wl.get("twod") and args.impl != "reference":
        run_2d(args, wl)
    elif wl.get("straggler") and args.impl != "reference":
        run_straggler(args, wl)
    elif args.impl == "reference":
        if wl.get("twod"):
            raise SystemExit("--impl reference times the one-dimensional workloads only")
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
