#!/usr/bin/env python
"""Bond-update throughput of QR-based TEBD on B300 (one JSON line on stdout).

Workload: one two-site update at chi = 1024, d = 5 (theta of shape (chi, d, d, chi),
complex64, i.i.d. complex Gaussian with unit Frobenius norm, a random 25 x 25
unitary gate, B^n a random right isometry, eta = chi, plain QR truncation),
the single-gate benchmark of Sec. IV / Fig. 5. A step is one full update:
gate, X = theta~ B^n^dag, Householder QR, Y^dag = theta~^dag Q, Householder QR
(the LQ), B~^m = theta~' B~^n^dag, FP64 norms and eps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the update has no exchange step; N ranks run independent replicas
(one process per GPU, NCCL only for the barrier and the max-over-ranks time).
--impl reference times the complex128 CPU oracle on this host's cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QR-TEBD bond updates/s & % TC roofline at χ=1024,d=5 c64; p99 step latency"
UNIT = "bond updates/s"
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate on B300


# FP32 / FP64 CUDA-core peaks of a B300 (148 SMs, 128 FP32 FMA lanes per SM, 2032 MHz
# maximum SM clock; FP64 at the nominal 1.25 TFLOP/s): the denominators of the kernels
# that run on CUDA cores
FP32_ALU_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
FP64_ALU_TFLOPS = 1.25


# DRAM traffic of the panel kernel (k_qr_panel_rf) from one ncu capture
# (profiles/k_qr_panel_chi512.md: complex64, 2464 x 32 panel, 697344 bytes read, 0 written,
# against 3 x 2464 x 32 x 8 algorithmic bytes). Traffic grows with the panel's rows, so a
# launch's traffic is this ratio times its algorithmic bytes.
PANEL_NCU_DRAM_OVER_ALGORITHMIC = 697344 / (3 * 2464 * 32 * 8)


def prof_families(L):
    names = {L.PROF_BOND_GEMM: "bond_gemm", L.PROF_TC_GEMM: "qr_tc_gemm", L.PROF_QR_PANEL: "qr_panel",
             L.PROF_SIMT_GEMM: "simt_gemm", L.PROF_PREP: "tc_prep", L.PROF_GATE: "gate"}
    return list(names), names


def family_roofline(L, fam, ms, n, flops, nbytes, prec, peaks, src):
    """Roofline entry of one kernel family: algorithmic flops (or bytes) per launch over
    the family's average launch duration, against the measured peak of the unit that
    bounds it."""
    sec = ms / 1e3 / n
    tc = prec in (L.C64_3XTF32, L.C64_TF32)
    out = {"launches": n, "launch_ms": ms / n, "traffic": None}
    if fam in (L.PROF_BOND_GEMM, L.PROF_TC_GEMM) and tc:
        # The step is short and mostly latency-bound: its clocks stay at the maximum (see
        # "clocks"), so the burst figure is the denominator; the power-capped sustained one
        # (measured at a median ~1200 MHz over a 4 s GEMM loop) is reported beside it.
        achieved = flops / n / sec / 1e12
        peak = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]) * TF32_PER_BF16
        sus = peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]) * TF32_PER_BF16
        issued = achieved * (3 if prec == L.C64_3XTF32 else 1)
        out.update({"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "issued_frac": issued / peak,
                    "issued_frac_vs_sustained": issued / sus,
                    "kernel": "k_tc_gemm (3xTF32 complex GEMM)" if prec == L.C64_3XTF32 else "k_tc_gemm (TF32)",
                    "peak_source": f"{src} bf16 burst x nominal TF32/BF16 ratio {TF32_PER_BF16:.3f}",
                    "algorithmic_flops_per_launch": flops / n})
    elif fam in (L.PROF_PREP, L.PROF_GATE):
        achieved = nbytes / n / sec / 1e9
        peak = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
        out.update({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": f"{src} copy bandwidth",
                    "kernel": "k_prep (A' and B'^T, one launch)" if fam == L.PROF_PREP else "k_gate",
                    "algorithmic_bytes_per_launch": nbytes / n})
    else:
        achieved = flops / n / sec / 1e12
        peak = FP64_ALU_TFLOPS if L.is_c128(prec) else FP32_ALU_TFLOPS
        out.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "peak_source": "derived CUDA-core peak (SMs x lanes x clock)",
                    "algorithmic_flops_per_launch": flops / n,
                    "kernel": {L.PROF_QR_PANEL: "k_qr_panel_g (grid form; k_qr_panel clusters for short panels)"
                               if L.is_c128(prec) else "k_qr_panel_rf",
                               L.PROF_SIMT_GEMM: "k_apply_wy / k_gemm",
                               L.PROF_BOND_GEMM: "k_gemm", L.PROF_TC_GEMM: "k_gemm"}[fam]})
        if fam == L.PROF_QR_PANEL:
            out["limiter"] = ("FP64 work per CTA (~40 slab rows and the 32 pivot rows) and one grid barrier per column"
                              if L.is_c128(prec) else
                              "latency: one cluster-wide exchange per column (sequential in the column)")
            out["achieved_hbm_gbs"] = nbytes / n / sec / 1e9
            out["algorithmic_bytes_per_launch"] = nbytes / n
            if prec == L.C64_3XTF32:
                out["traffic"] = PANEL_NCU_DRAM_OVER_ALGORITHMIC * nbytes / n
                out["traffic_source"] = "ncu dram bytes of a 2464-row panel, scaled by rows"
    return out


def measure_matmul_peaks(torch):
    """TF32 and FP64 dense peaks measured on this GPU the way MEASURED_PEAKS.json measures
    BF16: torch.matmul, best of several CUDA-event-timed runs (TF32 at 8192^3 with TF32
    tensor cores allowed, FP64 at 4096^3)."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for key, dt, n, reps, tf32 in (("tf32_tflops", torch.float32, 8192, 10, True),
                                        ("fp64_tflops", torch.float64, 4096, 4, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            c = torch.empty(n, n, device="cuda", dtype=dt)
            torch.matmul(a, b, out=c)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[key] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            out[key + "_how"] = f"torch.matmul {n}^3, best of {reps}, CUDA events"
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def update_flops(chi_l, d, chi_m, chi_r, eta, theta_given=True, xi_dense=False):
    """Algorithmic real flops of one plain bond update (8 per complex MAC): the gate, X = theta~ Y0^dag,
    the QR of X (factor + explicit Q), Y = Q^dag theta~, the QR of Y^dag, B~^m = theta~' B~^n^dag,
    plus theta' = B^m B^n and a dense Xi when they are formed."""
    m1, m2 = d * chi_l, d * chi_r
    qr = lambda m, n: 2 * (m * n * n - n ** 3 / 3.0)
    cmac = d ** 4 * chi_l * chi_r + 3 * d * d * chi_l * chi_r * eta + qr(m1, eta) + qr(m2, eta)
    if not theta_given:
        cmac += d * d * chi_l * chi_m * chi_r
    if xi_dense:
        cmac += d * d * chi_l * chi_l * chi_r
    return 8.0 * cmac


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(base, rank):
    """Seed of one replica's synthetic workload: every rank updates its own bond."""
    return base + 2 + rank


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (replicas run independently; the job ends with the last)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ws, t_max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / (t_max_ms / 1e3)


def cpu_oracle_update(wl, chi, want_result=False):
    from oracle import bond
    th = wl["theta"].astype(np.complex128)
    Bn = wl["Bn"].astype(np.complex128)
    t0 = time.perf_counter()
    out = bond.qr_update(None, None, Bn, wl["U"], chi_max=chi, theta=th)
    dt = time.perf_counter() - t0
    return (dt, out) if want_result else dt


def cpu_oracle_one_thread(chi, d, seed):
    """Seconds of one oracle update in a fresh interpreter whose BLAS/LAPACK runs on one
    thread (the thread count is fixed when the library loads, hence the child process)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, time; sys.path.insert(0, %r); import numpy as np; "
            "from paper_2212_09782_b300 import workloads as W; from oracle import bond; "
            "wl = W.bond_microbench(%d, %d, seed=%d); t0 = time.perf_counter(); "
            "bond.qr_update(None, None, wl['Bn'].astype(np.complex128), wl['U'], chi_max=%d, "
            "theta=wl['theta'].astype(np.complex128)); print(time.perf_counter() - t0)"
            % (ROOT, chi, d, seed, chi))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2212_09782_b300 import workloads as W
    wl = W.bond_microbench(args.chi, args.d)
    for _ in range(args.warmup):
        cpu_oracle_update(wl, args.chi)
    times = [cpu_oracle_update(wl, args.chi) for _ in range(args.steps)]
    tot = sum(times)
    v = args.steps / tot
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "p50_ms": 1e3 * statistics.median(times),
        "p99_ms": 1e3 * float(np.percentile(times, 99)),
        "config": {"workload": f"single QR-TEBD bond update chi={args.chi} d={args.d} eta=chi plain",
                   "global_batch": 1, "parallelism": "none (host oracle)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full bond updates (complex128 NumPy/LAPACK)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2212_09782_b300 import lib as L
    from paper_2212_09782_b300 import workloads as W

    chi, d = args.chi, args.d
    prec = L.PRECISIONS[args.precision]
    wl = W.bond_microbench(chi, d, seed=replica_seed(W.BASE_SEED, rank))
    cdt = torch.complex128 if L.is_c128(prec) else torch.complex64
    th = torch.from_numpy(wl["theta"]).to(dtype=cdt, device="cuda")
    bn = torch.from_numpy(wl["Bn"]).to(dtype=cdt, device="cuda")
    gate = torch.from_numpy(wl["U"]).to("cuda")
    tr = L.trunc_default(L.PLAIN, chi)
    # the dense tensor peaks the metric's roofline is taken against (before any workspace)
    mpk = None if args.no_peaks else measure_matmul_peaks(torch)
    up = L.BondUpdater(prec, chi, d, chi, chi, tr, xi_kind=0, theta_given=True)
    stream = torch.cuda.current_stream()
    tune = None
    if args.autotune_load:  # a table tuned earlier (e.g. outside a profiler)
        tune = {"loaded_entries": L.autotune_load(args.autotune_load), "from": args.autotune_load}
    elif args.autotune:  # tile shapes of this update's tensor-core products, before any timing
        tune = autotune_shapes(L, prec, [(chi, d, chi, chi)], tr, xi_kind=0, theta_given=True)
    if args.autotune_save:
        L.autotune_save(args.autotune_save)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up
    for _ in range(args.warmup):
        up.run(gate, bn, theta=th)
    L.stream_check()
    barrier()

    # ---- timed region (inputs live in HBM; theta = 210 MB > 126 MB L2); no per-kernel
    #      events here, so kernels overlap their launches as they do in production
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    n0 = L.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        ev[i][0].record(stream)
        up.run(gate, bn, theta=th)
        ev[i][1].record(stream)
    barrier()
    launches = L.launch_count() - n0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    L.stream_check()
    t_max = max_over_ranks(total_ms, dist, "cuda")
    value = job_throughput(args.steps, ws, t_max)

    # ---- per-kernel durations: the same steps again, every launch bracketed by CUDA
    #      events on its stream (the brackets cost a little, hence a separate pass)
    L.profile_enable(True)
    barrier()
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(stream)
    for i in range(args.steps):
        up.run(gate, bn, theta=th)
    pb.record(stream)
    barrier()
    prof_step_ms = pa.elapsed_time(pb) / args.steps
    fams, PROF_NAMES = prof_families(L)
    prof = {f: L.profile_read(f) for f in fams}
    L.profile_enable(False)
    L.stream_check()

    # ---- end to end through the public API with host buffers: every step copies its
    #      inputs from pinned host memory and reads its outputs back, all inside the
    #      timed region. Two updaters (workspaces) alternate, so step i+1's host->device
    #      copy and step i's device->host copy run on copy streams under step i+1's
    #      compute, as a caller of the asynchronous API would arrange it.
    e2e = None
    if not args.no_e2e:
        h_th = torch.from_numpy(wl["theta"]).to(cdt).pin_memory()
        h_bn = torch.from_numpy(wl["Bn"]).to(cdt).pin_memory()
        h_u = torch.from_numpy(wl["U"]).pin_memory()
        ups = [up, L.BondUpdater(prec, chi, d, chi, chi, tr, xi_kind=0, theta_given=True)]
        outs = [tuple(torch.empty(x.shape, dtype=x.dtype).pin_memory()
                      for x in (u.bm_out, u.xi_out, u.bn_out, u.stats)) for u in ups]
        dins = [(torch.empty_like(th), torch.empty_like(bn), torch.empty_like(gate)) for _ in ups]
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        ev = lambda: torch.cuda.Event()
        in_ready = [ev(), ev()]
        computed = [ev(), ev()]
        out_read = [ev(), ev()]
        for k in range(2):  # nothing pending yet
            computed[k].record(stream)
            out_read[k].record(stream)

        def e2e_step(i):
            k = i % 2
            d_th, d_bn, d_u = dins[k]
            with torch.cuda.stream(h2d):
                h2d.wait_event(computed[k])        # step i-2 has finished reading these inputs
                d_th.copy_(h_th, non_blocking=True)
                d_bn.copy_(h_bn, non_blocking=True)
                d_u.copy_(h_u, non_blocking=True)
                in_ready[k].record(h2d)
            stream.wait_event(in_ready[k])
            stream.wait_event(out_read[k])         # step i-2's outputs have been read back
            ups[k].run(d_u, d_bn, theta=d_th, stream=stream)
            computed[k].record(stream)
            with torch.cuda.stream(d2h):
                d2h.wait_event(computed[k])
                for o, x in zip(outs[k], (ups[k].bm_out, ups[k].xi_out, ups[k].bn_out, ups[k].stats)):
                    o.copy_(x, non_blocking=True)
                out_read[k].record(d2h)

        for i in range(args.warmup):
            e2e_step(i)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(args.steps):
            e2e_step(i)
        for k in range(2):
            stream.wait_event(out_read[k])
        b.record(stream)
        barrier()
        e_ms = max_over_ranks(a.elapsed_time(b), dist, "cuda")
        esz = lambda x: x.numel() * x.element_size()
        e2e = {"value": job_throughput(args.steps, ws, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": esz(h_th) + esz(h_bn) + esz(h_u),
               "d2h_bytes_per_step": sum(esz(o) for o in outs[0]),
               "pipelining": "two updaters alternate; copies overlap the next step's compute"}
        L.stream_check()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel family (by device time), and of the others
    peaks, src = load_peaks()
    breakdown = {PROF_NAMES[f]: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                 for f, v in prof.items() if v[1] > 0}
    roofs = {}
    for f, (ms, n, fl, by) in prof.items():
        if n > 0:
            roofs[PROF_NAMES[f]] = family_roofline(L, f, ms, n, fl, by, prec, peaks, src)
    dom = max((f for f in prof if prof[f][1] > 0), key=lambda f: prof[f][0])
    roof = roofs.get(PROF_NAMES[dom])

    # ---- the metric's "% TC roofline": the whole update's algorithmic flops over its time,
    #      against the TF32 (complex128: FP64) peak measured on this GPU just now
    tc_roof = None
    if mpk:
        fl = update_flops(chi, d, chi, chi, chi)
        key = "fp64_tflops" if L.is_c128(prec) else "tf32_tflops"
        ach = fl / (t_max / args.steps / 1e3) / 1e12
        tc_roof = {"algorithmic_flops_per_update": fl, "achieved_tflops": ach, "peak_tflops": mpk[key],
                   "frac": ach / mpk[key], "peak_source": f"measured in this run: {mpk[key + '_how']}",
                   "note": "the whole update (GEMMs, QRs, gate) against the dense tensor peak of its "
                           "arithmetic; 3xTF32 issues three TF32 products per complex GEMM MAC"}
        if prec == L.C128_OZ:
            tc_roof["note"] = ("complex128 with its GEMMs emulated on the TF32 tensor cores, against the "
                               "native FP64 peak: a fraction above 1 is FP64 work done faster than FP64 units")
        if not L.is_c128(prec):
            tc_roof["frac_vs_derived_tf32"] = ach / (peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
                                                     * TF32_PER_BF16)

    cpu = None
    err = None
    if not args.no_cpu_baseline and ws == 1:
        t, orc = cpu_oracle_update(wl, chi, want_result=True)
        cpu = {"value": 1.0 / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"1 full bond update chi={chi} d={d} (complex128 NumPy/LAPACK)"}
        t1 = cpu_oracle_one_thread(chi, d, replica_seed(W.BASE_SEED, rank))
        if t1:
            cpu["one_thread"] = {"value": 1.0 / t1, "cores": 1,
                                 "sample": "the same update in a child process with BLAS/LAPACK on one thread"}
        # the timed update's result against the FP64 oracle on the same inputs (gauge
        # invariant: the Schmidt values of Xi~ and eps)
        _bm, xi_g, _bn, st_g = up.outputs()
        s_g = np.linalg.svd(xi_g.cpu().numpy().astype(np.complex128), compute_uv=False)
        s_o = np.linalg.svd(orc["Xi_new"], compute_uv=False)
        err = {"schmidt_rel": float(np.linalg.norm(s_g - s_o) / np.linalg.norm(s_o)),
               "eps_rel": float(abs(float(st_g[0]) - orc["eps"]) / orc["eps"]),
               "reference": "oracle (complex128), same inputs"}

    # ---- the paper's comparison (Fig. 5) on this GPU, outside every timed region above
    arms = None
    if not args.no_svd_arm and ws == 1:
        up = ups = None  # release the timed updaters' workspaces
        torch.cuda.empty_cache()
        arms = comparison_arms(torch, L, wl, chi, d, prec, cdt, 1, 3, stream)
        arms["qr_precision"] = args.precision

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"c128": "c128", "c128_oz": "c128 (FP64 emulated on TF32 tensor cores, Ozaki slices)",
                  "c64_3xtf32": "c64 (3xTF32 tensor cores, FP32 accum, FP64 norms)",
                  "c64_tf32": "c64 (TF32 tensor cores)", "c64_fp32": "c64 (FP32 CUDA cores)"}[args.precision],
        "data": "synthetic",
        "p50_ms": statistics.median(step_ms), "p99_ms": float(np.percentile(step_ms, 99)),
        "config": {"workload": f"single QR-TEBD bond update chi={chi} d={d} eta=chi plain "
                               f"(theta given, Xi=1)", "global_batch": ws,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (theta 210 MB)", "precision": args.precision},
        "roofline": roof, "tc_roofline": tc_roof, "measured_peaks": mpk, "comparison_arms": arms,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "kernel_breakdown": breakdown, "dominant_family": PROF_NAMES[dom],
        "roofline_by_family": roofs, "profiled_ms_per_step": prof_step_ms, "clocks": clk,
        "autotune": tune, "error_vs_oracle": err,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def autotune_shapes(L, prec, shapes, tr, xi_kind, theta_given):
    """Run the library's autotuner on each bond shape (chi_l, d, chi_m, chi_r); summary."""
    t0 = time.perf_counter()
    n = 0
    for (cl, dd, cm, cr) in shapes:
        n += L.autotune_bond(prec, cl, dd, cm, cr, tr, xi_kind=xi_kind, theta_given=theta_given)
    ents = L.autotune_entries()
    return {"bond_shapes": len(shapes), "products_tuned": n, "seconds": round(time.perf_counter() - t0, 2),
            "changed_from_heuristic": sum(1 for e in ents if tuple(e["config"]) != (256, 0, 1)),
            "sum_ms_tuned": round(sum(e["ms_tuned"] for e in ents), 4),
            "sum_ms_heuristic": round(sum(e["ms_default"] for e in ents), 4)}


def run_chain(args):
    """Finite-chain TEBD throughput: L = 128, d = 4 clock model (g = 1.0), bond dimensions
    min(4^k, 4^(L-k), 512) from a seeded random right-canonical state, plain QR at saturated
    eta, complex64; each Strang step is three layers, batched across the chain's bonds
    (--no-batch: one bond after another). A step = 64 + 63 + 64 bond updates."""
    import torch
    from paper_2212_09782_b300 import lib as L
    from paper_2212_09782_b300 import workloads as W
    Lc, d, chi, g, dt = args.chain_L, 4, args.chain_chi, 1.0, 0.05
    dims, B, Xi = W.random_right_canonical_mps(Lc, d, chi, seed=W.BASE_SEED + 4)
    s = L.MPS(Lc, d, chi, precision=args.precision)
    for m in range(Lc):
        s.set_site(m, B[m])
    for b in range(Lc + 1):
        s.set_bond(b, Xi[b], diagonal=True)
    gh = L.clock_layer_gates(Lc, d, g, dt / 2)
    gf = L.clock_layer_gates(Lc, d, g, dt)
    tr = L.trunc_default(L.PLAIN, chi)
    tune = None
    if args.autotune:
        # every distinct bond shape of the chain (dense Xi after the first update, theta formed)
        shapes = sorted({(dims[m], d, dims[m + 1], dims[m + 2]) for m in range(Lc - 1)})
        tune = autotune_shapes(L, L.PRECISIONS[args.precision], shapes, tr, xi_kind=1, theta_given=False)
    # a Strang step layer by layer (the library's tebd_step / tebd_step_batched), each layer
    # between two events on the state's stream (torch's current stream) when `lay` is given
    def step(lay=None):
        for p, gates in ((0, gh), (1, gf), (0, gh)):
            a = torch.cuda.Event(enable_timing=True) if lay is not None else None
            if a is not None:
                a.record()
            if args.no_batch:
                s.apply_layer(p, gates, tr)
            else:
                L.apply_layer_batched([s], p, [gates], tr)
            if a is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                lay.append((p, a, e))
    for _ in range(args.warmup):
        step()
    s.sync()
    torch.cuda.synchronize()
    n0 = L.launch_count()
    t0 = time.perf_counter()
    ev = []
    lay = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        a.record()
        step(lay)
        ev.append(a)
    b = torch.cuda.Event(enable_timing=True)
    b.record()
    s.sync()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = ev[0].elapsed_time(b)
    per_step = [ev[i].elapsed_time(ev[i + 1] if i + 1 < len(ev) else b) for i in range(len(ev))]
    nupd = sum(len(range(p, Lc - 1, 2)) for p in (0, 1, 0))
    # per-layer latency: even layers (64 bonds at L = 128) and odd layers (63 bonds)
    lay_ms = {p: [a.elapsed_time(e) for q, a, e in lay if q == p] for p in (0, 1)}
    layer_latency = {("even" if p == 0 else "odd"): {
        "bonds": len(range(p, Lc - 1, 2)), "p50_ms": statistics.median(v),
        "p99_ms": float(np.percentile(v, 99)), "layers": len(v)} for p, v in lay_ms.items() if v}
    line = {
        "metric": "TEBD bond updates/s, finite chain L=128 d=4 chi<=512 (batched layers)",
        "value": args.steps * nupd / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "p50_ms": statistics.median(per_step), "p99_ms": float(np.percentile(per_step, 99)),
        "host_wall_s": wall, "updates_per_step": nupd, "layer_latency": layer_latency,
        "gpu_launches": L.launch_count() - n0,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"finite chain L={Lc} d=4 chi<={chi} plain, Strang step",
                   "batched": not args.no_batch},
        "autotune": tune,
    }
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def run_serve(args):
    """Continuous-batching quench service: a seeded Poisson mix (rate 4/s) with L in
    {32, 64, 128}, d in {3, 4, 5}, chi_max in {128, 256, 512, 1024}, g in [0.5, 2],
    dt = 0.05, plain QR, complex64; --serve-requests / --serve-steps bound the run."""
    from paper_2212_09782_b300 import serve
    reqs = serve.poisson_mix(args.serve_requests, 4.0, seed=2212_09782 + 5, steps=args.serve_steps)
    srv = serve.QuenchServer(precision=args.precision)
    for r in reqs:
        srv.submit(r)
    m = srv.run(max_seconds=args.serve_max_seconds)
    # per-request parity: the cheapest finished requests replayed by the complex128 oracle
    # (same L, d, g, dt, chi_max, steps, plain scheme), <Z> of the middle site step by step
    parity = []
    if args.serve_oracle > 0:
        from oracle import clock as oclock
        from oracle import mps as omps
        done = sorted(srv.done, key=lambda r: r.L * r.chi_max ** 2 * r.d ** 3)[: args.serve_oracle]
        for r in done:
            t0 = time.perf_counter()
            o = omps.product_state(r.L, r.d, 0, True)
            half, full = omps.strang_gates(r.L, r.d, r.g, r.dt, True)
            Z, _X = oclock.clock_operators(r.d)
            zo = []
            for _ in range(len(r.z_mid)):
                omps.tebd_step(o, half, full, scheme="plain", chi_max=r.chi_max)
                zo.append(omps.expectation_1site(o, r.L // 2, Z))
            dz = np.abs(np.array(r.z_mid) - np.array(zo))
            parity.append({"rid": r.rid, "L": r.L, "d": r.d, "chi_max": r.chi_max, "g": round(r.g, 4),
                           "steps": len(zo), "max_abs_dZ_mid": float(dz.max()),
                           "oracle_seconds": round(time.perf_counter() - t0, 1)})
    line = {"metric": "quench serving: aggregate bond updates/s, p50/p99 per-step latency",
            "value": m["bond_updates_per_s"], "unit": UNIT, "n_gpus": 1,
            "p50_ms": m["p50_step_latency_ms"], "p99_ms": m["p99_step_latency_ms"],
            "higher_is_better": True, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": f"{args.serve_requests} quench requests, Poisson 4/s, "
                                   f"{args.serve_steps} Strang steps each"},
            "detail": m, "oracle_parity": parity}
    print(json.dumps(line), flush=True)
    return 0


def comparison_arms(torch, L, wl, chi, d, prec, cdt, warmup, steps, stream):
    """QR update of this library against the SVD-based and the eigendecomposition-based
    updates run through torch's cuSOLVER calls, on the same theta (chi, d, d, chi): the
    paper's Fig. 5 comparison restated on this GPU. Measurement only: the library never
    calls a solver. SVD arm: theta = U S V^dag (reduced), keep chi, B~m = theta V_chi.
    EIG arm: theta^dag theta = V S^2 V^dag (Hermitian eigensolver), keep the chi largest,
    B~m = theta V_chi. Both arms skip the gate (theta supplied); the QR arm runs every
    step of the update, gate included."""
    def timed(fn, n_warm, n_steps):
        for _ in range(n_warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n_steps

    th = torch.from_numpy(wl["theta"]).to(dtype=cdt, device="cuda")
    bn = torch.from_numpy(wl["Bn"]).to(dtype=cdt, device="cuda")
    gate = torch.from_numpy(wl["U"]).to("cuda")
    tr = L.trunc_default(L.PLAIN, chi)
    up = L.BondUpdater(prec, chi, d, chi, chi, tr, xi_kind=0, theta_given=True)
    qr_ms = timed(lambda: up.run(gate, bn, theta=th), warmup, steps)
    L.stream_check()
    M = th.reshape(chi * d, d * chi)

    def svd_arm():
        _U, _S, Vh = torch.linalg.svd(M, full_matrices=False)
        return M @ Vh[:chi].conj().T

    def eig_arm():
        _w, V = torch.linalg.eigh(M.conj().T @ M)
        return M @ V[:, -chi:]

    svd_ms = timed(svd_arm, 1, max(1, min(steps, 2)))
    eig_ms = timed(eig_arm, 1, max(1, min(steps, 5)))
    out = {"qr_ms": qr_ms, "svd_ms": svd_ms, "eig_ms": eig_ms, "qr_speedup_over_svd": svd_ms / qr_ms,
           "qr_speedup_over_eig": eig_ms / qr_ms,
           "svd_eig_solver": "torch.linalg.svd / torch.linalg.eigh (cuSOLVER), measurement only"}
    del th, bn, up, M
    torch.cuda.empty_cache()
    return out


def run_svd_arm(args):
    """Comparison arms of the single-gate benchmark as their own JSON line (see
    comparison_arms); --svd-c128 adds the complex128 arms."""
    import torch
    from paper_2212_09782_b300 import lib as L
    from paper_2212_09782_b300 import workloads as W
    chi, d = args.chi, args.d
    wl = W.bond_microbench(chi, d, seed=W.BASE_SEED + 2)
    stream = torch.cuda.current_stream()
    out = {"metric": f"single bond update time, QR (this library) vs SVD / EIG (cuSOLVER via torch), chi={chi} d={d}",
           "unit": "ms per update", "higher_is_better": False, "data": "synthetic",
           "steps": args.steps, "warmup": args.warmup, "arms": {}}
    arms = [("c64_3xtf32", torch.complex64)] + ([("c128", torch.complex128)] if args.svd_c128 else [])
    for prec, cdt in arms:
        key = "c64" if prec != "c128" else "c128"
        out["arms"][key] = comparison_arms(torch, L, wl, chi, d, L.PRECISIONS[prec], cdt, args.warmup,
                                           args.steps, stream)
        out["arms"][key]["qr_precision"] = prec
    print(json.dumps(out), flush=True)
    return 0


def run_cbe_eig(args):
    """CBE step (iv) alone (qrtebd_cbe_decompose) on an upper-triangular Rz of order n with a
    decaying spectrum, the shape C3 reaches at chi = 1024 (eta = 1126): ms per decomposition,
    Jacobi sweeps, and the error of the eigenvalues against numpy (FP64, host)."""
    import torch
    from paper_2212_09782_b300 import lib as L
    from paper_2212_09782_b300 import workloads as W
    n = args.eig_n
    r = W.rng(W.BASE_SEED + n)
    A = W.complex_gaussian(r, (n, n)) * np.exp(-np.arange(n) / (n / 6))[None, :]
    Rz = np.linalg.qr(A)[1]
    dt = torch.complex128 if args.precision.startswith("c128") else torch.complex64
    Rd = torch.from_numpy(Rz).to(device="cuda", dtype=dt)
    for _ in range(args.warmup):
        w, Vh, sw = L.cbe_decompose(args.precision, Rd)
    torch.cuda.synchronize()
    n0 = L.launch_count()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        w, Vh, sw = L.cbe_decompose(args.precision, Rd)
    b.record()
    torch.cuda.synchronize()
    L.stream_check()
    ms = a.elapsed_time(b) / args.steps
    Rr = Rd.cpu().numpy().astype(np.complex128)
    ref = np.sort(np.linalg.eigvalsh(Rr @ Rr.conj().T))[::-1]
    wv, V = w.cpu().numpy(), Vh.cpu().numpy()
    line = {"metric": "CBE step (iv) decompositions/s (L^dag L = V^dag S^2 V)", "value": 1e3 / ms,
            "unit": "decompositions/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "n_gpus": 1, "dtype": args.precision, "data": "synthetic",
            "sweeps": int(sw.item()), "gpu_launches": L.launch_count() - n0,
            "max_abs_dw_over_w0": float(np.abs(wv - ref).max() / ref[0]),
            "max_abs_VVdag_minus_1": float(np.abs(V @ V.conj().T - np.eye(n)).max()),
            "config": {"workload": f"CBE decomposition n={n} (Rz = R of a Gaussian matrix with "
                                   f"column scales exp(-6 j / n))"}}
    print(json.dumps(line), flush=True)
    return 0


def run_sym(args):
    """Charge-sector CBE (Sec. III with Z_d charges) at chi = --chi, d = --d: theta' of the C2
    shape restricted to the Z_d charge rule (bond charges drawn uniformly and sorted, so each
    block is chi x chi and holds 1/d of the entries), a random charge-conserving gate, the
    middle bond's chi states spread over the charges (chi_q ~ chi/d, eta_q = chi_q + 100),
    chi_max = chi. Updates/s of qrtebd_sym_bond_update beside the dense CBE update on the same
    theta' (eta = chi + 103), and the result against the oracle on the same inputs."""
    import torch
    from paper_2212_09782_b300 import lib as L
    from paper_2212_09782_b300 import workloads as W
    sys.path.insert(0, ROOT)
    from oracle import symmetric as osym
    chi, d, prec = args.chi, args.d, args.precision
    r = W.rng(W.BASE_SEED + 31)
    cl, cm, cr = (W.random_charges(r, chi, d) for _ in range(3))
    th = W.symmetric_theta(r, cl, cr, d)
    U = W.charge_conserving_unitary(r, d)
    cdt = torch.complex128 if prec.startswith("c128") else torch.complex64
    th_d = torch.from_numpy(th).to(device="cuda", dtype=cdt)
    gate = torch.from_numpy(U).cuda()
    tr = L.trunc_default(L.CBE, chi)
    up = L.SymBondUpdater(prec, d, cl, cm, cr, tr, xi_kind=0)
    dense = L.BondUpdater(prec, chi, d, chi, chi, tr, xi_kind=0, theta_given=True)
    bn_d = torch.zeros(chi * d * chi, dtype=cdt, device="cuda")  # not read by CBE (Y0 from theta~)

    def timed(fn, n):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(n):
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts
    sym_fn = lambda: up.run(gate, theta=th_d)
    den_fn = lambda: dense.run(gate, bn_d, theta=th_d)
    timed(sym_fn, args.warmup)
    n0 = L.launch_count()
    ts = timed(sym_fn, args.steps)
    launches = (L.launch_count() - n0) / max(args.steps, 1)
    L.stream_check()
    Bm, x, Bn, ch, st = up.outputs()
    got_S = np.real(x.cpu().numpy().astype(np.complex128))
    got_eps = float(st[0].item())
    timed(den_fn, args.warmup)
    td = timed(den_fn, max(3, args.steps // 2))
    L.stream_check()
    line = {"metric": f"charge-sector CBE bond updates/s, chi={chi} d={d} (Z_{d} charges)",
            "value": 1e3 / statistics.median(ts), "unit": "bond updates/s", "higher_is_better": True,
            "ms_per_step": statistics.median(ts), "ms_p99": sorted(ts)[max(0, int(0.99 * len(ts)) - 1)],
            "dense_cbe_ms": statistics.median(td), "speedup_vs_dense_cbe": statistics.median(td) / statistics.median(ts),
            "chi_new": up.info.chi_new, "eta_sum": up.info.eta, "chi_sector": up.chi_sector.tolist(),
            "gpu_launches_per_update": launches, "steps": args.steps, "warmup": args.warmup,
            "n_gpus": 1, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"theta' (chi={chi}, d={d}, d, chi) on the Z_{d} charge rule, "
                                   f"unit norm; chi_max={chi}, dchi_min=100, dchi_frac=0.1",
                       "l2": "theta' larger than L2"}}
    if not args.no_cpu_baseline:
        thr = th.astype(np.complex64).astype(np.complex128) if not prec.startswith("c128") else th
        t0 = time.perf_counter()
        o = osym.sym_qr_update(thr, None, U, cl, cm, cr, chi_max=chi)
        t_or = time.perf_counter() - t0
        ok = np.array_equal(up.chi_sector, o["chi_sector"])
        errS = None
        if ok:
            errS = max(float(np.max(np.abs(got_S[o["charge_new"] == q] - o["xi_new"][o["charge_new"] == q])))
                       for q in range(d) if np.any(o["charge_new"] == q))
        line["error_vs_oracle"] = {"chi_sector_equal": bool(ok), "max_abs_dS": errS,
                                   "abs_deps": abs(got_eps - o["eps"])}
        line["cpu_baseline"] = {"value": 1.0 / t_or, "unit": "bond updates/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": "one update (complex128 NumPy/LAPACK)"}
    print(json.dumps(line), flush=True)
    return 0


def run_c1(args):
    """C1: finite chain L = 16, d = 3, g = 1.5, quench from |0...0>, Strang dt = 0.05,
    20 steps, chi_max = 32, plain QR, complex128. The whole run on the GPU (wall time,
    synchronised at every step to read <Z> on the middle site) against the oracle's run on
    the host cores; max |<Z>_gpu - <Z>_oracle| over the steps."""
    import torch
    from paper_2212_09782_b300 import lib as L
    sys.path.insert(0, ROOT)
    from oracle import mps as omps
    Lc, d, g, dt, steps, chi = 16, 3, 1.5, 0.05, 20, 32
    Z = np.diag(np.exp(2j * np.pi * np.arange(d) / d))
    tr = L.trunc_default(L.PLAIN, chi)
    half = L.clock_layer_gates(Lc, d, g, dt / 2)
    full = L.clock_layer_gates(Lc, d, g, dt)

    def gpu_run():
        s = L.MPS(Lc, d, chi, precision="c128")
        zs = []
        for _ in range(steps):
            L.tebd_step(s, half, full, tr)
            zs.append(s.expectation(Lc // 2, Z))
        s.close()
        return zs
    for _ in range(max(1, args.warmup)):
        gpu_run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    zg = gpu_run()
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0

    o = omps.product_state(Lc, d, 0)
    oh, of = omps.strang_gates(Lc, d, g, dt)
    zo = []
    t0 = time.perf_counter()
    for _ in range(steps):
        omps.tebd_step(o, oh, of, scheme="plain", chi_max=chi)
        zo.append(omps.expectation_1site(o, Lc // 2, Z))
    t_cpu = time.perf_counter() - t0
    nb = Lc - 1
    upd = steps * (2 * len(range(0, nb, 2)) + len(range(1, nb, 2)))
    out = {"metric": "C1 quench run time, L=16 d=3 chi<=32 plain c128 (20 Strang steps)",
           "value": upd / t_gpu, "unit": "bond updates/s", "higher_is_better": True,
           "gpu_run_s": t_gpu, "bond_updates": upd,
           "cpu_baseline": {"value": upd / t_cpu, "unit": "bond updates/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": "the whole C1 run (complex128 NumPy/LAPACK)",
                            "run_s": t_cpu},
           "max_abs_dZ": float(np.max(np.abs(np.array(zg) - np.array(zo)))),
           "data": "synthetic", "dtype": "c128"}
    print(json.dumps(out), flush=True)
    return 0


def run_c3(args):
    """C3: uniform two-site cell, d = 5, g = 2.0, |00>, dt = 0.02, CBE with
    dchi = max(100, ceil(0.1 chi)), chi_max = 1024, svd_min = 1e-14, complex64 3xTF32.
    Steps until --c3-steps or --c3-seconds; each step's device time (synchronised) is
    binned by the largest bond dimension after the step."""
    import torch
    from paper_2212_09782_b300 import lib as L
    Lc, d, g, dt, chi = 2, 5, 2.0, 0.02, 1024
    tr = L.trunc_default(L.CBE, chi, reorth=args.reorth)
    half = L.clock_layer_gates(Lc, d, g, dt / 2, infinite=True)
    full = L.clock_layer_gates(Lc, d, g, dt, infinite=True)
    s = L.MPS(Lc, d, chi, precision=args.precision, infinite=True)
    Z = np.diag(np.exp(2j * np.pi * np.arange(d) / d))
    buckets = [(1, 64), (64, 256), (256, 512), (512, 1025)]
    acc = {b: [0.0, 0] for b in buckets}
    t_start = time.perf_counter()
    rows = []
    n = 0
    for step in range(args.c3_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.tebd_step(s, half, full, tr)
        s.sync()
        dtm = time.perf_counter() - t0
        chis = s.bond_dims()
        cmax = max(chis)
        for b in buckets:
            if b[0] <= cmax < b[1]:
                acc[b][0] += dtm
                acc[b][1] += 3
        n += 1
        if step % 10 == 9 or step == args.c3_steps - 1:
            rows.append({"step": step + 1, "chi": chis, "z": [s.expectation(0, Z).real],
                         "eps": s.truncation_error(-1), "s_vN": s.entropy(0)})
        if time.perf_counter() - t_start > args.c3_seconds:
            break
    out = {"metric": "C3 uniform CBE, d=5 g=2 dt=0.02, chi 1->1024: bond updates/s per chi bucket",
           "unit": "bond updates/s", "higher_is_better": True, "steps_done": n,
           "per_bucket": {f"{a}-{b - 1}": {"updates": v[1], "updates_per_s": v[1] / v[0] if v[0] else None}
                          for (a, b), v in acc.items()},
           "trace": rows, "dtype": args.precision, "data": "synthetic"}
    print(json.dumps(out), flush=True)
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="c64_3xtf32",
                    choices=["c64_3xtf32", "c64_tf32", "c64_fp32", "c128", "c128_oz"])
    ap.add_argument("--chi", type=int, default=1024)
    ap.add_argument("--d", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-svd-arm", action="store_true",
                    help="bond workload: skip the SVD / EIG comparison arms after the timed runs")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the TF32 / FP64 matmul peak measurement (and the tc_roofline it feeds)")
    ap.add_argument("--workload", choices=["bond", "chain", "serve", "svd", "c1", "c3", "cbe_eig",
                                           "sym"],
                    default="bond")
    ap.add_argument("--eig-n", type=int, default=1126, help="cbe_eig workload: the order n")
    ap.add_argument("--c3-steps", type=int, default=200)
    ap.add_argument("--c3-seconds", type=float, default=240.0)
    ap.add_argument("--serve-requests", type=int, default=12)
    ap.add_argument("--serve-steps", type=int, default=6)
    ap.add_argument("--serve-max-seconds", type=float, default=None,
                    help="serve workload: stop admitting and ticking after this wall time")
    ap.add_argument("--serve-oracle", type=int, default=2,
                    help="serve workload: replay this many of the cheapest finished requests on the oracle")
    ap.add_argument("--chain-L", type=int, default=128)
    ap.add_argument("--chain-chi", type=int, default=512)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--autotune-save", default=None,
                    help="bond workload: write the tuned table (JSON) after tuning")
    ap.add_argument("--autotune-load", default=None,
                    help="bond workload: load a tuned table instead of tuning (for runs under a "
                         "profiler, whose serialised replay would skew the tuner's timings)")
    ap.add_argument("--reorth", type=int, default=-1, choices=[-1, 0, 1],
                    help="re-orthogonalisation pass (qrtebd_trunc.reorth; -1 = the library default)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the library's tile autotuner (run by default on the bond and chain "
                         "workloads' shapes before any timing)")
    ap.add_argument("--svd-c128", action="store_true",
                    help="svd workload: add the complex128 arms (the cuSOLVER SVD alone takes ~165 s)")
    ap.add_argument("--tc-prep", choices=["separate", "kernel"], default="separate",
                    help="operand preparation of the complex64 tensor-core products: a separate "
                         "pass (default) or inside the GEMM kernel (128-column tiles)")
    args = ap.parse_args()
    if args.impl == "ours" and args.tc_prep == "kernel":
        from paper_2212_09782_b300 import lib as L
        L.tc_operand_prep(0)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "chain":
        return run_chain(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "svd":
        return run_svd_arm(args)
    if args.workload == "c1":
        return run_c1(args)
    if args.workload == "c3":
        return run_c3(args)
    if args.workload == "sym":
        return run_sym(args)
    if args.workload == "cbe_eig":
        return run_cbe_eig(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
