"""Continuous-batching quench server on one GPU.

Requests are global quenches of the d-state clock model (Sec. IV, Eqs. 2-3) from the
|0...0> product state: a finite chain of L sites, field g, time step dt, a number of
second-order Strang steps, a bond-dimension cap chi_max. The server

* admits a request when its worst-case device footprint (site tensors and bond
  matrices at the bond-dimension caps, plus its share of the bond-update workspaces)
  fits the free device memory and a slot is free; a request that could never fit is
  rejected (QRTEBD_ERR_NOT_ADMITTED semantics);
* keeps every admitted state resident on the device and advances all of them one
  Strang step per tick, each layer batched across all resident states
  (qrtebd_apply_gate_layer_batched), so requests that arrive while others run join at
  the next tick and their work overlaps on the device;
* retires a request after its last step (its memory is freed for the next admission)
  and records, per step, <Z> on the middle site and the time the step completed.

Metrics: per-step latency = time between successive step completions of one request
(p50/p99 over all (request, step) pairs); aggregate bond updates/s.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import lib as L

# mirrors of qrtebd.h's QRTEBD_LAYER_BIG_BOND_BYTES / QRTEBD_LAYER_BIG_WORKERS
LAYER_BIG_BOND_BYTES = 1024 << 20
LAYER_BIG_WORKERS = 8


@dataclass
class Request:
    rid: int
    L: int
    d: int
    chi_max: int
    g: float
    steps: int
    dt: float = 0.05
    arrival: float = 0.0          # seconds after the server starts
    # results
    z_mid: list = field(default_factory=list)
    step_done: list = field(default_factory=list)
    eps: float = 0.0
    bond_dims: list = field(default_factory=list)
    admitted_at: float = None
    finished_at: float = None
    status: str = "pending"


def chain_caps(Lc, d, chi_max):
    return [min(d ** min(b, Lc - b), chi_max) if min(b, Lc - b) < 40 else chi_max
            for b in range(Lc + 1)]


def state_bytes(req, precision):
    """Device bytes of one resident state at its bond-dimension caps."""
    esz = 16 if L.is_c128(precision) else 8
    caps = chain_caps(req.L, req.d, req.chi_max)
    sites = sum(caps[m] * req.d * caps[m + 1] for m in range(req.L))
    bonds = sum(c * c + c for c in caps)
    gates = req.L * req.d ** 4 * 16
    return (sites + bonds) * esz + gates + 64 * 1024


def workspace_bytes(req, precision):
    """One bond-update workspace for this request's largest bond."""
    prec = L.PRECISIONS.get(precision, precision)
    chi = max(chain_caps(req.L, req.d, req.chi_max))
    tr = L.trunc_default(L.PLAIN, chi)
    return L.bond_workspace_size(prec, chi, req.d, chi, chi, tr, xi_kind=1)


class QuenchServer:
    def __init__(self, precision="c64_3xtf32", max_active=32, reserve_bytes=2 << 30,
                 mem_free=None, mem_total=None, workers=None):
        self.precision = precision
        self.max_active = max_active
        self.reserve = reserve_bytes
        # one bond-update workspace per executor worker stream
        self.workers = workers if workers is not None else L.layer_workers()
        self._mem_free = mem_free
        self._mem_total = mem_total
        self.pending = []
        self.active = []          # (request, mps, half gates, full gates)
        self.done = []
        self.rejected = []
        self.ws_peak = 0          # bytes held by the executor's worker workspaces
        self.trunc = None

    def submit(self, req):
        self.pending.append(req)

    def mem_free(self):
        if self._mem_free is not None:
            return self._mem_free()
        import torch
        free, _total = torch.cuda.mem_get_info()
        return free

    def mem_total(self):
        if self._mem_total is not None:
            return self._mem_total()
        import torch
        return torch.cuda.mem_get_info()[1]

    def executor_bytes(self, ws):
        """Workspace the executor holds once it has run bonds needing `ws` bytes each: bonds
        above QRTEBD_LAYER_BIG_BOND_BYTES use only the first LAYER_BIG_WORKERS workers, the
        other workers hold workspaces of at most that size."""
        if ws > LAYER_BIG_BOND_BYTES:
            return LAYER_BIG_WORKERS * ws + (self.workers - LAYER_BIG_WORKERS) * LAYER_BIG_BOND_BYTES
        return self.workers * ws

    def footprint(self, req):
        """Bytes admitting `req` would add: its state plus any growth of the shared
        worker workspaces."""
        need_ws = self.executor_bytes(workspace_bytes(req, self.precision))
        return state_bytes(req, self.precision) + max(0, need_ws - self.ws_peak)

    def _fits(self, req):
        """(fits now, could ever fit)."""
        need = self.footprint(req) + self.reserve
        alone = state_bytes(req, self.precision) + self.executor_bytes(workspace_bytes(req, self.precision))
        return need <= self.mem_free(), alone + self.reserve <= self.mem_total()

    def _admit(self, now):
        ready = [r for r in self.pending if r.arrival <= now]
        for req in sorted(ready, key=lambda r: r.arrival):
            if len(self.active) >= self.max_active:
                break
            ok, ever = self._fits(req)
            if not ever:
                req.status = "rejected"
                self.pending.remove(req)
                self.rejected.append(req)
                continue
            if not ok:
                break  # first come, first served: later requests wait too
            self.pending.remove(req)
            mps = L.MPS(req.L, req.d, req.chi_max, precision=self.precision)
            half = L.clock_layer_gates(req.L, req.d, req.g, req.dt / 2)
            full = L.clock_layer_gates(req.L, req.d, req.g, req.dt)
            req.admitted_at = now
            req.status = "running"
            self.ws_peak = max(self.ws_peak, self.executor_bytes(workspace_bytes(req, self.precision)))
            self.active.append((req, mps, half, full))

    def _tick(self, t0):
        states = [a[1] for a in self.active]
        halves = [a[2] for a in self.active]
        fulls = [a[3] for a in self.active]
        L.apply_layer_batched(states, 0, halves, self.trunc)
        L.apply_layer_batched(states, 1, fulls, self.trunc)
        L.apply_layer_batched(states, 0, halves, self.trunc)
        now = time.perf_counter() - t0
        finished = []
        for req, mps, _h, _f in self.active:
            Z = np.diag(np.exp(2j * np.pi * np.arange(req.d) / req.d))
            req.z_mid.append(mps.expectation(req.L // 2, Z))   # synchronises the state
            req.step_done.append(time.perf_counter() - t0)
            if len(req.z_mid) >= req.steps:
                finished.append((req, mps))
        for req, mps in finished:
            req.eps = mps.truncation_error(-1)
            req.bond_dims = mps.bond_dims()
            req.finished_at = time.perf_counter() - t0
            req.status = "done"
            mps.close()
            self.active = [a for a in self.active if a[0] is not req]
            self.done.append(req)
        return now

    def run(self, scheme=L.PLAIN, max_seconds=None):
        """Serve every submitted request; returns the metrics dict."""
        self.trunc = L.trunc_default(scheme, 1 << 20)
        t0 = time.perf_counter()
        while self.pending or self.active:
            now = time.perf_counter() - t0
            self._admit(now)
            if not self.active:
                nxt = min((r.arrival for r in self.pending), default=None)
                if nxt is None:
                    break
                time.sleep(max(0.0, min(0.05, nxt - now)))
                continue
            self._tick(t0)
            if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
                break
        wall = time.perf_counter() - t0
        return self.metrics(wall)

    def metrics(self, wall):
        lat = []
        updates = 0
        # finished requests, and the steps that requests still running at a time cap completed
        for r in self.done + [a[0] for a in self.active]:
            prev = r.admitted_at
            for t in r.step_done:
                lat.append(t - prev)
                prev = t
            nb = r.L - 1
            per_step = len(range(0, nb, 2)) * 2 + len(range(1, nb, 2))
            updates += per_step * len(r.step_done)
        lat = np.array(lat) if lat else np.zeros(1)
        return {"requests_done": len(self.done), "requests_rejected": len(self.rejected),
                "requests_running_at_end": len(self.active), "requests_waiting_at_end": len(self.pending),
                "step_latency_samples": int(lat.size),
                "wall_s": wall, "bond_updates": updates,
                "bond_updates_per_s": updates / wall if wall > 0 else 0.0,
                "p50_step_latency_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_step_latency_ms": 1e3 * float(np.percentile(lat, 99)),
                "executor_workspace_bytes": self.ws_peak}


def poisson_mix(n, rate, seed, Ls=(32, 64, 128), ds=(3, 4, 5), chis=(128, 256, 512, 1024),
                g_range=(0.5, 2.0), steps=50, dt=0.05):
    """A seeded request mix: Poisson arrivals, uniform L, d, chi_max and g."""
    from .workloads import rng
    r = rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += r.exponential(1.0 / rate)
        out.append(Request(rid=i, L=int(r.choice(Ls)), d=int(r.choice(ds)),
                           chi_max=int(r.choice(chis)), g=float(r.uniform(*g_range)),
                           steps=steps, dt=dt, arrival=t))
    return out
