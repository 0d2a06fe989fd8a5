"""Serving loop: continuous batching of TJM simulation requests on one GPU.

Requests (each its own Hamiltonian, rates, chi_max, trajectory count and
end time) arrive over time.  A request is admitted when its trajectory state
fits in the device-memory budget; every tick launches ONE persistent kernel
over the trajectories of all admitted requests (tjm_run_group_advance), each
advanced by at most `steps_per_tick` time steps, then retires finished
requests and frees their memory so queued ones can be admitted.  A request's
result does not depend on what it was batched with: every trajectory runs in
its own CTA and draws from its own Philox counter.

Host-side control only; all arithmetic is in libtjm.so.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs as I
from . import tjm


def state_bytes(wl, precision) -> int:
    """Device bytes of a request's trajectory state (sites, environments, outputs); the per-CTA scratch
    the batched launches hold is accounted for separately (Server._scratch_need)."""
    szc = 16 if precision == tjm.PREC_FP64 else 8
    chi = wl.chi_max
    D = max(int(np.shape(w)[1]) for w in wl.W)
    per = (wl.L * 2 * chi * chi + 2 * (wl.L + 1) * D * chi * chi) * szc
    per += (wl.L + 1) * 4 + len(wl.sample_steps) * len(wl.observables) * 8 + 512
    return int(wl.n_traj * per)


@dataclass
class Request:
    rid: int
    wl: object
    arrival: float
    ctx: object = None
    run: int = -1
    admitted: float = -1.0
    done: float = -1.0
    mean: np.ndarray = None
    sem: np.ndarray = None
    per_traj: np.ndarray = None
    bytes: int = 0
    work: float = 0.0          # trajectory*site*steps
    meta: dict = field(default_factory=dict)


class Server:
    def __init__(self, precision=tjm.PREC_FP32_DF64, mem_budget=None, steps_per_tick=1, device=0,
                 keep_per_traj=False, tuner=None, backend=tjm, clock=time.perf_counter):
        # backend: the library binding (tjm); a stand-in with the same names lets the host logic
        # run without a GPU
        self.tj = backend
        self.clock = clock
        self.tj.load()
        # GEMM tile rules tuned by earlier stepped runs of this process (autotune.TileAutotuner);
        # a request whose (precision, chi_max) has no tuned rule runs with the default
        self.tuner = tuner
        self.precision = precision
        self.steps = steps_per_tick
        self.device = device
        self.keep = keep_per_traj
        if mem_budget is None:
            import torch
            free, total = torch.cuda.mem_get_info(device)
            mem_budget = int(0.6 * free)
        self.budget = mem_budget
        self.used = 0
        self.queue = []
        self.active = []
        self.finished = []
        self.next_id = 0
        self.launches = 0
        # anchor context: owns the launch stream and the per-CTA scratch of every batched launch
        W = I.xxx_mpo(2, 0.0, 0.0)
        self.anchor = self.tj.Context(W, [], 0.1, 1, 0.0, precision=precision, device=device)
        self.anchor_run = self.anchor.prepare(None, 1, 0, [], [0.0])

    def submit(self, wl, arrival=None):
        r = Request(self.next_id, wl, self.clock() if arrival is None else arrival)
        r.bytes = state_bytes(wl, self.precision)
        r.work = float(wl.n_traj) * wl.L * wl.n_steps
        self.next_id += 1
        self.queue.append(r)
        return r.rid

    def _scratch_need(self, extra=None):
        """Bytes of the launch scratch for the largest (chi_max, L) among the active requests (and `extra`):
        every resident CTA holds one trajectory's scratch, sized by the largest request in the launch."""
        wls = [r.wl for r in self.active] + ([extra] if extra is not None else [])
        if not wls or not hasattr(self.anchor, "scratch_bytes"):
            return 0
        return self.anchor.scratch_bytes(max(w.chi_max for w in wls), max(w.L for w in wls))

    def _admit(self, now):
        still = []
        for r in self.queue:
            if r.arrival > now:
                still.append(r)
                continue
            if self.used + r.bytes + self._scratch_need(r.wl) > self.budget and self.active:
                # waits for memory; later arrivals that fit are still admitted (backfilling), and a
                # request is always admitted once nothing else runs, so none waits forever
                still.append(r)
                continue
            wl = r.wl
            rule = self.tuner.best.get((int(self.precision), int(wl.chi_max)), 0) if self.tuner else 0
            r.ctx = self.tj.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=self.precision,
                                    device=self.device, tile_rule=rule)
            psi = np.array(wl.psi0_per_traj) if wl.psi0_per_traj is not None else np.array(wl.psi0)
            r.run = r.ctx.prepare(psi, wl.n_traj, wl.seed, wl.observables, wl.times,
                                  first_traj=wl.meta.get('first_traj', 0))
            r.admitted = now
            self.used += r.bytes
            self.active.append(r)
        self.queue = still

    def tick(self):
        """Admit, run one batched launch, retire.  Returns False when idle with nothing queued."""
        now = self.clock()
        self._admit(now)
        if not self.active:
            return bool(self.queue)
        pairs = [(self.anchor, self.anchor_run)] + [(r.ctx, r.run) for r in self.active]
        self.tj.group_advance(pairs, self.steps)      # asynchronous
        self.launches += 1
        # requests that arrive while the launch runs are prepared now and join the next launch
        self._admit(self.clock())
        self.anchor.sync()
        still = []
        launched = {id(c) for (c, _) in pairs}
        for r in self.active:
            if id(r.ctx) not in launched:
                still.append(r)          # admitted during the launch
                continue
            st = r.ctx.stats(r.run)
            if st['steps_done_min'] >= r.wl.n_steps or st['failed'] == st['n_traj']:
                r.mean, r.sem, pt = r.ctx.result(r.run, per_traj=self.keep, allow_numeric=True)
                if self.keep:
                    r.per_traj = pt
                r.done = self.clock()
                r.ctx.free(r.run)
                r.ctx.close()
                self.used -= r.bytes
                self.finished.append(r)
            else:
                still.append(r)
        self.active = still
        return bool(self.active or self.queue)

    def drain(self):
        while self.tick():
            if not self.active and self.queue:
                time.sleep(max(0.0, min(q.arrival for q in self.queue) - self.clock()))
        return self.finished

    def report(self, t0, t1):
        lat = np.array([r.done - r.arrival for r in self.finished])
        work = sum(r.work for r in self.finished)
        arrivals = [r.arrival for r in self.finished]
        window = max(arrivals) - min(arrivals) if len(arrivals) > 1 else 0.0
        return {"requests": len(self.finished), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "sustained": work / (t1 - t0), "offered": work / window if window > 0 else None,
                "unit": "trajectory*site*steps/s", "launches": self.launches, "wall_s": t1 - t0}

    def close(self):
        for r in self.active:
            r.ctx.close()
        self.anchor.close()


def main():
    p = argparse.ArgumentParser(description="replay the Poisson request stream through the serving loop")
    p.add_argument("--requests", type=int, default=8)
    p.add_argument("--traj-scale", type=float, default=1.0 / 64, help="scale each request's trajectory count")
    p.add_argument("--max-steps", type=int, default=10, help="cap each request's number of time steps")
    p.add_argument("--steps-per-tick", type=int, default=1)
    a = p.parse_args()
    stream = I.request_stream()[:a.requests]
    srv = Server(steps_per_tick=a.steps_per_tick)
    t0 = time.perf_counter()
    for (t_arr, wl) in stream:
        wl.n_traj = max(1, int(math.ceil(wl.n_traj * a.traj_scale)))
        wl.n_steps = min(wl.n_steps, a.max_steps)
        wl.sample_steps = [wl.n_steps]
        srv.submit(wl, t0 + t_arr)
    srv.drain()
    t1 = time.perf_counter()
    rep = srv.report(t0, t1)
    rep["stream"] = ("first %d arrivals of the Poisson stream (20/s, seed 11), trajectory counts x %.4g, "
                     "at most %d steps each" % (a.requests, a.traj_scale, a.max_steps))
    print(json.dumps(rep))
    srv.close()


if __name__ == "__main__":
    main()
