"""GEMM tile autotuner for the trajectory kernel.

The kernel has two GEMM tile rules (tjm_run_set_tile_rule): 64x64 output
tiles everywhere, or 32x32 tiles for products with an output side <= 32.
Which is faster depends on the bond dimensions a run goes through (chi_max,
chain length, the growth phase from a product state), so it is measured: the
first launches for a key (precision, chi_max) try the rules in turn, each
timed on the host around the launch and its completion and normalised by the
contraction flops the device counted during that launch -- so bond growth
between the trial launches does not bias the comparison.  The faster rule is
then cached for the key and set on every later launch with that key in this
process.  Trial launches are ordinary steps of the run; no work is thrown away.

Host-side control only: the rule is a launch setting of libtjm.so.
"""
from __future__ import annotations

import time

RULES = (0, 1)


class TileAutotuner:
    def __init__(self, clock=time.perf_counter):
        self.best = {}       # key -> rule
        self.trials = {}     # key -> {rule: contraction flops per second}
        self._clock = clock

    @staticmethod
    def key(ctx):
        return (int(ctx.precision), int(ctx.chi_max))

    def next_rule(self, key):
        """The cached rule, else the first rule not yet timed for the key."""
        if key in self.best:
            return self.best[key]
        done = self.trials.get(key, {})
        for r in RULES:
            if r not in done:
                return r
        return max(done, key=done.get)

    def record(self, key, rule, flops, seconds):
        """One timed launch; launches without contraction work (initialisation only) are not evidence."""
        if not (flops > 0 and seconds > 0):
            return
        t = self.trials.setdefault(key, {})
        t[rule] = max(t.get(rule, 0.0), flops / seconds)
        if all(r in t for r in RULES):
            self.best[key] = max(t, key=t.get)

    def advance(self, ctx, run_id, max_steps):
        """ctx.advance(run_id, max_steps) under the tuned (or next trial) rule; returns the rule used."""
        key = self.key(ctx)
        rule = self.next_rule(key)
        ctx.set_tile_rule(run_id, rule)
        if key in self.best:
            ctx.advance(run_id, max_steps)
            return rule
        f0 = ctx.stats(run_id)["flops_contract"]
        t0 = self._clock()
        ctx.advance(run_id, max_steps)
        ctx.sync()
        t1 = self._clock()
        f1 = ctx.stats(run_id)["flops_contract"]
        self.record(key, rule, f1 - f0, t1 - t0)
        return rule

    def report(self):
        names = {0: "f64", 1: "f32+f64", 2: "f32", 3: "f32+df64"}
        return {"%s/chi%d" % (names.get(k[0], str(k[0])), k[1]):
                {"best": self.best.get(k), "rates_tflops": {r: v / 1e12 for r, v in t.items()}}
                for k, t in self.trials.items()}
