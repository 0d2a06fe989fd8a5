"""Host logic of the GEMM tile autotuner, against a fake context (no GPU)."""
from paper_2501_17913_gb300.autotune import RULES, TileAutotuner


class FakeCtx:
    """Launches cost `cost[rule]` seconds per flop; every launch does `flops` of contraction work."""

    def __init__(self, precision, chi_max, cost, flops=1e12, clock=None):
        self.precision, self.chi_max = precision, chi_max
        self.cost, self.flops, self.clock = cost, flops, clock
        self.rule, self.done, self.rules_used = 0, 0.0, []

    def set_tile_rule(self, run_id, rule):
        assert rule in RULES
        self.rule = rule

    def advance(self, run_id, max_steps):
        self.rules_used.append(self.rule)
        self.done += self.flops
        self.clock.t += self.flops * self.cost[self.rule]

    def sync(self):
        pass

    def stats(self, run_id):
        return {"flops_contract": self.done}


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def test_tries_each_rule_then_keeps_the_faster():
    clk = Clock()
    tu = TileAutotuner(clock=clk)
    ctx = FakeCtx(2, 16, {0: 2e-12, 1: 1e-12}, clock=clk)
    for _ in range(5):
        tu.advance(ctx, 1, 1)
    assert ctx.rules_used == [0, 1, 1, 1, 1]
    assert tu.best[(2, 16)] == 1
    ctx64 = FakeCtx(2, 64, {0: 1e-12, 1: 3e-12}, clock=clk)
    for _ in range(4):
        tu.advance(ctx64, 1, 1)
    assert ctx64.rules_used == [0, 1, 0, 0]
    assert tu.best[(2, 64)] == 0
    rep = tu.report()
    assert rep["f32/chi16"]["best"] == 1 and rep["f32/chi64"]["best"] == 0


def test_launches_without_contraction_work_are_not_evidence():
    clk = Clock()
    tu = TileAutotuner(clock=clk)
    ctx = FakeCtx(0, 32, {0: 1e-12, 1: 2e-12}, flops=0.0, clock=clk)
    tu.advance(ctx, 1, 0)
    tu.advance(ctx, 1, 0)
    assert (0, 32) not in tu.best and ctx.rules_used == [0, 0]
    ctx.flops = 1e12
    for _ in range(3):
        tu.advance(ctx, 1, 1)
    assert ctx.rules_used[2:] == [0, 1, 0] and tu.best[(0, 32)] == 0


def test_rates_are_normalised_by_work():
    """A trial launch that does more work is not penalised for taking longer."""
    clk = Clock()
    tu = TileAutotuner(clock=clk)
    ctx = FakeCtx(2, 64, {0: 1e-12, 1: 1.5e-12}, flops=1e12, clock=clk)
    tu.advance(ctx, 1, 1)          # rule 0: 1 s for 1e12
    ctx.flops = 0.5e12
    tu.advance(ctx, 1, 1)          # rule 1: 0.75 s for 0.5e12 -- shorter, but slower per flop
    assert tu.best[(2, 64)] == 0
