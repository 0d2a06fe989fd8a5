"""Host logic of the serving loop (admission by memory budget, batched ticks, retirement), on a
stand-in for the library binding -- no GPU."""
import numpy as np

from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import serve
from paper_2501_17913_gb300 import tjm


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """The names serve.Server uses from the binding; every launch advances its runs and takes 1 s."""
    PREC_FP64, PREC_FP32, PREC_FP32_DEC32 = tjm.PREC_FP64, tjm.PREC_FP32, tjm.PREC_FP32_DEC32

    def __init__(self, clock):
        self.clock = clock
        self.launches = []
        backend = self

        class Ctx:
            def __init__(self, W, jumps, dt, chi_max, trunc_eps, precision=0, device=0, tile_rule=0):
                self.runs, self.closed, self.backend = {}, False, backend

            def prepare(self, psi, n_traj, seed, obs, times, first_traj=0):
                rid = len(self.runs) + 1
                self.runs[rid] = {"n": n_traj, "steps": -1, "shape": (len(times), max(1, len(obs)))}
                return rid

            def stats(self, rid):
                r = self.runs[rid]
                return {"steps_done_min": r["steps"], "failed": 0, "n_traj": r["n"]}

            def result(self, rid, per_traj=False, allow_numeric=False):
                r = self.runs[rid]
                return np.zeros(r["shape"]), np.zeros(r["shape"]), None

            def free(self, rid):
                del self.runs[rid]

            def close(self):
                self.closed = True

            def sync(self):
                pass

        self.Context = Ctx

    def load(self):
        pass

    def group_advance(self, pairs, steps):
        ids = []
        for ctx, rid in pairs:
            r = ctx.runs[rid]
            r["steps"] = max(r["steps"], 0) + steps      # the first launch also initialises
            ids.append((id(ctx), rid))
        self.launches.append(ids)
        self.clock.t += 1.0


def _wl(n_traj, n_steps):
    wl = I.config_small_fp64(n_traj)
    wl.n_steps = n_steps
    wl.sample_steps = [n_steps]
    return wl


def test_memory_budget_serialises_admission_and_everything_finishes():
    clk = Clock()
    be = FakeBackend(clk)
    a, b, c = _wl(100, 3), _wl(100, 2), _wl(10, 1)
    budget = serve.state_bytes(a, tjm.PREC_FP32_DEC32) + serve.state_bytes(c, tjm.PREC_FP32_DEC32)
    srv = serve.Server(mem_budget=budget, backend=be, clock=clk)
    for wl in (a, b, c):
        srv.submit(wl, arrival=0.0)
    peak = 0
    while srv.tick():
        peak = max(peak, srv.used)
        assert srv.used <= budget
    done = {r.rid: r for r in srv.finished}
    assert sorted(done) == [0, 1, 2]
    # a and c run together; b waits for memory until a retires
    assert done[1].admitted >= done[0].done
    assert done[2].admitted == 0.0
    assert all(r.ctx.closed for r in srv.finished)
    assert srv.used == 0
    rep = srv.report(0.0, clk.t)
    assert rep["requests"] == 3 and rep["p99_latency_s"] >= rep["p50_latency_s"] > 0
    srv.close()


def test_one_launch_per_tick_covers_all_active_runs():
    clk = Clock()
    be = FakeBackend(clk)
    srv = serve.Server(mem_budget=10 ** 12, steps_per_tick=2, backend=be, clock=clk)
    for n in (4, 2, 6):
        srv.submit(_wl(8, n), arrival=0.0)
    srv.drain()
    assert len(srv.finished) == 3
    # every launch carries the anchor run plus every request still active
    sizes = [len(x) for x in be.launches]
    assert sizes == [4, 3, 2]
    assert srv.launches == 3
    srv.close()


def test_arrivals_in_the_future_wait():
    clk = Clock()
    be = FakeBackend(clk)
    srv = serve.Server(mem_budget=10 ** 12, backend=be, clock=clk)
    srv.submit(_wl(4, 1), arrival=0.0)
    srv.submit(_wl(4, 1), arrival=5.0)
    assert srv.tick()              # first request admitted and run
    assert len(srv.active) + len(srv.finished) == 1 and len(srv.queue) == 1
    clk.t = 5.0
    while srv.tick():
        pass
    assert len(srv.finished) == 2 and srv.finished[1].admitted >= 5.0
    srv.close()


def test_replay_of_the_first_200_arrivals_of_the_request_stream():
    """C5's finite replay on the stand-in: the first 200 arrivals of the Poisson stream (20/s, seed 11),
    trajectory counts scaled by 1/64 and at most 5 steps each, under a 20 GB budget.  Every request
    finishes after it arrived, memory stays within the budget (or one oversize request running
    alone), requests that arrive while others run join the running batch, and the report is
    consistent."""
    import math
    clk = Clock()
    be = FakeBackend(clk)
    budget = 20 * 10 ** 9
    srv = serve.Server(mem_budget=budget, backend=be, clock=clk)
    stream = I.request_stream()[:200]
    biggest = 0
    for t_arr, wl in stream:
        wl.n_traj = max(1, int(math.ceil(wl.n_traj / 64)))
        wl.n_steps = min(wl.n_steps, 5)
        wl.sample_steps = [wl.n_steps]
        biggest = max(biggest, serve.state_bytes(wl, srv.precision))
        srv.submit(wl, arrival=t_arr)
    while srv.tick():
        assert srv.used <= max(budget, biggest)
        if not srv.active and srv.queue:       # idle until the next arrival: the stand-in clock jumps
            clk.t = max(clk.t, min(q.arrival for q in srv.queue))
    done = srv.finished
    assert len(done) == 200 and srv.used == 0 and not srv.queue
    assert all(r.admitted >= r.arrival and r.done > r.admitted for r in done)
    assert all(r.ctx.closed for r in done)
    assert any(a.admitted > b.admitted and a.admitted < b.done for a in done for b in done if a is not b)
    rep = srv.report(0.0, clk.t)
    assert rep["requests"] == 200 and rep["launches"] == len(be.launches)
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] > 0
    assert rep["sustained"] > 0 and rep["offered"] > rep["sustained"]
    srv.close()
