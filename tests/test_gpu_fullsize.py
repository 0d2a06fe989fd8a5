"""Parity at the full workload sizes, on trajectories the oracle computes one by one.

The oracle values are stored by tests/golden/make_golden.py (oracle only).
Every trajectory of a full-size run is also checked for properties that hold
at any size: finite outputs, |<Z_i>| <= 1, status OK, bonds <= chi_max.

A TJM trajectory is a chaotic map of its state: a difference of one rounding
unit grows by roughly an order of magnitude every few steps, and once it
exceeds the margin of a jump decision the two runs draw different jumps.
Per-trajectory agreement with the oracle therefore holds up to a horizon that
depends on the arithmetic (FP64 contractions and factorizations; FP32
contractions with FP64 factorizations; everything in FP32); beyond it the
ensembles are compared within their standard errors.
"""
import os

import numpy as np
import pytest

from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready, run_gpu

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# (last step checked, tolerance, decision margin) per precision on the L=30 chain: a decision can
# flip only when its margin is below the difference in the state, so the FP64 margin is tiny
HORIZON = {tjm.PREC_FP64: (25, 1e-10, 1e-8), tjm.PREC_FP32: (20, 1e-4, 1e-4),
           tjm.PREC_FP32_DF64: (20, 1e-4, 1e-4), tjm.PREC_FP32_DEC32: (5, 1e-4, 1e-4)}
FP64_ALL_STEPS = 1e-6
_CACHE = {}     # the FP64 L=30 ensemble, shared by the FP32-path comparisons


def _gold(name):
    p = os.path.join(GOLD, "oracle_%s.npz" % name)
    if not os.path.exists(p):
        pytest.skip("stored oracle values %s missing (tests/golden/make_golden.py %s)" % (p, name))
    return np.load(p)


def _check_properties(pt, st, chi_max):
    assert np.isfinite(pt).all()
    assert np.abs(pt).max() <= 1.0 + 1e-5
    assert st['failed'] == 0
    assert st['final_bond_max'] <= chi_max


def _compare_sampled(pt, g, tol, margin, last_step=None):
    """Sampled trajectories pt[traj] against the stored oracle values up to last_step."""
    ok = 0
    sl = slice(None) if last_step is None else slice(0, last_step + 1)
    for k, t in enumerate(g['traj']):
        # the smallest margin of the decisions taken up to the last compared step
        if g['margin_upto'][k][-1 if last_step is None else last_step] < margin:
            continue
        err = float(np.abs(pt[t][sl] - g['values'][k][sl]).max())
        assert err < tol, (int(t), err)
        ok += 1
    # at L = 1000 a jump is picked among 2000 channels of ~5e-4 weight each, so pick margins below the
    # FP32 threshold are common; at least half of the sampled trajectories must be comparable
    assert ok >= max(1, len(g['traj']) // 2), (ok, len(g['traj']))
    return ok


def _sampled_runs(wl, g, prec, extra=0):
    """The sampled L=30 trajectories, each its own run, all in one launch -- with `extra` more
    trajectories (global ids 1024 ...) in the same launch for an ensemble; returns ({id: values}, extra
    per-trajectory values, their stats)."""
    lib_ready()
    ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=prec)
    runs = [ctx.prepare(np.array(wl.psi0), 1, wl.seed, wl.observables, wl.times, first_traj=int(t))
            for t in g['traj']]
    pairs = [(ctx, r) for r in runs]
    if extra:
        rx = ctx.prepare(np.array(wl.psi0), extra, wl.seed, wl.observables, wl.times, first_traj=wl.n_traj)
        pairs.append((ctx, rx))
    tjm.group_advance(pairs, wl.n_steps + 1)
    pt = {}
    for t, r in zip(g['traj'], runs):
        pt[int(t)] = ctx.result(r)[2][0]
    ptx = stx = None
    if extra:
        ptx = ctx.result(rx)[2]
        stx = ctx.stats(rx)
    ctx.close()
    return pt, ptx, stx


def _fp64_l30(g, wl):
    """FP64 on the L=30 chain, computed once: the 32 sampled trajectories plus 272 more, all in one
    launch (one resident wave of 304 CTAs, so the ensemble costs no more time than the sampled
    trajectories)."""
    if "l30_fp64" not in _CACHE:
        pt, ptx, stx = _sampled_runs(wl, g, tjm.PREC_FP64, extra=272)
        _check_properties(ptx, stx, wl.chi_max)
        allv = np.concatenate([np.array([pt[int(t)] for t in g['traj']]), ptx])
        _CACHE["l30_fp64"] = (pt, allv.mean(axis=0), allv.std(axis=0, ddof=1) / np.sqrt(len(allv)))
    return _CACHE["l30_fp64"]


@pytest.mark.parametrize("prec", [tjm.PREC_FP64, tjm.PREC_FP32, tjm.PREC_FP32_DF64, tjm.PREC_FP32_DEC32])
def test_l30_sampled_trajectories_to_horizon(prec):
    """L=30, chi_max=32, 100 steps: the 32 sampled trajectories against the oracle up to the precision's
    horizon."""
    g = _gold("l30")
    wl = I.config_l30()
    pt = _fp64_l30(g, wl)[0] if prec == tjm.PREC_FP64 else _sampled_runs(wl, g, prec)[0]
    last, tol, margin = HORIZON[prec]
    _compare_sampled(pt, g, tol, margin, last_step=last)
    if prec == tjm.PREC_FP64:
        _compare_sampled(pt, g, FP64_ALL_STEPS, margin)


@pytest.mark.parametrize("prec", [tjm.PREC_FP32_DF64])
def test_l30_1024_trajectories_ensemble_fp32_vs_fp64(prec):
    """All 1024 L=30 trajectories for 100 steps in the benchmark's arithmetic: properties of every
    trajectory, the sampled ones to the horizon, and the ensemble mean within 3 standard errors of an
    FP64 ensemble of 304 trajectories (FP64 runs at GB300's FP64 rate; the combined standard error
    accounts for the smaller sample).  The all-FP32 mode is checked per trajectory above."""
    g = _gold("l30")
    wl = I.config_l30()
    pt, mean, sem, st, _, ctx = run_gpu(wl, prec)
    ctx.close()
    _check_properties(pt, st, wl.chi_max)
    last, tol, margin = HORIZON[prec]
    _compare_sampled(pt, g, tol, margin, last_step=last)
    _, mean64, sem64 = _fp64_l30(g, wl)
    se = np.sqrt(sem ** 2 + sem64 ** 2)
    se = np.maximum(se, 1e-4)
    z = np.abs(mean - mean64) / se
    assert (z <= 3.0).mean() >= 0.99, (z > 3.0).mean()
    assert z.max() <= 5.0, z.max()


@pytest.mark.parametrize("prec,tol", [(tjm.PREC_FP64, 1e-10), (tjm.PREC_FP32, 1e-4), (tjm.PREC_FP32_DF64, 1e-4),
                                      (tjm.PREC_FP32_DEC32, 1e-4)])
def test_l1000_neel_first_steps(prec, tol):
    """L=1000, chi_max=64, 256 trajectories from Neel, 3 steps: sampled trajectories against the oracle."""
    g = _gold("l1000")
    wl = I.config_l1000()
    pt, mean, sem, st, _, ctx = run_gpu(wl, prec, n_steps=int(g['n_steps']))
    ctx.close()
    _check_properties(pt, st, wl.chi_max)
    _compare_sampled(pt, g, tol, 1e-8 if prec == tjm.PREC_FP64 else 2e-5)


@pytest.mark.parametrize("prec,tol", [(tjm.PREC_FP32_DF64, 1e-4), (tjm.PREC_FP32, 1e-4)])
def test_bench_workload_one_step(prec, tol):
    """The benchmark launch: L=1000, chi=64-saturated random MPS, 256 trajectories, one step, in the
    benchmark's mode (FP32 contractions, emulated-FP64 factorizations) and with native FP64
    factorizations (the all-FP32 mode is checked at L=1000 from Neel)."""
    g = _gold("bench")
    wl = I.config_bench()
    pt, mean, sem, st, _, ctx = run_gpu(wl, prec, n_steps=1, psi=wl.meta['mps'])
    ctx.close()
    _check_properties(pt, st, wl.chi_max)
    _compare_sampled(pt, g, tol, 1e-5)


LONG = os.environ.get("TJM_LONG_GPU_TESTS") == "1"


@pytest.mark.parametrize("n_steps", [
    25, pytest.param(100, marks=pytest.mark.skipif(not LONG, reason="the full T = 5: minutes of GPU time; "
                                                   "run with TJM_LONG_GPU_TESTS=1"))])
def test_uneven_batch_one_launch_matches_alone_and_oracle(n_steps):
    """The uneven batch: all 32 groups (L in {50,100,200}, chi_max in {16,32,64}, gamma in {0.01,0.1,1},
    g ~ U[0,1], Haar-random product states from seed 7, dt = 0.05) in ONE persistent launch, for the
    full 100 steps (T = 5; run on request) or the first 25, PER_GROUP trajectories per group (the full
    128 per group is 48 M trajectory*site*steps, hours of GPU time).  Every group's trajectories equal,
    bit for bit, the same trajectories run in a launch of their own (all 32 single-group launches in
    flight at once on their own streams), and one trajectory of every group matches the oracle over the
    first 3 steps."""
    from _pool import oracle_pool
    from oracle_jobs import run_traj
    lib_ready()
    PER_GROUP = 4
    groups = I.uneven_groups()
    assert groups[0].n_steps == 100
    samples = [0, 1, 2, 3, n_steps // 2, n_steps]
    ctxs, runs = [], []
    for wl in groups:
        ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=tjm.PREC_FP32_DF64)
        r = ctx.prepare(np.array(wl.psi0_per_traj[:PER_GROUP]), PER_GROUP, wl.seed, wl.observables,
                        [s * wl.dt for s in samples], first_traj=wl.meta['first_traj'])
        ctxs.append(ctx)
        runs.append(r)
    tjm.group_advance(list(zip(ctxs, runs)), n_steps + 1)
    mixed = []
    for ctx, r, wl in zip(ctxs, runs, groups):
        pt = ctx.result(r)[2]
        st = ctx.stats(r)
        _check_properties(pt, st, wl.chi_max)
        assert st['steps_done_min'] == n_steps
        mixed.append(pt)
    # alone: each group in its own launch, all launched before any result is read
    alone_ctx, alone_run = [], []
    for wl in groups:
        ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=tjm.PREC_FP32_DF64)
        r = ctx.run(np.array(wl.psi0_per_traj[:2]), 2, wl.seed, wl.observables, [s * wl.dt for s in samples],
                    first_traj=wl.meta['first_traj'])
        alone_ctx.append(ctx)
        alone_run.append(r)
    for gi, (ctx, r) in enumerate(zip(alone_ctx, alone_run)):
        alone = ctx.result(r)[2]
        assert np.array_equal(alone, mixed[gi][:2]), gi
        ctx.close()
    # oracle: trajectory 0 of every group over the first 3 steps (product start: cheap)
    jobs = [('uneven_group', {'gi': gi, 'n_steps': 3}, 0, {'n_steps': 3, 'traj_offset': groups[gi].meta['first_traj']})
            for gi in range(len(groups))]
    with oracle_pool() as pool:
        res = pool.map(run_traj, jobs)
    checked = 0
    for gi, (v, stt) in enumerate(res):
        if min(stt['min_margin1'], stt['min_margin2']) < 1e-5:
            continue
        assert np.abs(mixed[gi][0][:4] - v).max() < 1e-4, (gi, np.abs(mixed[gi][0][:4] - v).max())
        checked += 1
    assert checked >= len(groups) - 4, checked
    for ctx in ctxs:
        ctx.close()
