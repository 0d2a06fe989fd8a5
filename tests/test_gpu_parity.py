"""CUDA path against the oracle, trajectory by trajectory (through the C ABI).

Tolerances: 1e-10 absolute on every observable in the FP64 path, 1e-4 in the
FP32 paths.  Trajectories whose oracle run had a jump decision closer than
the decision margin (|u1 - dp| or the pick gap) are excluded from the
per-trajectory comparison (their branch can legitimately flip); they are
counted and must stay rare.
"""
import numpy as np
import pytest

from oracle import dense as O2
from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from _pool import oracle_pool
from gpu_common import run_gpu
from oracle_jobs import run_traj

pytestmark = pytest.mark.gpu


def _oracle(name, kw, trajs, opts):
    with oracle_pool() as pool:
        return pool.map(run_traj, [(name, kw, t, opts) for t in trajs])


def _compare(gpu_vals, oracle_res, tol, margin):
    ok, skipped, worst = 0, 0, 0.0
    for g, (v, st) in zip(gpu_vals, oracle_res):
        if min(st['min_margin1'], st['min_margin2']) < margin:
            skipped += 1
            continue
        worst = max(worst, float(np.abs(g - v).max()))
        ok += 1
    return ok, skipped, worst


@pytest.mark.parametrize("chi_max,kind", [(16, 'two'), (2, 'one'), (4, 'mixed')])
def test_exact_mode_fp64(chi_max, kind):
    """Full bond dimension: the GPU trajectory equals the dense Strang MCWF (via the oracle) to 1e-10."""
    L, n = 5, 8
    wl = I.Workload('exact', I.xxx_mpo(L, 1.0, 0.5), I.noise(L, 0.2, 0.1), 0.1, n, chi_max, 0.0, 6, 5,
                    I.neel(L), I.z_observables(L) + [(2, I.X)], list(range(n + 1)))
    pt, mean, sem, st, _, _ = run_gpu(wl, tjm.PREC_FP64, exact=True)
    prob = O1.Problem(wl.W, wl.jumps, wl.dt, chi_max, 0.0, exact=True)
    for t in range(wl.n_traj):
        v, _ = O1.run_trajectory(prob, O1.padded_product_mps(wl.psi0), t, wl.seed, wl.observables, n,
                                 wl.sample_steps)
        assert np.abs(pt[t] - v).max() < 1e-10, (t, np.abs(pt[t] - v).max())
    assert st['failed'] == 0
    if kind == 'one':
        assert st['matvec_two_site'] == 0
    if kind == 'two':
        assert st['matvec_bond'] == 0


def test_small_chain_fp64_all_trajectories_and_lindblad():
    """L=6, chi_max=16, 200 trajectories: per trajectory vs the oracle (1e-10), ensemble vs exact Lindblad."""
    wl = I.config_small_fp64()
    pt, mean, sem, st, _, _ = run_gpu(wl, tjm.PREC_FP64)
    res = _oracle('config_small_fp64', {}, range(wl.n_traj), {})
    ok, skipped, worst = _compare(pt, res, 1e-10, 1e-9)
    assert worst < 1e-10, worst
    assert skipped <= 2 and ok >= wl.n_traj - 2
    H = O2.mpo_to_dense(wl.W)
    psi = O2.product_state(wl.psi0)
    rhos = O2.lindblad_evolve(H, wl.jumps, wl.L, np.outer(psi, psi.conj()), wl.times)
    exact = np.array([[O2.expect(r, I.Z, l, wl.L) for l in range(wl.L)] for r in rhos])
    z = np.abs(mean - exact)[1:] / np.maximum(sem[1:], 1e-3)
    assert np.mean(z < 3) >= 0.99 and z.max() < 5
    # the library's mean / sem are the plain statistics of its per-trajectory values
    assert np.allclose(mean, pt.mean(axis=0), atol=1e-14)
    assert np.allclose(sem, pt.std(axis=0, ddof=1) / np.sqrt(wl.n_traj), atol=1e-14)


@pytest.mark.parametrize("prec", [tjm.PREC_FP32, tjm.PREC_FP32_DF64, tjm.PREC_FP32_DEC32])
def test_small_chain_fp32_paths(prec):
    """L=6, 64 trajectories, FP32 contractions: per trajectory within 1e-4 of the FP64 oracle for the
    first 30 of 50 steps (rounding differences grow along a trajectory; the margins counted are those
    of the decisions up to step 30), and the ensemble within the 3-SE rule of the oracle's at all steps."""
    horizon = 30
    wl = I.config_small_fp64(64)
    pt, mean, sem, st, _, _ = run_gpu(wl, prec)
    res = _oracle('config_small_fp64', {'n_traj': 64}, range(64), {})
    ok, worst = 0, 0.0
    for g, (v, so) in zip(pt, res):
        if so['margin_upto'][horizon] < 1e-5:
            continue
        worst = max(worst, float(np.abs(g[:horizon + 1] - v[:horizon + 1]).max()))
        ok += 1
    assert worst < 1e-4, worst
    assert ok >= 60
    om = np.array([v for v, _ in res])
    se = np.sqrt(sem ** 2 + (om.std(axis=0, ddof=1) / np.sqrt(len(om))) ** 2)
    z = np.abs(mean - om.mean(axis=0))[1:] / np.maximum(se[1:], 1e-4)
    assert np.mean(z < 3) >= 0.99 and z.max() < 5


@pytest.mark.parametrize("prec", [tjm.PREC_FP32, tjm.PREC_FP32_DF64, tjm.PREC_FP32_DEC32])
def test_small_chain_tensor_core_path(prec):
    """The tcgen05 build of the trajectory kernel with every FP32 contraction sent to the tensor cores
    (tc_min_work = 1): per trajectory within 1e-4 of the FP64 oracle for the first 20 steps, as the
    CUDA-core build is held to."""
    horizon = 20
    wl = I.config_small_fp64(32)
    pt, _, _, st, _, ctx = run_gpu(wl, prec, n_steps=horizon, tensor_cores=True, tc_min_work=1)
    assert ctx.resident_ctas() > 0
    res = _oracle('config_small_fp64', {'n_traj': 32}, range(32), {})
    ok, worst = 0, 0.0
    for g, (v, so) in zip(pt, res):
        if so['margin_upto'][horizon] < 1e-5:
            continue
        worst = max(worst, float(np.abs(g[:horizon + 1] - v[:horizon + 1]).max()))
        ok += 1
    assert worst < 1e-4, worst
    assert ok >= 28


def test_cuda_core_kernels_run_two_ctas_per_sm():
    """The CUDA-core builds of the trajectory kernel hold no tcgen05 code and are resident at two CTAs
    (of 256 threads, 128 registers) per SM; the tensor-core build at one."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    wl = I.config_small_fp64(4)
    for prec in (tjm.PREC_FP64, tjm.PREC_FP32, tjm.PREC_FP32_DF64, tjm.PREC_FP32_DEC32):
        ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=prec)
        assert ctx.resident_ctas() == 2 * sms, (prec, ctx.resident_ctas())
        ctx.close()
    ctx = tjm.Context(wl.W, wl.jumps, wl.dt, wl.chi_max, wl.trunc_eps, precision=tjm.PREC_FP32_DF64,
                      tensor_cores=True)
    assert ctx.resident_ctas() == sms
    ctx.close()


def test_edge_cases_fp64():
    """Two sites, chi_max = 1, one trajectory, no noise, only t = 0, H = 0."""
    obs = I.z_observables(2) + [(0, I.X)]
    for (W, jumps, chi, steps) in [
        (I.xxx_mpo(2, 1.0, 0.5), I.noise(2, 0.3, 0.2), 4, 6),      # two sites
        (I.xxx_mpo(4, 1.0, 0.5), I.noise(4, 0.3, 0.2), 1, 5),      # chi_max = 1: product-state TDVP
        (I.xxx_mpo(3, 1.0, 0.5), [], 4, 5),                        # no jump operators
        (I.xxx_mpo(3, 0.0, 0.0), I.noise(3, 0.5, 0.0), 4, 5),      # H = 0: Lanczos breakdown at once
        (I.xxx_mpo(3, 1.0, 0.5), I.noise(3, 0.1, 0.1), 4, 0),      # only t = 0
    ]:
        L = len(W)
        ob = [(s, o) for (s, o) in obs if s < L]
        wl = I.Workload('edge', W, jumps, 0.1, steps, chi, 1e-10, 3, 9, I.neel(L), ob, list(range(steps + 1)))
        pt, mean, sem, st, _, _ = run_gpu(wl, tjm.PREC_FP64)
        prob = O1.Problem(wl.W, wl.jumps, wl.dt, chi, 1e-10)
        for t in range(wl.n_traj):
            v, _ = O1.run_trajectory(prob, O1.product_mps(wl.psi0), t, wl.seed, wl.observables, steps,
                                     wl.sample_steps)
            assert np.abs(pt[t] - v).max() < 1e-10, (L, chi, steps, t, np.abs(pt[t] - v).max())


def test_invalid_arguments_are_rejected():
    from gpu_common import lib_ready
    lib_ready()
    W = I.xxx_mpo(3)
    with pytest.raises(tjm.TJMError):
        tjm.Context(W, I.noise(3), -0.1, 4, 1e-10)           # dt <= 0
    with pytest.raises(tjm.TJMError):
        tjm.Context(W, [(7, I.SM, 0.1)], 0.1, 4, 1e-10)      # jump site out of range
    ctx = tjm.Context(W, I.noise(3), 0.1, 4, 1e-10)
    with pytest.raises(tjm.TJMError):
        ctx.run(I.neel(3), 2, 0, I.z_observables(3), [0.0, 0.15])   # off the dt grid
    with pytest.raises(tjm.TJMError):
        ctx.run(I.neel(3), 2, 0, [(5, I.Z)], [0.1])                 # observable site out of range
    ctx.close()
