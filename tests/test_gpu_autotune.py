"""GEMM tile rules on the GPU: both rules compute the same trajectories, and the autotuner drives real runs."""
import numpy as np
import pytest

from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm
from paper_2501_17913_gb300.autotune import TileAutotuner

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _stepped(prec, rule=None, tuner=None, L=24, chi=16, n=48, steps=8):
    lib_ready()
    W, jumps = I.xxx_mpo(L, 1.0, 0.5), I.noise(L, 0.1, 0.1)
    ctx = tjm.Context(W, jumps, 0.1, chi, 1e-10, precision=prec)
    r = ctx.prepare(np.array(I.neel(L)), n, 3, I.z_observables(L), [0.1 * j for j in range(steps + 1)])
    used = []
    for _ in range(steps + 1):
        if tuner is None:
            ctx.set_tile_rule(r, rule)
            ctx.advance(r, 1)
        else:
            used.append(tuner.advance(ctx, r, 1))
    ctx.sync()
    pt = ctx.result(r)[2]
    ctx.close()
    return pt, used


def test_tile_rules_agree_fp64():
    a, _ = _stepped(tjm.PREC_FP64, rule=0)
    b, _ = _stepped(tjm.PREC_FP64, rule=1)
    assert np.abs(a - b).max() < 1e-10


def test_autotuned_run_matches_fixed_rule_fp32():
    tu = TileAutotuner()
    a, _ = _stepped(tjm.PREC_FP32_DEC32, rule=0, steps=4)
    b, used = _stepped(tjm.PREC_FP32_DEC32, tuner=tu, steps=4)
    assert set(used[:3]) == {0, 1}          # both rules timed (the first launch only initialises)
    assert (tjm.PREC_FP32_DEC32, 16) in tu.best
    assert np.abs(a - b).max() < 1e-4


def test_tile_rule_rejects_unknown_rule():
    lib_ready()
    ctx = tjm.Context(I.xxx_mpo(4, 1.0, 0.5), [], 0.1, 4, 1e-10)
    r = ctx.prepare(None, 1, 0, I.z_observables(4), [0.0])
    with pytest.raises(tjm.TJMError):
        ctx.set_tile_rule(r, 2)
    ctx.close()
