"""Bounded host wait (tjm_wait): TJM_ETIMEOUT while a launch is still running, TJM_OK once it is done."""
import numpy as np
import pytest

from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def test_wait_times_out_then_completes():
    lib_ready()
    L, chi = 200, 64
    ctx = tjm.Context(I.xxx_mpo(L, 1.0, 0.5), I.noise(L, 0.1, 0.1), 0.1, chi, 1e-10,
                      precision=tjm.PREC_FP32_DEC32)
    r = ctx.prepare(I.random_mps(L, chi, 5), 304, 0, I.z_observables(L), [0.1 * j for j in range(3)])
    ctx.advance(r, 1)                      # initialisation and one step: seconds of device work
    assert ctx.wait(r, 0.0) is False       # returned at once, the launch still running
    assert ctx.wait(r, 900.0) is True
    assert ctx.poll(r) is True
    with pytest.raises(tjm.TJMError):
        ctx.wait(r, -1.0)
    ctx.close()
