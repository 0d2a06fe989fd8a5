"""Element-wise parity of the kernel's contractions with the oracle's.

The one-site, two-site and bond effective Hamiltonians (Fig. 2) and the left /
right environment updates, applied by the trajectory kernel's own device
functions (tjm_selftest_contract), against oracle.mps_tjm.heff1 / heff2 /
heff0 / env_left_update / env_right_update on random tensors at chi in
{16, 32, 64} with the XXX MPO (D = 5): FP64 to 1e-12, FP32 on the CUDA cores
and on the tensor cores (3xTF32) element by element within a few FP32 units of
the same contraction taken over absolute values.
"""
import numpy as np
import pytest

from oracle import mps_tjm as O1
from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def _rand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


ARMS = [("fp64", tjm.PREC_FP64, False, 1e-12), ("fp32", tjm.PREC_FP32, False, 1e-5),
        ("tf32x3", tjm.PREC_FP32, True, 1e-5)]


@pytest.mark.parametrize("chi", [16, 32, 64])
@pytest.mark.parametrize("arm", ARMS, ids=[a[0] for a in ARMS])
def test_contractions_match_oracle(chi, arm):
    _, prec, tc, tol = arm
    lib_ready()
    rng = np.random.default_rng(chi)
    W = I.xxx_mpo(6, 1.0, 0.5)
    Wb = np.asarray(W[2])                      # a bulk site, D = 5
    D = Wb.shape[0]
    chl, chr_ = chi, chi if chi < 64 else 48   # a ragged right bond at the largest size
    Lenv = _rand(rng, chl, D, chl)
    Renv = _rand(rng, D, chr_, chr_)
    M = _rand(rng, chl, 2, chr_)
    th = _rand(rng, chl, 2, 2, chr_)
    C = _rand(rng, chl, chr_)
    cases = [
        (1, dict(Lenv=Lenv, Renv=Renv, x=M, W1=Wb), O1.heff1(Lenv, Wb, Renv, M),
         O1.heff1(abs(Lenv), abs(Wb), abs(Renv), abs(M))),
        (2, dict(Lenv=Lenv, Renv=Renv, x=th, W1=Wb, W2=Wb), O1.heff2(Lenv, Wb, Wb, Renv, th),
         O1.heff2(abs(Lenv), abs(Wb), abs(Wb), abs(Renv), abs(th))),
        (0, dict(Lenv=Lenv, Renv=Renv[:, :, :], x=C), O1.heff0(Lenv, Renv, C),
         O1.heff0(abs(Lenv), abs(Renv), abs(C))),
        (3, dict(Lenv=Lenv, Renv=np.zeros((1, 1, 1)), x=M, W1=Wb), O1.env_left_update(Lenv, M, Wb),
         O1.env_left_update(abs(Lenv), abs(M), abs(Wb))),
        (4, dict(Lenv=np.zeros((1, 1, 1)), Renv=Renv, x=M, W1=Wb), O1.env_right_update(Renv, M, Wb),
         O1.env_right_update(abs(Renv), abs(M), abs(Wb))),
    ]
    for kind, kw, ref, mag in cases:
        got = tjm.selftest_contract(kind, prec, tensor_cores=tc, **kw)
        assert got.shape == ref.shape, (kind, got.shape, ref.shape)
        err = np.abs(got - ref)
        assert (err <= tol * mag + 1e-300).all(), (kind, chi, float((err / mag).max()))
