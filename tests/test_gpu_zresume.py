"""Checkpoint / resume through the C ABI: a trajectory saved after step 2 and loaded into a fresh
run continues exactly as if it had never stopped (counter-based random numbers, FP64)."""
import numpy as np
import pytest

from paper_2501_17913_gb300 import inputs as I
from paper_2501_17913_gb300 import tjm

from gpu_common import lib_ready

pytestmark = pytest.mark.gpu


def test_resume_from_saved_state_matches_uninterrupted_run():
    lib_ready()
    L, chi, n, steps, cut = 8, 8, 4, 6, 2
    W, jumps, obs = I.xxx_mpo(L, 1.0, 0.5), I.noise(L, 0.2, 0.1), I.z_observables(L) + [(3, I.X)]
    times = [0.1 * j for j in range(steps + 1)]
    mk = lambda: tjm.Context(W, jumps, 0.1, chi, 1e-10, precision=tjm.PREC_FP64)
    psi = np.array(I.neel(L))
    a = mk()
    ra = a.run(psi, n, 11, obs, times)
    full = a.result(ra)[2]
    b = mk()
    rb = b.prepare(psi, n, 11, obs, times)
    b.advance(rb, cut)
    b.sync()
    saved = [b.get_state(rb, t) for t in range(n)]
    assert all(s[0] == cut for s in saved)
    c = mk()
    rc = c.prepare(psi, n, 11, obs, times)
    for t, (step, chi_t, sites) in enumerate(saved):
        c.set_state(rc, t, step, sites)
    c.advance(rc, steps - cut)
    resumed = c.result(rc)[2]
    assert np.abs(resumed[:, cut + 1:] - full[:, cut + 1:]).max() < 1e-10
    for x in (a, b, c):
        x.close()


def test_checkpoint_refused_between_the_halves_of_a_step():
    """After advance(-1) a trajectory holds X = U[dt] Phi_j, not a state a run can resume from:
    tjm_run_get_state refuses it (TJM_EBUSY); after advance(-2) completes the step it is Phi_{j+1}
    and the checkpoint resumes exactly."""
    lib_ready()
    L, chi, n, steps = 6, 8, 2, 4
    W, jumps, obs = I.xxx_mpo(L, 1.0, 0.5), I.noise(L, 0.2, 0.1), I.z_observables(L)
    times = [0.1 * j for j in range(steps + 1)]
    mk = lambda: tjm.Context(W, jumps, 0.1, chi, 1e-10, precision=tjm.PREC_FP64)
    psi = np.array(I.neel(L))
    b = mk()
    rb = b.prepare(psi, n, 5, obs, times)
    b.advance(rb, 1)
    b.advance(rb, -1)
    b.sync()
    with pytest.raises(tjm.TJMError) as err:
        b.get_state(rb, 0)
    assert err.value.status == tjm.TJM_EBUSY
    b.advance(rb, -2)
    b.sync()
    saved = [b.get_state(rb, t) for t in range(n)]
    assert all(s[0] == 2 for s in saved)
    a = mk()
    ra = a.run(psi, n, 5, obs, times)
    full = a.result(ra)[2]
    c = mk()
    rc = c.prepare(psi, n, 5, obs, times)
    for t, (step, chi_t, sites) in enumerate(saved):
        c.set_state(rc, t, step, sites)
    c.advance(rc, steps - 2)
    resumed = c.result(rc)[2]
    assert np.abs(resumed[:, 3:] - full[:, 3:]).max() < 1e-10
    for x in (a, b, c):
        x.close()
