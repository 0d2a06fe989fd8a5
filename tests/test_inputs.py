"""The seeded input recipes are what they claim to be (no method arithmetic here; CPU only)."""
import math

import numpy as np

from paper_2501_17913_gb300 import inputs as I


def test_uneven_batch_enumerates_the_grid_then_draws():
    groups = I.uneven_groups()
    assert len(groups) == 32 and all(g.n_traj == 128 for g in groups)
    params = [(g.L, g.chi_max, g.meta['gamma']) for g in groups]
    grid = {(L, c, gm) for L in (50, 100, 200) for c in (16, 32, 64) for gm in (0.01, 0.1, 1.0)}
    assert set(params[:27]) == grid
    assert all(p[0] in (50, 100, 200) and p[1] in (16, 32, 64) and p[2] in (0.01, 0.1, 1.0) for p in params[27:])
    assert [g.meta['first_traj'] for g in groups] == [128 * i for i in range(32)]
    for g in groups[:3]:
        assert 0.0 <= g.meta['g'] <= 1.0 and g.n_steps == 100 and abs(g.dt - 0.05) < 1e-15
        psis = np.array(g.psi0_per_traj)
        assert psis.shape == (128, g.L, 2)
        assert np.allclose(np.linalg.norm(psis, axis=2), 1.0)
    assert [g.name for g in I.uneven_groups()] == [g.name for g in groups]     # seeded


def test_request_stream_ranges_and_rate():
    st = I.request_stream()
    assert len(st) == 200
    t = np.array([a for a, _ in st])
    assert np.all(np.diff(t) > 0)
    assert 0.5 * 200 / 20.0 < t[-1] < 2.0 * 200 / 20.0          # Poisson at 20/s
    for _, wl in st:
        assert 20 <= wl.L <= 500 and wl.chi_max in (16, 32, 64) and 100 <= wl.n_traj <= 2000
        assert 10 <= wl.n_steps <= 100 and abs(wl.dt - 0.1) < 1e-15
        rates = {r for (_, _, r) in wl.jumps}
        assert len(rates) == 1 and 0.01 <= rates.pop() <= 1.0


def test_random_mps_bonds_and_scale():
    chi, sites = I.random_mps(40, 64, 3)
    assert chi[0] == chi[-1] == 1 and max(chi) == 64
    assert chi[:8] == [1, 2, 4, 8, 16, 32, 64, 64]
    assert all(s.shape == (chi[l], 2, chi[l + 1]) for l, s in enumerate(sites))
    # entries of variance 1/(2 chi_right): the right transfer map keeps the identity on average
    b = sites[20]
    assert abs(np.mean(np.abs(b) ** 2) * 2 * b.shape[2] - 1.0) < 0.05


def test_bench_workload_matches_its_description():
    wl = I.config_bench()
    assert (wl.L, wl.chi_max, wl.n_traj, wl.dt) == (1000, 64, 256, 0.1)
    chi, sites = wl.meta['mps']
    assert len(sites) == 1000 and max(chi) == 64 and sum(c == 64 for c in chi) == 1001 - 2 * 6
    assert len(wl.jumps) == 2000 and {r for (_, _, r) in wl.jumps} == {0.1}
    assert math.isclose(float(np.sum(np.abs(np.asarray(wl.W[1])) > 0)), float(np.sum(np.abs(np.asarray(wl.W[2])) > 0)))
