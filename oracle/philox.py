"""Philox4x32-10 counter-based generator (oracle side).

TEST INFRASTRUCTURE ONLY: this package is the CPU reference ("oracle") for the
tensor-jump-method hot path.  Only tests, the smoke check and the CPU baseline
leg of the benchmark may import it; the product path never does.

Published definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11 -- the Philox-4x32 round
(two 32x32->64 multiplies, xor with key and the other counter words) and the
Weyl key schedule, 10 rounds.  The paper being reproduced (TJM, Sec. "Stochastic
jump process") only needs a uniform epsilon in [0,1]; the generator choice and
the (key, counter) layout below are this project's reading:

    key     = (seed & 0xffffffff, seed >> 32)
    counter = (traj_id & 0xffffffff, traj_id >> 32, step, branch)

One block gives four 32-bit words -> two 53-bit uniforms u1 = U(x0, x1),
u2 = U(x2, x3) with U(a, b) = ((a >> 5) * 2**26 + (b >> 6)) * 2**-53, which lies
in [0, 1).  u1 decides whether a jump happens, u2 selects which.
"""
from __future__ import annotations

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85


def _round(c, k):
    p0 = PHILOX_M0 * c[0]
    p1 = PHILOX_M1 * c[2]
    hi0, lo0 = p0 >> 32, p0 & MASK32
    hi1, lo1 = p1 >> 32, p1 & MASK32
    return [(hi1 ^ c[1] ^ k[0]) & MASK32, lo1, (hi0 ^ c[3] ^ k[1]) & MASK32, lo0]


def philox4x32_10(counter, key):
    """Ten Philox-4x32 rounds on a 4-word counter with a 2-word key."""
    c = [int(x) & MASK32 for x in counter]
    k = [int(x) & MASK32 for x in key]
    for r in range(10):
        if r:
            k = [(k[0] + PHILOX_W0) & MASK32, (k[1] + PHILOX_W1) & MASK32]
        c = _round(c, k)
    return c


def u53(a: int, b: int) -> float:
    """Two 32-bit words -> a double in [0, 1) with 53 random bits."""
    return ((a >> 5) * 67108864 + (b >> 6)) * (1.0 / 9007199254740992.0)


def uniforms(seed: int, traj_id: int, step: int, branch: int):
    """(u1, u2) for one trajectory, one step and one branch (0 main, 1 sampling)."""
    key = (seed & MASK32, (seed >> 32) & MASK32)
    ctr = (traj_id & MASK32, (traj_id >> 32) & MASK32, step & MASK32, branch & MASK32)
    x = philox4x32_10(ctr, key)
    return u53(x[0], x[1]), u53(x[2], x[3])
