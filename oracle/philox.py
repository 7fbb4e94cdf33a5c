"""Philox4x32-10 and the draws the trajectory consumes (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Philox4x32-10 is the counter-based generator of Salmon et al., SC'11, Sec. 4:
a 4 x 32-bit counter and a 2 x 32-bit key go through ten rounds; each round
multiplies counter words 0 and 2 by the constants M0, M1 into 64-bit
products, swaps and xors the halves with the key, and the key is advanced by
the Weyl constants W0, W1 between rounds.

The measurement randomness of App. A (the site choice and Born draw of the
projective protocol, the Gaussian increments dW of the homodyne protocol) is
taken from this stream at the counter

    ctr = (site, step, traj_id & 0xffffffff, tag | ((traj_id >> 32) << 8)),
    key = (seed & 0xffffffff, seed >> 32),

with tag MEASURE for the projective draws and NOISE for the Gaussian ones.
One call yields four 32-bit words w0..w3.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

TAG_MEASURE = 1
TAG_NOISE = 2
TAG_EVENT = 3           # continuous-time projective protocol: waiting time and site of event e
TAG_EVENT_OUTCOME = 4   # ... and its Born draw


def philox4x32_10(ctr, key):
    """Ten Philox rounds.  ``ctr``: 4 arrays (or ints) of uint32 values, ``key``: 2.

    Returns four uint64 arrays holding the 32-bit output words.
    """
    c = [np.asarray(x, dtype=np.uint64) & MASK32 for x in ctr]
    c = list(np.broadcast_arrays(*c))
    c = [x.copy() for x in c]
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c[0]          # < 2^64, exact in uint64
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def counter(site, step, traj_id, tag):
    """The counter words for (site, step, trajectory, tag); ``site`` may be an array."""
    traj_id = int(traj_id)
    return (np.asarray(site, dtype=np.uint64),
            np.uint64(step & 0xFFFFFFFF),
            np.uint64(traj_id & 0xFFFFFFFF),
            np.uint64((tag | ((traj_id >> 32) << 8)) & 0xFFFFFFFF))


def key_of(seed):
    seed = int(seed)
    return (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def uniform53(wa, wb):
    """Uniform double in [0, 1) from two words: 27 high bits of wa, 26 of wb."""
    a = (np.asarray(wa, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(wb, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0)


def measure_draws(seed, traj_id, step, L):
    """Projective protocol: (u_select, u_outcome) for every site of one step."""
    w = philox4x32_10(counter(np.arange(L), step, traj_id, TAG_MEASURE), key_of(seed))
    return uniform53(w[0], w[1]), uniform53(w[2], w[3])


def noise_normals(seed, traj_id, step, L):
    """Homodyne protocol: xi_i ~ N(0,1) per site by the Box-Muller transform."""
    w = philox4x32_10(counter(np.arange(L), step, traj_id, TAG_NOISE), key_of(seed))
    u1 = uniform53(w[0], w[1])
    u2 = uniform53(w[2], w[3])
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def poisson_event(seed, traj_id, e, L):
    """Continuous-time projective protocol (App. A): the draws of event e of a trajectory.

    Counter (e & 0xffffffff, e >> 32, trajectory, tag): u_wait from words 0-1 of tag
    EVENT (the waiting time is -ln(1 - u_wait) / rate), the site floor(u_site L) from
    words 2-3, the Born draw u from words 0-1 of tag EVENT_OUTCOME."""
    e = int(e)
    w = philox4x32_10(counter(e & 0xFFFFFFFF, e >> 32, traj_id, TAG_EVENT), key_of(seed))
    v = philox4x32_10(counter(e & 0xFFFFFFFF, e >> 32, traj_id, TAG_EVENT_OUTCOME), key_of(seed))
    u_wait = float(uniform53(w[0], w[1]))
    site = min(int(float(uniform53(w[2], w[3])) * L), L - 1)
    return u_wait, site, float(uniform53(v[0], v[1]))
