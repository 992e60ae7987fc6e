"""Counter-based random draws for the active sets (oracle; test infrastructure).

Algorithm 1 step 3 generates the active set: block i is used at iteration t
with probability p_i, independently of everything else (Sec. 3, "Algorithm
convergence": entries of A chosen independently at each iteration). The paper
names no generator. Reading: Philox-4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11),
with key (seed, 0) and counter (t, stream, index, 0); stream 0 draws the data
blocks, stream 1 the sparsity bases. Word 0 of the output gives
u = (word0 >> 11) * 2^-53 in [0, 1), and the item is active iff u < p.
Written from the published round function in pure Python (integers).
"""

_MASK = (1 << 64) - 1
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B

STREAM_BLOCKS = 0
STREAM_BASES = 1


def philox4x64_10(counter, key):
    """Ten rounds of Philox-4x64 on a 4-word counter with a 2-word key."""
    c0, c1, c2, c3 = (int(w) & _MASK for w in counter)
    k0, k1 = (int(w) & _MASK for w in key)
    for rnd in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 64, p0 & _MASK
        hi1, lo1 = p1 >> 64, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if rnd < 9:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def uniform(seed, t, stream, index):
    """u in [0, 1) for item ``index`` of ``stream`` at iteration ``t``."""
    w0 = philox4x64_10((t, stream, index, 0), (seed, 0))[0]
    return (w0 >> 11) * (2.0 ** -53)


def active_set(seed, t, stream, probs):
    """Boolean activity of every item at iteration t: u < p_i (Alg. 1 step 3)."""
    return [uniform(seed, t, stream, i) < float(p) for i, p in enumerate(probs)]
