"""Counter-free seeded RNG: splitmix64 seeding a xoshiro256** generator.

Both are the published public-domain generators of Vigna and Blackman
("Scrambled linear pseudorandom number generators", 2018/2021): splitmix64
expands one 64-bit seed into the 256-bit xoshiro state; xoshiro256** then
produces 64-bit outputs.  Written here in plain Python from those definitions
so that every input draw is reproducible on any host.
"""
import math

_M64 = (1 << 64) - 1


def splitmix64(state):
    """One splitmix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & _M64


class Xoshiro256ss:
    """xoshiro256** with the state filled by splitmix64(seed)."""

    def __init__(self, seed):
        st = seed & _M64
        s = []
        for _ in range(4):
            st, out = splitmix64(st)
            s.append(out)
        self.s = s

    def next_u64(self):
        s = self.s
        result = (_rotl((s[1] * 5) & _M64, 7) * 9) & _M64
        t = (s[1] << 17) & _M64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self, lo=0.0, hi=1.0):
        """Uniform double in [lo, hi) from the top 53 bits."""
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, mu=0.0, sd=1.0):
        """Gaussian draw by the Box-Muller transform (one output per call)."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return mu + sd * math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def choice(self, items):
        return items[int(self.uniform() * len(items)) % len(items)]
