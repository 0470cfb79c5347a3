"""Writes sample_stream.txt: expected sample-stream states and sample indices of the
sampling step (Section 6, "a random sample of size abr"), computed with plain Python
integers from the generator's published definition and the stream rule that
include/ams.h states for ams_step_sample.  It imports nothing from this repository,
so the file pins the oracle from outside.

SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), stateful form: next() adds the golden
gamma 0x9E3779B97F4A7C15 to the state (mod 2^64) and returns the state passed
through the finaliser z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
z *= 0x94D049BB133111EB; z ^= z >> 31.

Stream rule: the generator of the segment that starts at position `begin` at level
`level` (1-based) starts at state
    mix(mix(seed + (level+1)*gamma) + (begin+1)*gamma),
which is the first output of a generator seeded with (first output of a generator
seeded with seed + level*gamma) + begin*gamma.  Draw j (j = 0, 1, ...) is the
(j+1)-th output u_j, mapped to the index floor(u_j * n_g / 2^64).

    python tests/golden/make_sample_stream.py > tests/golden/sample_stream.txt
"""

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    def __init__(self, state):
        self.state = state & MASK

    def next(self):
        self.state = (self.state + GAMMA) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)


def stream_state(seed, level, begin):
    first = SplitMix64(seed + level * GAMMA).next()
    return SplitMix64(first + begin * GAMMA).next()


def draws(seed, level, begin, n_g, count):
    g = SplitMix64(stream_state(seed, level, begin))
    return [(g.next() * n_g) >> 64 for _ in range(count)]


CASES = [  # seed, level, begin, n_g
    (0, 1, 0, 1 << 20),
    (0, 2, 0, 1 << 20),
    (0, 1, 1, 1 << 20),
    (7, 1, 0, 1000),
    (7, 3, 123456, 4097),
    (123456789, 2, 65536, 1 << 28),
    (2**64 - 1, 1, 4294967295, 3),
    (5, 8, 17, 2**32 - 1),
]

if __name__ == "__main__":
    # the published outputs of the generator started at state 0 (the reference
    # implementation splitmix64.c) hold for this implementation
    g = SplitMix64(0)
    assert [g.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    print("# Sample stream of the sampling step (Section 6), from make_sample_stream.py")
    print("# (plain Python integers, SplitMix64 from its published definition).")
    print("# seed level begin n_g stream_state(hex) ; first 8 indices")
    for seed, level, begin, n_g in CASES:
        st = stream_state(seed, level, begin)
        idx = draws(seed, level, begin, n_g, 8)
        print(f"{seed} {level} {begin} {n_g} {st:016x} ; {' '.join(str(i) for i in idx)}")
