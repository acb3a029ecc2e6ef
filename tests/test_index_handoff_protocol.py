"""The index pass kernel's hand-offs between its compute warps and its
look-back warp (k_simplex_index), modelled on the host: hardware named
barriers complete a generation when the expected thread count has arrived
(compute warps 480, look-back warp 32, of 512), `sync` waits for the
generation it arrived in, `arrive` does not wait.  Over random interleavings
and 0..6 tiles a block, the protocol must never over-arrive on a barrier,
never deadlock, and leave every barrier idle at the end."""
import random

import pytest

COUNT = 512


def simulate(n_tiles, seed, per_parity=True):
    rnd = random.Random(seed)
    bars = {}  # id -> [arrived in the current generation, generation]

    def arrive(bid, n):
        c, gen = bars.setdefault(bid, [0, 0])
        c += n
        assert c <= COUNT, f"over-arrival on {bid}"
        bars[bid] = [0, gen + 1] if c == COUNT else [c, gen]
        return gen

    valid = [True] * n_tiles

    def compute():  # the compute warps, as one actor
        i = 0
        while True:
            b = i & 1 if per_parity else 0
            yield ("arrive", f"tile{b}", 480)        # tile i counted (or no tile)
            if i > 0:
                yield ("sync", f"base{(b ^ 1) if per_parity else 0}", 480)  # tile i - 1's base, then its offsets
            if not (i < n_tiles and valid[i]):
                return
            i += 1

    def look_back():
        i = 0
        while True:
            b = i & 1 if per_parity else 0
            yield ("sync", f"tile{b}", 32)
            if not (i < n_tiles and valid[i]):
                return
            yield ("arrive", f"base{b}", 32)         # after the look-back
            i += 1

    actors = {"compute": compute(), "look_back": look_back()}
    op = {a: next(g) for a, g in actors.items()}
    waiting, done = {}, set()
    for _ in range(100000):
        if len(done) == len(actors):
            break
        runnable = [a for a in actors if a not in done and
                    (a not in waiting or bars[waiting[a][0]][1] > waiting[a][1])]
        assert runnable, f"deadlock: {waiting}"
        a = rnd.choice(runnable)
        if a in waiting:
            del waiting[a]
        else:
            kind, bid, n = op[a]
            gen = arrive(bid, n)
            if kind == "sync" and bars[bid][1] == gen:
                waiting[a] = (bid, gen)
                continue
        try:
            op[a] = next(actors[a])
        except StopIteration:
            done.add(a)
    assert len(done) == len(actors)
    assert all(c == 0 for c, _ in bars.values()), bars


@pytest.mark.parametrize("n_tiles", range(7))
def test_handoffs_never_deadlock_or_over_arrive(n_tiles):
    for seed in range(200):
        simulate(n_tiles, seed)


def test_model_catches_one_barrier_per_side():
    """With one tile barrier and one base barrier instead of one per parity,
    some interleaving over-arrives (the look-back warp can arrive for tile
    i + 1 on the base barrier before the compute warps have waited for tile
    i), so the model does distinguish the two designs."""
    failures = 0
    for seed in range(200):
        try:
            simulate(4, seed, per_parity=False)
        except AssertionError:
            failures += 1
    assert failures > 0
