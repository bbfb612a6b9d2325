"""Host model of how the persistent kernel hands out the queue entries of a wide
BFS level (guided self-scheduling in step_expand, csrc/bm_device.cuh): every
entry must be expanded exactly once, whatever order the blocks' counter
atomics land in.  The model restates the kernel's integer arithmetic; the GPU
parity tests check the kernel itself."""
import random

import pytest


def _clamp_w(w, T):
    return min(T, max(32, (w + 31) & ~31))


def _guided_cover(q, G, T, seed):
    rnd = random.Random(seed)
    w0 = _clamp_w((q + 2 * G - 1) // (2 * G), T)
    base = G * w0
    ctr = 0
    seen = [0] * q
    state = [[min(b * w0, q), w0] for b in range(G)]
    active = [b for b in range(G) if state[b][0] < q]
    while active:
        b = rnd.choice(active)  # any block may issue its next atomic first
        first, width = state[b]
        grab = _clamp_w((q - first - width) // (2 * G), T)
        nxt = base + ctr        # atomicAdd(counter, grab), prefetched by tile_load
        ctr += grab
        for i in range(first, min(first + width, q)):  # tile_load keeps i < q
            seen[i] += 1
        state[b] = [nxt, grab]
        if nxt >= q:
            active.remove(b)
    return seen


@pytest.mark.parametrize("seed", range(40))
def test_guided_ranges_cover_every_entry_once(seed):
    r = random.Random(seed)
    G = r.choice([1, 2, 3, 7, 16, 40])
    T = r.choice([32, 64, 128, 512])
    q = r.randint(G * T + 1, G * T * 6)  # the guided path serves levels wider than G x T
    assert all(v == 1 for v in _guided_cover(q, G, T, seed))


def test_guided_ranges_at_the_rmat21_level_sizes():
    # 304 blocks of 512 threads, the level sizes of an rmat21 run
    for q in (155_649, 214_141, 477_862, 530_483):
        assert all(v == 1 for v in _guided_cover(q, 304, 512, q))
