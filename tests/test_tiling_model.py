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


# ---------------------------------------------------------------- warp levels
# Host model of warp_expand_sb's edge ownership (csrc/bm_device.cuh): a warp's
# 32 queue columns with degrees deg[] (0 for a column whose root is served, or
# that was set aside for the whole block), an inclusive shuffle scan, the
# columns with edges compacted by rank, and for each 32-edge chunk the OR of
# the columns' start bits; edge j belongs to the last column starting at or
# before it.  Every edge of every kept column must be visited exactly once, at
# its own row_idx position.
HUB_DEG, HUB_MAX = 256, 16


def _warp_visits(beg, deg, ilp=4):
    assert len(beg) == len(deg) == 32
    incl, run = [], 0
    for d in deg:
        run += d
        incl.append(run)
    total = incl[31]
    start = [incl[i] - deg[i] for i in range(32)]
    s_base, s_col = {}, {}
    rank = 0
    for i in range(32):  # __popc(ballot(deg > 0) & lanes below i)
        if deg[i] > 0:
            s_base[rank] = beg[i] - start[i]
            s_col[rank] = i
            rank += 1
    visits = []
    before = 0
    for j0 in range(0, total, 32 * ilp):
        for u in range(ilp):
            J0 = j0 + 32 * u
            starts = 0
            for i in range(32):
                if deg[i] > 0 and J0 <= start[i] < J0 + 32:
                    starts |= 1 << (start[i] - J0)
            for lane in range(32):
                j = J0 + lane
                if j < total:
                    k = before + bin(starts & (0xFFFFFFFF >> (31 - lane))).count("1") - 1
                    visits.append((s_col[k], s_base[k] + j))
            before += bin(starts).count("1")
    return visits


@pytest.mark.parametrize("seed", range(60))
def test_warp_edge_owners_cover_every_edge_once(seed):
    r = random.Random(seed)
    hi = r.choice([1, 3, 8, 40, 300])
    deg = [0 if r.random() < r.choice([0.0, 0.2, 0.7]) else r.randint(1, hi) for _ in range(32)]
    beg, pos = [], 0
    for d in deg:  # each column's rows at a distinct place of row_idx
        pos += r.randint(0, 5)
        beg.append(pos)
        pos += d
    seen = {}
    for col, at in _warp_visits(beg, deg, ilp=r.choice([1, 4])):
        assert beg[col] <= at < beg[col] + deg[col]  # inside the owner's own rows
        seen[at] = seen.get(at, 0) + 1
    want = {beg[i] + k for i in range(32) for k in range(deg[i])}
    assert set(seen) == want and all(v == 1 for v in seen.values())


def test_warp_edge_owners_special_groups():
    for deg in ([0] * 32, [1] * 32, [0] * 31 + [7], [5] + [0] * 31, [32] * 32, [33, 0] * 16):
        beg = [1000 * i for i in range(32)]
        got = sorted(at for _, at in _warp_visits(beg, deg))
        assert got == sorted(beg[i] + k for i in range(32) for k in range(deg[i]))


@pytest.mark.parametrize("seed", range(20))
def test_hub_columns_set_aside_or_kept(seed):
    # Columns of more than HUB_DEG edges are set aside by whichever warp meets
    # them, up to HUB_MAX a level (a shared counter, warps in any order); the
    # rest stay with their warp.  Either way each is expanded exactly once.
    r = random.Random(seed)
    degs = [r.choice([1, 2, 5, HUB_DEG, HUB_DEG + 1, 1000]) for _ in range(32 * r.randint(1, 6))]
    groups = [list(range(g, min(g + 32, len(degs)))) for g in range(0, len(degs), 32)]
    r.shuffle(groups)
    nhub, aside, by_warp = 0, [], []
    for grp in groups:
        for c in grp:
            if degs[c] > HUB_DEG:
                h, nhub = nhub, nhub + 1
                if h < HUB_MAX:
                    aside.append(c)
                    continue
            by_warp.append(c)
    assert len(aside) == min(HUB_MAX, sum(d > HUB_DEG for d in degs))
    assert sorted(aside + by_warp) == list(range(len(degs)))
