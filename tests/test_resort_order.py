"""Host-side facts behind the local re-sort (mppic_resort.cuh): its run order (k_rs_offsets),
and a host model of its five steps, which must give the stable sort by key for any input
order.

Destination brick B receives a run of parcels from each neighbour b = B - d, d in
{-1,0,1}^3, slot (dx+1) + 3 (dy+1) + 9 (dz+1). The bucket is in source order only if the
runs are laid out in ascending source index; the kernel takes them in descending slot order.
That is the same order for every brick of every grid of bricks: brute force over small grids,
including the degenerate ones (one or two bricks along an axis), where some neighbours
do not exist.
"""
import itertools


def _sources(nbx, nby, nbz, bx, by, bz):
    """(slot, source index) of every neighbour of brick (bx, by, bz) inside the grid."""
    out = []
    for s in range(27):
        dx, dy, dz = s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1
        sx, sy, sz = bx - dx, by - dy, bz - dz
        if 0 <= sx < nbx and 0 <= sy < nby and 0 <= sz < nbz:
            out.append((s, sx + nbx * (sy + nby * sz)))
    return out


def test_descending_slot_is_ascending_source_index():
    for nbx, nby, nbz in itertools.product(range(1, 6), repeat=3):
        for bx, by, bz in itertools.product(range(nbx), range(nby), range(nbz)):
            src = _sources(nbx, nby, nbz, bx, by, bz)
            by_slot = [b for _, b in sorted(src, key=lambda t: -t[0])]
            assert by_slot == sorted(by_slot), (nbx, nby, nbz, bx, by, bz)
            assert len(set(by_slot)) == len(by_slot)


def test_slot_of_destination_inverts_source_of_slot():
    """The hist pass files a parcel of source b going to B under slot(B - b); the count pass
    reads slot s of B from source B - d(s): the same pair."""
    for nbx, nby, nbz in ((3, 2, 4), (1, 5, 2), (4, 4, 1)):
        for bx, by, bz in itertools.product(range(nbx), range(nby), range(nbz)):
            for s, b in _sources(nbx, nby, nbz, bx, by, bz):
                sx, sy, sz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
                d = (bx - sx, by - sy, bz - sz)
                assert (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1) == s


def _local_resort_model(key, ranges, nb):
    """The local re-sort's steps on the host: key[q] = brick * 256 + cell of the parcel at
    position q; ranges[b] = (s0, s1) of brick b in the current order (a partition of the
    positions); nb = (nbx, nby, nbz). Returns the new order (source positions)."""
    nbx, nby, nbz = nb
    nbricks = nbx * nby * nbz

    def coords(b):
        return b % nbx, (b // nbx) % nby, b // (nbx * nby)

    def slot(b, B):
        (x, y, z), (X, Y, Z) = coords(b), coords(B)
        d = (X - x, Y - y, Z - z)
        if max(abs(t) for t in d) > 1:
            return -1
        return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1)

    # hist: per source brick and slot; far parcels per destination
    cnt = [[0] * 27 for _ in range(nbricks)]
    far = [0] * nbricks
    for b, (s0, s1) in enumerate(ranges):
        for q in range(s0, s1):
            B = key[q] // 256
            s = slot(b, B)
            if s >= 0:
                cnt[b][s] += 1
            else:
                far[B] += 1
    # count and offsets: runs in descending slot order, far parcels after the runs
    start, run_off, far_next = [0] * nbricks, {}, [0] * nbricks
    total = 0
    for B in range(nbricks):
        start[B] = total
        X, Y, Z = coords(B)
        r = total
        for s in range(26, -1, -1):
            sx, sy, sz = X - (s % 3 - 1), Y - ((s // 3) % 3 - 1), Z - (s // 9 - 1)
            if 0 <= sx < nbx and 0 <= sy < nby and 0 <= sz < nbz:
                b = sx + nbx * (sy + nby * sz)
                run_off[(b, s)] = r
                r += cnt[b][s]
        far_next[B] = r
        total = r + far[B]
    # scatter: each run in source order; far parcels in any order (here: reversed)
    bucket = [None] * len(key)
    far_items = []
    for b, (s0, s1) in enumerate(ranges):
        for q in range(s0, s1):
            B = key[q] // 256
            s = slot(b, B)
            if s >= 0:
                bucket[run_off[(b, s)]] = q
                run_off[(b, s)] += 1
            else:
                far_items.append((B, q))
    for B, q in reversed(far_items):
        bucket[far_next[B]] = q
        far_next[B] += 1
    # build: a bucket with far parcels is sorted by source index; then stable by cell
    out = []
    for B in range(nbricks):
        bk = bucket[start[B]:start[B] + sum(1 for q in range(len(key)) if key[q] // 256 == B)]
        if far[B]:
            bk = sorted(bk)
        bk = sorted(bk, key=lambda q: key[q] % 256)       # Python's sort is stable
        out.extend(bk)
    return out


def test_local_resort_model_is_the_stable_sort():
    """Runs in descending slot order, far parcels re-sorted by source index, then a stable
    pass by cell: the stable sort of the current order by key, for parcels near and far and
    for an order unrelated to the ranges."""
    import numpy as np
    rng = np.random.default_rng(7)
    for nb in ((3, 2, 2), (1, 4, 3), (2, 2, 1)):
        nbricks = nb[0] * nb[1] * nb[2]
        for mode in ("near", "far", "shuffled"):
            n = 600
            # a previous layout: keys sorted by brick, ranges from it
            old = np.sort(rng.integers(0, nbricks * 256, n))
            ranges, pos = [], 0
            for b in range(nbricks):
                c = int(np.sum(old // 256 == b))
                ranges.append((pos, pos + c))
                pos += c
            # new keys: mostly the same brick or a neighbour, some anywhere
            key = old.copy()
            move = rng.random(n) < 0.3
            for q in np.nonzero(move)[0]:
                b = key[q] // 256
                x, y, z = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
                x = min(max(x + rng.integers(-1, 2), 0), nb[0] - 1)
                y = min(max(y + rng.integers(-1, 2), 0), nb[1] - 1)
                z = min(max(z + rng.integers(-1, 2), 0), nb[2] - 1)
                key[q] = (x + nb[0] * (y + nb[1] * z)) * 256 + rng.integers(0, 256)
            if mode == "far":
                far = rng.random(n) < 0.1
                key[far] = rng.integers(0, nbricks * 256, int(far.sum()))
            if mode == "shuffled":
                key = rng.permutation(key)
            got = _local_resort_model([int(k) for k in key], ranges, nb)
            want = list(np.argsort(key, kind="stable"))
            assert got == want, (nb, mode)
