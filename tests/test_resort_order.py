"""Host-side fact behind the local re-sort's run order (mppic_resort.cuh, k_rs_offsets).

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
