"""Host-side check of the site-coordinate arithmetic of the gradient kernel
(lgf_common.cuh, site_coords_r): the quotient s / L is taken as the high 32
bits of s * ceil(2^32 / L).  That is exact for 0 <= s < 2^32 / L, so for every
site index of every lattice the library accepts (extents in [2, 64], products
of 2, 3 and 5, V <= 64^4 = 2^24).  Checked here for all such extents over the
whole index range, in exact integer arithmetic."""
import numpy as np

EXTENTS = [n for n in range(2, 65) if all(p in (2, 3, 5) for p in
                                          [q for q in range(2, n + 1) if n % q == 0 and
                                           all(q % r for r in range(2, q))])]


def rcp(L):
    return 0xFFFFFFFF // L + 1  # geom_init_rcp


def test_extent_list():
    assert EXTENTS[:8] == [2, 3, 4, 5, 6, 8, 9, 10] and EXTENTS[-1] == 64 and 7 not in EXTENTS


def test_multiply_high_quotient_is_exact_for_every_site_index():
    s = np.arange(64 ** 4, dtype=np.uint64)
    for L in EXTENTS:
        q = (s * np.uint64(rcp(L))) >> np.uint64(32)
        assert np.array_equal(q, s // np.uint64(L)), L


def test_coordinates_of_a_mixed_lattice():
    dims = (48, 20, 12, 30)
    V = int(np.prod(dims))
    s = np.arange(V, dtype=np.uint64)
    m = [np.uint64(rcp(L)) for L in dims[:3]]
    q0 = (s * m[0]) >> np.uint64(32)
    q1 = (q0 * m[1]) >> np.uint64(32)
    q2 = (q1 * m[2]) >> np.uint64(32)
    c = [s - q0 * np.uint64(dims[0]), q0 - q1 * np.uint64(dims[1]), q1 - q2 * np.uint64(dims[2]), q2]
    ref = np.unravel_index(np.arange(V), dims[::-1])[::-1]
    for a in range(4):
        assert np.array_equal(c[a].astype(np.int64), ref[a])
