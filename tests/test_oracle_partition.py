"""Brute-force pins of the oracle's partition and coarse numbering (Sec. 2.1, Fig. 1)."""

import itertools

import numpy as np
import pytest

from oracle.partition import Partition

CASES = [
    (2, (12, 8, 1), (4, 4, 1), 0),
    (2, (12, 8, 1), (4, 2, 1), 1),
    (2, (64, 64, 1), (16, 16, 1), 2),
    (2, (40, 24, 1), (8, 12, 1), 7),
    (3, (8, 6, 4), (4, 3, 2), 1),
    (3, (12, 12, 8), (4, 4, 4), 3),
    # grids the subdomain size does not divide: the last subdomain along an axis is shorter
    (2, (13, 9, 1), (4, 4, 1), 0),
    (2, (14, 11, 1), (4, 3, 1), 1),
    (2, (30, 7, 1), (8, 16, 1), 5),
    (3, (10, 8, 6), (4, 3, 4), 1),
]


@pytest.mark.parametrize("dim,n,sub,l", CASES)
def test_partition_invariants(dim, n, sub, l):
    P = Partition(dim, n, sub, l)
    owner = -np.ones((n[2], n[1], n[0]), dtype=np.int64)
    for s in range(P.S):
        lo, hi = P.box[s, 0], P.box[s, 1]
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        assert (owner[sl] == -1).all()
        owner[sl] = s
        # full size, except the last subdomain along an axis, which ends on the grid boundary
        for a in range(3):
            assert lo[a] == P.coord[s, a] * sub[a]
            assert hi[a] - lo[a] == (sub[a] if lo[a] + sub[a] <= n[a] else n[a] - lo[a])
            assert a >= dim or P.m[a] == 1 or hi[a] - lo[a] > l
            assert (hi[a] == n[a]) == (P.coord[s, a] == P.m[a] - 1)
        olo, ohi = P.obox[s, 0], P.obox[s, 1]
        for a in range(3):
            assert 0 <= olo[a] <= lo[a] and hi[a] <= ohi[a] <= n[a]
            if a < dim:
                assert olo[a] == max(lo[a] - l, 0) and ohi[a] == min(hi[a] + l, n[a])
            # Robin side iff not on the domain boundary
            if a < dim:
                assert P.robin[s, 2 * a] == (lo[a] > 0)
                assert P.robin[s, 2 * a + 1] == (hi[a] < n[a])
            else:
                assert not P.robin[s, 2 * a] and not P.robin[s, 2 * a + 1]
    assert (owner >= 0).all()
    assert P.E2 == int(P.N.sum()) == 2 * len(P.interfaces)
    assert (P.off == np.concatenate([[0], np.cumsum(P.N)[:-1]])).all()
    # interface faces: every face whose two cells have different owners, seen once from each side
    seen = {}
    for s in range(P.S):
        for side in range(6):
            if P.robin[s, side]:
                for (pos, inside, outside) in P.gamma_faces(s, side):
                    assert owner[inside[2], inside[1], inside[0]] == s
                    assert owner[outside[2], outside[1], outside[0]] != s
                    fid = P.face_id(side // 2, pos)
                    seen[fid] = seen.get(fid, 0) + 1
    brute = set()
    for a in range(dim):
        for k, j, i in itertools.product(range(n[2]), range(n[1]), range(n[0])):
            c = [i, j, k]
            if c[a] == 0:
                continue
            c2 = list(c)
            c2[a] -= 1
            if owner[c[2], c[1], c[0]] != owner[c2[2], c2[1], c2[0]]:
                brute.add(P.face_id(a, c))
    assert set(seen) == brute and all(v == 2 for v in seen.values())
    # interfaces: lower / upper neighbours along the axis, x-normal first, ascending lower index
    for (a, s, s2) in P.interfaces:
        assert (P.coord[s2] - P.coord[s] == np.eye(3, dtype=np.int64)[a]).all()
    keys = [(int(a), int(s)) for (a, s, _s2) in P.interfaces]
    assert keys == sorted(keys)


def test_face_order_and_export_header():
    P = Partition(2, (8, 8, 1), (4, 4, 1), 1)
    faces = P.gamma_faces(0, 1)  # +x side of subdomain 0: x-faces at x = 4, y = 0..3
    assert [f[0] for f in faces] == [(4, y, 0) for y in range(4)]
    faces = P.gamma_faces(0, 3)  # +y side: y-faces at y = 4, x = 0..3
    assert [f[0] for f in faces] == [(x, 4, 0) for x in range(4)]
    ex = P.export()
    assert ex.dtype == np.int32
    assert list(ex[:11]) == [2, 8, 8, 1, 4, 4, 1, 1, 4, 8, 4]
    # x-face ids: flat index in the (nx+1) x ny x nz array; y-faces follow after all x-faces
    assert P.face_id(0, (4, 2, 0)) == 4 + 9 * 2
    assert P.face_id(1, (3, 4, 0)) == 9 * 8 + 3 + 8 * 4


@pytest.mark.parametrize("bad", [((13, 8, 1), (4, 4, 1), 1), ((12, 8, 1), (4, 4, 1), 4), ((12, 8, 1), (4, 4, 1), -1),
                                 ((12, 8, 1), (0, 4, 1), 0), ((14, 8, 1), (5, 4, 1), 4)])
def test_invalid_partition_rejected(bad):
    n, sub, l = bad
    with pytest.raises(ValueError):
        Partition(2, n, sub, l)
