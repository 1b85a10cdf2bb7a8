"""Domain decomposition geometry and coarse numbering (Sec. 2.1, Fig. 1; MRCM-OS step 1).

Integer work, compared bit-exactly with the CUDA library's host planner.

* Omega_s: box of ``sub`` cells per axis; s = I + m0 (J + m1 K) with m_a = ceil(n_a / sub_a).
  When sub_a does not divide n_a the last subdomain along axis a takes the remainder
  n_a - (m_a - 1) sub_a (a reading: the paper's grids are divisible).
* hat-Omega_s (oversampled region): Omega_s grown by l cells per side, clipped to the domain.
* Sides in the order -x, +x, -y, +y, -z, +z; a side is a Robin side (part of Gamma_s) iff it is
  not on the domain boundary.  N_s = number of Robin sides.  Because l is below the size of every
  subdomain along every axis that has interfaces, the Robin sides of hat-Omega_s are exactly
  those of Omega_s.
* Coarse unknowns c_{s,k}: index off_s + rank of side k among the Robin sides of s, where off_s is
  the exclusive prefix sum of N_s.
* Interfaces Gamma_{s,s'}: x-normal first, ordered by the lower subdomain index (K, J, I
  lexicographic, I fastest), then y-normal, then z-normal.  Interface e owns the coarse rows 2e
  (flux continuity, Eq. 13) and 2e+1 (pressure continuity, Eq. 14).
* Faces of a side are listed with the faster in-plane axis first (x before y before z).
* A face is identified by its flat index in the face array of its axis plus an axis offset:
  x-faces first, then y-faces, then z-faces.

Pinned by brute-force invariants (every cell in exactly one subdomain, 2E = sum N_s, the Gamma
faces are exactly the faces whose two cells lie in different subdomains) in
tests/test_oracle_partition.py.
"""

import numpy as np


class Partition:
    def __init__(self, dim, n, sub, l):
        n = [int(v) for v in n]
        sub = [int(v) for v in sub]
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        if dim == 2 and (n[2] != 1 or sub[2] != 1):
            raise ValueError("2-D problems have n[2] == sub[2] == 1")
        if any(sub[a] < 1 or n[a] < 1 for a in range(3)):
            raise ValueError("grid and subdomain sizes must be positive")
        m = [-(-n[a] // sub[a]) for a in range(3)]
        last = [n[a] - (m[a] - 1) * sub[a] for a in range(3)]
        if l < 0 or any(l >= sub[a] or (m[a] > 1 and l >= last[a]) for a in range(dim)):
            raise ValueError("oversampling must satisfy 0 <= l < the size of every subdomain")
        self.dim, self.n, self.sub, self.l = dim, n, sub, int(l)
        self.m = m
        S = m[0] * m[1] * m[2]
        self.S = S
        self.box = np.zeros((S, 2, 3), dtype=np.int64)
        self.obox = np.zeros((S, 2, 3), dtype=np.int64)
        self.robin = np.zeros((S, 6), dtype=bool)
        self.coord = np.zeros((S, 3), dtype=np.int64)
        for s in range(S):
            idx = (s % m[0], (s // m[0]) % m[1], s // (m[0] * m[1]))
            self.coord[s] = idx
            for a in range(3):
                lo = idx[a] * sub[a]
                hi = min(lo + sub[a], n[a])
                self.box[s, 0, a], self.box[s, 1, a] = lo, hi
                if a < dim:
                    self.obox[s, 0, a] = max(lo - l, 0)
                    self.obox[s, 1, a] = min(hi + l, n[a])
                    self.robin[s, 2 * a] = idx[a] > 0
                    self.robin[s, 2 * a + 1] = idx[a] < m[a] - 1
                else:
                    self.obox[s, 0, a], self.obox[s, 1, a] = lo, hi
        self.N = self.robin.sum(axis=1).astype(np.int64)
        self.off = np.concatenate([[0], np.cumsum(self.N)[:-1]]).astype(np.int64)
        self.E2 = int(self.N.sum())
        # rank of each Robin side among the Robin sides of its subdomain (-1 if not Robin)
        self.rank = -np.ones((S, 6), dtype=np.int64)
        for s in range(S):
            r = 0
            for side in range(6):
                if self.robin[s, side]:
                    self.rank[s, side] = r
                    r += 1
        strides = (1, m[0], m[0] * m[1])
        inter = []
        for a in range(dim):
            for s in range(S):  # s ascending is (K, J, I) lexicographic with I fastest
                if self.coord[s, a] < m[a] - 1:
                    inter.append((a, s, s + strides[a]))
        self.interfaces = np.array(inter, dtype=np.int64).reshape(-1, 3)
        assert 2 * len(inter) == self.E2
        fshape = []
        for a in range(3):
            fs = list(n)
            fs[a] += 1
            fshape.append(fs)  # (x extent, y extent, z extent) of the face array of axis a
        self.face_extent = fshape
        sizes = [fs[0] * fs[1] * fs[2] for fs in fshape]
        self.face_offset = (0, sizes[0], sizes[0] + sizes[1])

    # ------------------------------------------------------------------ faces of a box side
    def side_faces(self, lo, hi, side):
        """Faces of the box [lo, hi) on ``side``: list of (face position (x,y,z), inside cell,
        outside cell) with the faster in-plane axis first.  Cells are (x, y, z) triples; the
        outside cell may lie outside the domain."""
        a, d = side // 2, side % 2
        others = [b for b in range(3) if b != a]
        b1, b2 = others[0], others[1]
        plane = lo[a] if d == 0 else hi[a]
        out = []
        for t2 in range(lo[b2], hi[b2]):
            for t1 in range(lo[b1], hi[b1]):
                pos = [0, 0, 0]
                pos[a], pos[b1], pos[b2] = plane, t1, t2
                inside = list(pos)
                outside = list(pos)
                if d == 0:
                    outside[a] = plane - 1
                else:
                    inside[a] = plane - 1
                out.append((tuple(pos), tuple(inside), tuple(outside)))
        return out

    def face_id(self, a, pos):
        ex = self.face_extent[a]
        return self.face_offset[a] + pos[0] + ex[0] * (pos[1] + ex[1] * pos[2])

    def gamma_faces(self, s, side):
        """Faces of Gamma_s on a Robin side of Omega_s (see ``side_faces``)."""
        return self.side_faces(self.box[s, 0], self.box[s, 1], side)

    # ------------------------------------------------------------------ canonical export
    def export(self):
        """Flat int32 array: header, per-subdomain records, interfaces, Gamma face ids.

        header: dim, n0, n1, n2, sub0, sub1, sub2, l, S, 2E, E
        per s : box lo(3) hi(3), obox lo(3) hi(3), Robin side mask (bit k = side k), N_s, off_s
        per e : axis, s (lower), s' (upper)
        per s, per Robin side in side order: face count, face ids
        """
        out = [self.dim, *self.n, *self.sub, self.l, self.S, self.E2, len(self.interfaces)]
        for s in range(self.S):
            mask = sum(1 << k for k in range(6) if self.robin[s, k])
            out += [*self.box[s, 0], *self.box[s, 1], *self.obox[s, 0], *self.obox[s, 1],
                    mask, int(self.N[s]), int(self.off[s])]
        for e in self.interfaces:
            out += [int(e[0]), int(e[1]), int(e[2])]
        for s in range(self.S):
            for side in range(6):
                if self.robin[s, side]:
                    faces = self.gamma_faces(s, side)
                    out.append(len(faces))
                    out += [self.face_id(side // 2, f[0]) for f in faces]
        return np.array(out, dtype=np.int32)
