"""CPU model of the index arithmetic of the row-tiled batched one-sided SVD
kernel (k_batched_svd_tiled: the Gram from 4 x 4 blocks of staged 64-row
tiles, svd_rotate_rows with its column permutation, and the finalisation:
column norms, their descending rank, U = G Sigma^+), with the threads of a CTA
run one after another between its barriers.  Every access goes to a flat
buffer of exactly the size the kernel allocates (the caller's minimal G
buffer ld * (n - 1) + m, the tile kSvdTileLd x kq, V-hat and the accumulated
V kq x kq with leading dimension k) and is bounds-checked; each output must
be written exactly once and equal the product it stands for.  This is the
check of a kernel's grid and indexes against its buffers that precedes its
first run on a GPU; the arithmetic is modelled in FP64."""
from __future__ import annotations

import math

import numpy as np
import pytest

TR, TRS = 64, 65   # kSvdTileRows, kSvdTileLd
CT = 8             # columns per thread in svd_rotate_rows


def tri(i):
    return i * (i + 1) // 2


def tri_pad(k):
    return (k * (k + 1) // 2 + 1) & ~1


class Buf:
    """A flat buffer whose every read and write is bounds-checked."""

    def __init__(self, n, name):
        self.a = np.full(n, np.nan)
        self.name = name

    def __getitem__(self, i):
        assert 0 <= i < len(self.a), (self.name, i, len(self.a))
        return self.a[i]

    def __setitem__(self, i, v):
        assert 0 <= i < len(self.a), (self.name, i, len(self.a))
        self.a[i] = v


def gram(G, ldg, m, n, k, kq, nt):
    """The kernel's Gram pass: packed lower triangle of G^T G into Ap."""
    Ap = Buf(tri_pad(kq), "Ap")
    tile = Buf(TRS * kq, "tile")
    for idx in range(tri_pad(k)):
        Ap[idx] = 0.0
    nb4 = (n + 3) >> 2
    nbl = nb4 * (nb4 + 1) // 2
    for b0 in range(0, nbl, nt):
        owners, accs = {}, {}
        for tid in range(nt):
            bl = b0 + tid
            if bl < nbl:
                bi = int((math.sqrt(8.0 * bl + 1.0) - 1.0) * 0.5)
                while tri(bi + 1) <= bl:
                    bi += 1
                while tri(bi) > bl:
                    bi -= 1
                owners[tid] = (bi, bl - tri(bi))
                accs[tid] = np.zeros((4, 4))
        for r0 in range(0, m, TR):
            tr = min(TR, m - r0)
            for idx in range(tr * 4 * nb4):           # staging (all threads)
                rr, c = idx % tr, idx // tr
                tile[c * TRS + rr] = G[(r0 + rr) + ldg * c] if c < n else 0.0
            for tid, (bi, bj) in owners.items():       # accumulation
                for r in range(tr):
                    ai = [tile[(4 * bi + x) * TRS + r] for x in range(4)]
                    aj = [tile[(4 * bj + x) * TRS + r] for x in range(4)]
                    for x in range(4):
                        for y in range(4):
                            accs[tid][x, y] += ai[x] * aj[y]
        for tid, (bi, bj) in owners.items():
            for x in range(4):
                for y in range(4):
                    i, j = 4 * bi + x, 4 * bj + y
                    if i < n and j <= i:
                        Ap[tri(i) + j] = accs[tid][x, y]
    return Ap


def rotate(X, ldx, rows, n, k, Vh, dest, kq, nt):
    """svd_rotate_rows: X(:, dest[j]) <- (X Vh)(:, j) over staged row tiles."""
    tile = Buf(TRS * kq, "tile")
    nw = nt // 32
    for r0 in range(0, rows, TR):
        tr = min(TR, rows - r0)
        for idx in range(tr * n):
            rr, c = idx % tr, idx // tr
            tile[c * TRS + rr] = X[(r0 + rr) + ldx * c]
        writes = []
        for jc in range(0, n, nw * CT):
            for tid in range(nt):
                lane, w = tid & 31, tid >> 5
                acc0, acc1 = [0.0] * CT, [0.0] * CT
                for l in range(n):
                    a0 = tile[l * TRS + lane] if lane < tr else 0.0
                    a1 = tile[l * TRS + lane + 32] if lane + 32 < tr else 0.0
                    for y in range(CT):
                        j = jc + w + nw * y
                        b = Vh[l + k * j] if j < n else 0.0
                        acc0[y] += a0 * b
                        acc1[y] += a1 * b
                for y in range(CT):
                    j = jc + w + nw * y
                    if j >= n:
                        continue
                    col = ldx * dest[j]
                    if lane < tr:
                        writes.append(((r0 + lane) + col, acc0[y]))
                    if lane + 32 < tr:
                        writes.append(((r0 + lane + 32) + col, acc1[y]))
        seen = set()
        for i, v in writes:                            # after the tile's barrier
            assert i not in seen, "an output written twice"
            seen.add(i)
            X[i] = v


def finalize(G, ldg, m, n, kq, nt):
    """The kernel's finalisation: column norms over staged tiles (one FMA
    chain per column in row order), the descending stable rank, and
    G(:, dest[j]) <- G(:, j) / norm_j over staged tiles."""
    tile = Buf(TRS * kq, "tile")
    nrm = Buf(tri_pad(kq), "nrm")          # the packed-Gram area, reused
    for j in range(n):
        nrm[j] = 0.0
    for r0 in range(0, m, TR):
        tr = min(TR, m - r0)
        for idx in range(tr * n):
            rr, c = idx % tr, idx // tr
            tile[c * TRS + rr] = G[(r0 + rr) + ldg * c]
        for j in range(n):
            acc = nrm[j]
            for rr in range(tr):
                acc += tile[j * TRS + rr] * tile[j * TRS + rr]
            nrm[j] = acc
    norms = [math.sqrt(nrm[j]) for j in range(n)]
    dest = [sum(1 for y in range(n) if norms[y] > norms[x] or (norms[y] == norms[x] and y < x))
            for x in range(n)]
    for r0 in range(0, m, TR):
        tr = min(TR, m - r0)
        for idx in range(tr * n):
            rr, c = idx % tr, idx // tr
            tile[c * TRS + rr] = G[(r0 + rr) + ldg * c]
        for idx in range(tr * n):
            rr, j = idx % tr, idx // tr
            G[(r0 + rr) + ldg * dest[j]] = tile[j * TRS + rr] / norms[j] if norms[j] > 0 else 0.0
    return norms, dest


def _check(m, n, ldg_pad, nt, seed):
    rng = np.random.default_rng(seed)
    k = n + (n & 1)
    kq = (k + 3) // 4 * 4          # a batch of one size: kmax = k
    ldg = m + ldg_pad
    Gm = rng.standard_normal((m, n))
    G = Buf(ldg * (n - 1) + m, "G")
    for c in range(n):
        for r in range(m):
            G[r + ldg * c] = Gm[r, c]
    Ap = gram(G, ldg, m, n, k, kq, nt)
    C = Gm.T @ Gm
    for i in range(k):
        for j in range(i + 1):
            want = C[i, j] if i < n else 0.0
            assert abs(Ap[tri(i) + j] - want) <= 1e-9 * (1 + abs(want)), (i, j)
    # G <- G V P with a random orthogonal V and a random permutation
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Vh = Buf(kq * kq, "Vh")
    for idx in range(kq * kq):
        Vh[idx] = 0.0
    for l in range(n):
        for j in range(n):
            Vh[l + k * j] = V[l, j]
    dest = list(rng.permutation(n)) + list(range(n, k))
    rotate(G, ldg, m, n, k, Vh, dest, kq, nt)
    R = Gm @ V
    for j in range(n):
        for r in range(m):
            assert abs(G[r + ldg * dest[j]] - R[r, j]) <= 1e-9, (r, j)
    # the accumulated V in shared memory: n rows, leading dimension k
    Vacc = Buf(kq * kq, "Vacc")
    for idx in range(kq * kq):
        Vacc[idx] = 0.0
    for i in range(k):
        Vacc[i + k * i] = 1.0
    rotate(Vacc, k, n, n, k, Vh, dest, kq, nt)
    for j in range(n):
        for i in range(n):
            assert abs(Vacc[i + k * dest[j]] - V[i, j]) <= 1e-12
    # finalisation of the rotated G: sigma = column norms, U = G Sigma^+ sorted
    R = np.array([[G[r + ldg * c] for c in range(n)] for r in range(m)])
    norms, dest2 = finalize(G, ldg, m, n, kq, nt)
    want = np.linalg.norm(R, axis=0)
    assert np.allclose(norms, want, rtol=1e-12, atol=0)
    assert sorted(dest2) == list(range(n))
    order = np.argsort(-want, kind="stable")
    for pos, j in enumerate(order):
        assert dest2[j] == pos
        for r in range(m):
            assert abs(G[r + ldg * pos] - R[r, j] / want[j]) <= 1e-12


@pytest.mark.parametrize("m,n,ldg_pad,nt,seed", [
    (70, 9, 0, 128, 1),      # two row tiles, the second ragged
    (64, 64, 3, 256, 2),     # the 1024 x 64 workload's column count, padded ld
    (130, 13, 1, 128, 3),    # odd n: a padding column in the Gram
    (5, 5, 0, 32, 4),        # one warp, one short tile
    (200, 37, 2, 64, 5),     # several column chunks per warp
    (33, 1, 0, 128, 6),      # a single column
    (65, 66, 0, 64, 7),      # n > tile rows: the accumulated V spans two row tiles
    (100, 64, 0, 512, 8),    # the autotuner's largest CTA: 16 warps, one column chunk
])
def test_tiled_svd_indexing(m, n, ldg_pad, nt, seed):
    _check(m, n, ldg_pad, nt, seed)
