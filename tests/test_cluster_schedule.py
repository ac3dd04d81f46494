"""The cluster-resident V-cycle (csrc/cluster_mg.cuh, planned in csrc/precond.cuh), restated on the
host: its row partition and its communication schedule.

Partition.  At the finest level CTA r of C owns grid rows [r*n1 // C, (r+1)*n1 // C); at every
coarser level CTA r owns rows [lo // 2, hi // 2) where [lo, hi) is its range one level finer
(coarse row J sits at fine row 2J+1, 0-based).  Every level but the coarsest is distributed; the
coarsest is held whole by every CTA.  The plan is accepted only when every CTA owns at least one
row of every distributed level (neighbours store their edge rows only into non-empty CTAs, so a
CTA with an empty coarse range would interpolate from ghost rows nobody fills).

Schedule.  `cluster_vcycles` runs the kernel's steps CTA by CTA on a model of distributed shared
memory: per CTA and level three row blocks (x ping-pong and b) with a ghost row above and below;
a step that writes a CTA's first or last row also stores it into the neighbour's ghost row; steps
are separated by cluster barriers except where the kernel has only a block barrier (after the
restriction, between the fused interpolation and the first post-smoothing sweep, after the
gather of the coarsest solution).  Within each barrier interval a word written by one CTA and read
or written by another is a race.  Race-free, the model's CTA-by-CTA order gives the result any
interleaving gives, and that result must equal the oracle's V-cycles.  (Ordering among the threads
of one CTA is outside the model.)
"""
import itertools

import numpy as np
import pytest

import synth
from oracle.multigrid import Hierarchy, level_sizes
from oracle.operators import mass_fd, q1_matrices, stiffness_fd


def plan(ns, C):
    """Row ranges of the distributed levels, or None where the cluster path is not taken."""
    sizes = level_sizes(ns)
    T = len(sizes) - 1
    if len(ns) != 2 or T < 1 or sizes[0][1] < C:
        return sizes, None
    rlo = partition(sizes, C)
    if any(lo[r + 1] <= lo[r] for lo in rlo for r in range(C)):
        return sizes, None
    return sizes, rlo


def partition(sizes, C):
    rlo = []
    for l in range(len(sizes) - 1):
        rlo.append([r * sizes[0][1] // C for r in range(C + 1)] if l == 0 else [v // 2 for v in rlo[l - 1]])
    return rlo


def interp_rows(F):
    """Coarse rows of 1D interpolation at fine row F (0-based; -1 / nc are boundary zeros)."""
    g = F + 1
    return [g // 2 - 1] if g % 2 == 0 else [(g - 1) // 2 - 1, (g + 1) // 2 - 1]


SHAPES = [(256, 256), (255, 257), (33, 17), (40, 36), (34, 37), (100, 97), (64, 20), (20, 64), (129, 97),
          (48, 40), (300, 31), (17, 300), (70, 66), (511, 33), (120, 17), (100, 12), (1000, 700)]


@pytest.mark.parametrize("ns,C", list(itertools.product(SHAPES, (8, 16))))
def test_cluster_partition_invariants(ns, C):
    sizes, rlo = plan(ns, C)
    if rlo is None:
        pytest.skip("the cluster path is not planned for this shape and cluster size")
    for l, lo in enumerate(rlo):
        n1 = sizes[l][1]
        assert lo[0] == 0 and lo[C] == n1 and all(lo[r] < lo[r + 1] for r in range(C))
        for r in range(C):
            a, b = lo[r], lo[r + 1]
            if l + 1 < len(rlo):
                ac, bc = rlo[l + 1][r], rlo[l + 1][r + 1]
                for J in range(ac, bc):
                    assert a <= 2 * J + 1 < b          # coarse row J belongs to the owner of fine row 2J+1
                    for fj in (2 * J, 2 * J + 1, 2 * J + 2):
                        if 0 <= fj < n1:
                            assert a - 1 <= fj <= b, (l, r, J, fj)
                for F in range(a - 1, b + 1):         # own rows and the two ghost rows
                    if 0 <= F < n1:
                        for Jc in interp_rows(F):
                            assert ac - 1 <= Jc <= bc, (l, r, F, Jc)


def test_cluster_plan_rejects_empty_ranges():
    """Short, wide grids leave some CTA without a row of a coarse distributed level at C = 16;
    such a plan is rejected (the next cluster size, or the level kernels, take the solve)."""
    assert plan((120, 17), 16)[1] is None and plan((120, 17), 8)[1] is not None
    assert plan((100, 12), 16)[1] is None and plan((100, 12), 8)[1] is None
    assert plan((256, 256), 16)[1] is not None
    # square grids never hit the rule: the last distributed level keeps more than 16 rows
    for n in range(17, 600, 7):
        assert plan((n, n), 16)[1] is not None, n
    # the rejected case really has a CTA with fine rows but no coarse row
    r0, r1 = partition(level_sizes((120, 17)), 16)
    assert any(r0[r + 1] > r0[r] and r1[r + 1] == r1[r] for r in range(16))


# ---------------------------------------------------------------------------------------------
# schedule model


class _Shared:
    """Distributed shared memory of one cluster, with a race detector per barrier interval."""

    def __init__(self):
        self.v = {}
        self.log = []
        self.races = []

    def rd(self, cta, key):
        self.log.append((cta, False, key))
        return self.v[key]                      # KeyError: a word nobody wrote

    def wr(self, cta, key, val):
        self.log.append((cta, True, key))
        self.v[key] = val

    def barrier(self, where):
        writers = {}
        for cta, w, key in self.log:
            if w:
                writers.setdefault(key, set()).add(cta)
        for cta, w, key in self.log:
            ws = writers.get(key, ())
            if (not w and any(x != cta for x in ws)) or (w and len(ws) > 1):
                self.races.append((where, cta, key))
        self.log = []


def cluster_vcycles(H, b, cycles, C, rlo):
    """`cycles` V-cycles of hierarchy H from x = 0 on b (lexicographic, x fastest), following the
    kernel's steps on C CTAs with row ranges rlo.  Returns (x, races)."""
    sizes, L = H.sizes, len(H.sizes)
    T = L - 1
    nu1, nu2 = H.nu1, H.nu2
    W = [H.omega / d for d in H.D]
    PT = [P.T.tocsr() for P in H.P]
    mem = _Shared()
    cur = [0] * L                               # buffer holding each level's iterate

    def own(l, r):
        return (rlo[l][r], rlo[l][r + 1] - rlo[l][r]) if l < T else (0, sizes[l][1])

    def edge_targets(l, r):
        """(CTA, its local row) receiving this CTA's first and last rows."""
        a, nr = own(l, r)
        if l >= T or nr == 0:
            return None, None
        pr = r - 1
        while pr >= 0 and own(l, pr)[1] == 0:
            pr -= 1
        nx = r + 1
        while nx < C and own(l, nx)[1] == 0:
            nx += 1
        up = (pr, own(l, pr)[1]) if a > 0 and pr >= 0 else None
        dn = (nx, -1) if a + nr < sizes[l][1] and nx < C else None
        return up, dn

    def put(r, l, k, lr, c, val):
        mem.wr(r, (r, l, k, lr, c), val)
        up, dn = edge_targets(l, r)
        if lr == 0 and up:
            mem.wr(r, (up[0], l, k, up[1], c), val)
        if lr == own(l, r)[1] - 1 and dn:
            mem.wr(r, (dn[0], l, k, dn[1], c), val)

    def local(r, l, row):
        a, nr = own(l, r)
        assert -1 <= row - a <= nr, ("outside own and ghost rows", l, r, row)
        return row - a

    def apply(r, l, k, j, c):
        A, n0 = H.A[l], sizes[l][0]
        p = j * n0 + c
        acc = 0.0
        for q, v in zip(A.indices[A.indptr[p]:A.indptr[p + 1]], A.data[A.indptr[p]:A.indptr[p + 1]]):
            jj, cc = divmod(int(q), n0)
            acc += v * mem.rd(r, (r, l, k, local(r, l, jj), cc))
        return acc

    def rows(l, r):
        a, nr = own(l, r)
        return [(lr, a + lr) for lr in range(nr)]

    def sweep(l, kin, zero):
        n0 = sizes[l][0]
        for r in range(C):
            for lr, j in rows(l, r):
                for c in range(n0):
                    bp = mem.rd(r, (r, l, 2, lr, c))
                    w = W[l][j * n0 + c]
                    val = w * bp if zero else mem.rd(r, (r, l, kin, lr, c)) + w * (bp - apply(r, l, kin, j, c))
                    put(r, l, 1 - kin, lr, c, val)

    def residual(l, kin):
        for r in range(C):
            for lr, j in rows(l, r):
                for c in range(sizes[l][0]):
                    put(r, l, 1 - kin, lr, c, mem.rd(r, (r, l, 2, lr, c)) - apply(r, l, kin, j, c))

    def restrict(l, kr):
        lc, n0, n0c = l + 1, sizes[l][0], sizes[l + 1][0]
        R = PT[l]
        for r in range(C):
            for lr, J in rows(lc, r):
                for I in range(n0c):
                    pc = J * n0c + I
                    acc = 0.0
                    for q, w in zip(R.indices[R.indptr[pc]:R.indptr[pc + 1]], R.data[R.indptr[pc]:R.indptr[pc + 1]]):
                        fj, fi = divmod(int(q), n0)
                        if lc < T:
                            key = (r, l, kr, local(r, l, fj), fi)
                        else:                   # into the coarsest: any CTA's rows
                            o = max(x for x in range(C) if rlo[l][x] <= fj and own(l, x)[1] > 0)
                            key = (o, l, kr, fj - rlo[l][o], fi)
                        acc += w * mem.rd(r, key)
                    if lc < T:
                        put(r, lc, 2, lr, I, acc)
                    else:
                        mem.wr(r, (r, lc, 2, lr, I), acc)

    def interpolate(l, kx, kc, ghost):
        """x += P x_c in place: own rows (stored to neighbours) or own and ghost rows (local)."""
        n0, n0c, n1 = sizes[l][0], sizes[l + 1][0], sizes[l][1]
        P = H.P[l]
        for r in range(C):
            a, nr = own(l, r)
            lrs = range(-1, nr + 1) if ghost and nr > 0 else range(nr)
            for lr in lrs:
                F = a + lr
                if not 0 <= F < n1:
                    continue
                for c in range(n0):
                    p = F * n0 + c
                    acc = mem.rd(r, (r, l, kx, lr, c))
                    for q, w in zip(P.indices[P.indptr[p]:P.indptr[p + 1]], P.data[P.indptr[p]:P.indptr[p + 1]]):
                        J, I = divmod(int(q), n0c)
                        acc += w * mem.rd(r, (r, l + 1, kc, local(r, l + 1, J), I))
                    if ghost:
                        mem.wr(r, (r, l, kx, lr, c), acc)
                    else:
                        put(r, l, kx, lr, c, acc)

    # zero fill of every ghost row; b of the finest level staged with its ghost rows
    n0, n1 = sizes[0]
    bg = np.asarray(b).reshape(n1, n0)
    for r in range(C):
        for l in range(L):
            nr = own(l, r)[1]
            for k in range(3):
                for c in range(sizes[l][0]):
                    mem.v[(r, l, k, -1, c)] = 0.0
                    mem.v[(r, l, k, nr, c)] = 0.0
        a, nr = own(0, r)
        for lr in range(-1, nr + 1):
            if 0 <= a + lr < n1:
                for c in range(n0):
                    mem.v[(r, 0, 2, lr, c)] = float(bg[a + lr, c])
    mem.barrier("staging")
    Dinv = np.linalg.inv(H.A[-1].toarray())
    n0c, n1c = sizes[T]
    nc = n0c * n1c
    cs = [r * nc // C for r in range(C + 1)]

    for cyc in range(cycles):
        zero = cyc == 0
        for l in range(L - 1):
            k = cur[l]
            for sw in range(nu1):
                sweep(l, k, zero and sw == 0)
                k ^= 1
                mem.barrier((cyc, l, "pre", sw))
            if zero and nu1 == 0:
                for r in range(C):
                    a, nr = own(l, r)
                    for lr in range(-1, nr + 1) if nr > 0 else ():
                        for c in range(sizes[l][0]):
                            mem.wr(r, (r, l, k, lr, c), 0.0)
                kr = 2
                mem.barrier((cyc, l, "clear"))
            else:
                residual(l, k)
                kr = k ^ 1
                mem.barrier((cyc, l, "residual"))
            cur[l] = k
            restrict(l, kr)                     # block barrier only
            zero = True
        k = cur[T]
        for r in range(C):                      # each CTA's slice of the coarsest solve
            bvec = np.array([mem.rd(r, (r, T, 2, p // n0c, p % n0c)) for p in range(nc)])
            for p in range(cs[r], cs[r + 1]):
                mem.wr(r, (r, T, k, p // n0c, p % n0c), float(Dinv[p] @ bvec))
        mem.barrier((cyc, "coarsest"))
        for r in range(C):                      # gather the other slices (block barrier only)
            for p in range(nc):
                o = max(x for x in range(C) if cs[x] <= p and cs[x + 1] > cs[x])
                if o != r:
                    key = (p // n0c, p % n0c)
                    mem.wr(r, (r, T, k) + key, mem.rd(r, (o, T, k) + key))
        for l in range(L - 2, -1, -1):
            k, kc = cur[l], cur[l + 1]
            if nu2 > 0:
                interpolate(l, k, kc, ghost=True)   # then a block barrier only
                for sw in range(nu2):
                    sweep(l, k, False)
                    k ^= 1
                    mem.barrier((cyc, l, "post", sw))
            else:
                interpolate(l, k, kc, ghost=False)
                mem.barrier((cyc, l, "interpolate"))
            cur[l] = k
    x = np.zeros((n1, n0))
    for r in range(C):
        for lr, j in rows(0, r):
            for c in range(n0):
                x[j, c] = mem.v[(r, 0, cur[0], lr, c)]
    return x.ravel(), mem.races


def _hierarchy(ns, nu1, nu2, kappa=False, shift=0.05 / 128, q1=False):
    if q1:                                  # 9-point fine level (the kernel's stored fine stencil)
        M, K = q1_matrices(ns)
        return Hierarchy((M + shift * K).tocsr(), ns, 0.8, nu1, nu2)
    kap = None
    if kappa:
        kap = np.exp(synth.gaussian_random_field(ns, 0.15, 0.5, synth.rng_for(3, "kappa"), with_boundary=True))
    A = (mass_fd(ns) + shift * stiffness_fd(ns, kappa=kap)).tocsr()
    return Hierarchy(A, ns, 0.8, nu1, nu2)


@pytest.mark.parametrize("ns,C,nu1,nu2,kind", [
    ((40, 36), 16, 2, 2, "fd"), ((40, 36), 16, 0, 1, "fd"), ((40, 36), 16, 1, 0, "fd"),
    ((40, 36), 16, 0, 0, "fd"), ((34, 37), 16, 2, 2, "kappa"), ((120, 17), 8, 2, 2, "fd"),
    ((36, 70), 16, 1, 3, "fd"), ((40, 36), 16, 2, 2, "q1"), ((120, 17), 8, 0, 1, "q1")])
def test_cluster_schedule_matches_oracle(ns, C, nu1, nu2, kind):
    """FD (5-point fine level, constant or kappa field) and Q1 (9-point fine level, stored)."""
    sizes, rlo = plan(ns, C)
    assert rlo is not None
    H = _hierarchy(ns, nu1, nu2, kappa=kind == "kappa", q1=kind == "q1")
    b = synth.random_vector(int(np.prod(ns)), 70)
    x, races = cluster_vcycles(H, b, 2, C, rlo)
    assert not races, races[:3]
    ref = H.solve(b, 2)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_cluster_schedule_needs_nonempty_ranges():
    """Forcing the rejected 16-CTA partition of 120 x 17: no race is reported (nobody stores into
    the empty CTAs' coarse ghost rows), but those CTAs interpolate from zero-filled rows and the
    result is wrong -- the plan rule is what keeps this out of the kernel."""
    ns, C = (120, 17), 16
    H = _hierarchy(ns, 2, 2)
    b = synth.random_vector(int(np.prod(ns)), 71)
    x, races = cluster_vcycles(H, b, 1, C, partition(H.sizes, C))
    ref = H.solve(b, 1)
    assert not races
    assert np.abs(x - ref).max() > 1e-3 * np.abs(ref).max()


# ---------------------------------------------------------------------------------------------
# alignment of the cluster kernel's 16-byte vector accesses (csrc/cluster_mg.cuh), restated from
# its address formulas: rows padded by PAD columns on each side, level l's three buffers at an
# offset that is a multiple of 4 elements, row stride n0 + 2 PAD; a vector of VN = 16 / element
# bytes points is read or written at element offsets that must be multiples of VN.

PAD = 4


def _vector_offsets(sizes, C, VN, faces=False, q1=False):
    """Element offsets (relative to 16-byte aligned bases) of every vector access one V-cycle
    makes on CTA 0..C-1, for the dispatch rules of the kernel."""
    L = len(sizes)
    T = L - 1
    rlo = partition(sizes, C)
    maxr = [max(max(rlo[l][r + 1] - rlo[l][r] for r in range(C)), 1) if l < T else sizes[l][1] for l in range(L)]
    vec = [l < L - 1 and sizes[l][0] % VN == 0 and (l >= 1 or q1 or not faces) for l in range(L)]
    offs = []
    for r in range(C):
        for l in range(L - 1):
            n0 = sizes[l][0]
            ld = n0 + 2 * PAD
            xs = (maxr[l] + 2) * ld
            a, nr = rlo[l][r], rlo[l][r + 1] - rlo[l][r]

            def el(k, lr, c):
                return k * xs + (lr + 1) * ld + c + PAD

            if vec[l]:                                   # sweeps and residual
                for lr in range(nr):
                    for c in range(0, n0, VN):
                        p = lr * n0 + c
                        offs += [el(k, lr, c) for k in range(3)] + [el(0, lr, c) - ld, el(0, lr, c) + ld, p]
                        offs += [q * maxr[l] * n0 + p for q in range(9)]                 # staged stencil
                        offs += [q * sizes[l][0] * sizes[l][1] + a * n0 + p for q in range(9)]   # from L2
                for lr in range(-1, nr + 1):             # interpolation into this level
                    for c in range(0, n0, VN):
                        offs.append(el(0, lr, c))
            cv = l + 1
            if cv < T and vec[cv] and n0 % VN == 0:      # restriction into the next distributed level
                n0c = sizes[cv][0]
                ldc = n0c + 2 * PAD
                xsc = (maxr[cv] + 2) * ldc
                for lr in range(rlo[cv][r + 1] - rlo[cv][r]):
                    J = rlo[cv][r] + lr
                    for I0 in range(0, n0c, VN):
                        for dy in (-1, 0, 1):
                            row = el(0, 2 * J + 1 + dy - a, 0) + 2 * I0
                            offs += [row, row + VN]
                        offs.append(2 * xsc + (lr + 1) * ldc + I0 + PAD)
    return offs


@pytest.mark.parametrize("ns", [(256, 256), (129, 97), (97, 33), (130, 70), (48, 40), (64, 64), (33, 17), (120, 17),
                                (255, 257), (100, 97)])
@pytest.mark.parametrize("ebytes", [4, 8])
def test_vector_accesses_are_16_byte_aligned(ns, ebytes):
    VN = 16 // ebytes
    for C in (16, 8):
        sizes, rlo = plan(ns, C)
        if rlo is None:
            continue
        for faces in (False, True):
            offs = _vector_offsets(sizes, C, VN, faces=faces)
            bad = [o for o in offs if o % VN]
            assert not bad, (ns, C, faces, bad[:5])
