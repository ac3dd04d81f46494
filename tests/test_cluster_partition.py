"""Invariants of the row partition used by the cluster-resident V-cycle (csrc/cluster_mg.cuh and
the plan in csrc/precond.cuh), restated here on the host and checked over many grid shapes and
cluster sizes.

Partition: at the finest level CTA r of C owns grid rows [r*n1 // C, (r+1)*n1 // C); at every
coarser level CTA r owns rows [lo // 2, hi // 2) where [lo, hi) is its range one level finer
(coarse row J sits at fine row 2J+1, 0-based).  Every level but the coarsest is distributed; the
coarsest is held whole by every CTA.  The plan is accepted only when every CTA owns at least one
row of every distributed level (neighbours store their edge rows only into non-empty CTAs, so a
CTA with an empty coarse range would interpolate from ghost rows nobody fills).  For an accepted
plan the kernel relies on:
  * the ranges of each level tile [0, n1_l) in rank order;
  * a CTA's ghost rows are the last row of the previous CTA and the first row of the next one;
  * restriction of an own coarse row J reads fine rows 2J..2J+2, all within one row of the CTA's
    fine range (its own rows or a ghost row);
  * interpolation into an own fine row -- and into the CTA's two ghost rows, which the fused
    interpolation + first sweep computes locally -- reads coarse rows within one row of the CTA's
    coarse range.
"""
import itertools

import pytest

from oracle.multigrid import level_sizes


def plan(ns, C):
    """Row ranges of the distributed levels, or None where the cluster path is not taken."""
    sizes = level_sizes(ns)
    T = len(sizes) - 1
    if len(ns) != 2 or T < 1 or sizes[0][1] < C:
        return sizes, None
    rlo = []
    for l in range(T):
        n1 = sizes[l][1]
        rlo.append([r * n1 // C for r in range(C + 1)] if l == 0 else [v // 2 for v in rlo[l - 1]])
        if any(rlo[l][r + 1] <= rlo[l][r] for r in range(C)):
            return sizes, None
    return sizes, rlo


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
            assert r == 0 or lo[r - 1] < a            # ghost row above: last row of CTA r-1
            assert r == C - 1 or b < lo[r + 2]        # ghost row below: first row of CTA r+1
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
    sizes = level_sizes((120, 17))
    r0 = [r * 17 // 16 for r in range(17)]
    r1 = [v // 2 for v in r0]
    assert len(sizes) == 3 and any(r0[r + 1] > r0[r] and r1[r + 1] == r1[r] for r in range(16))
