"""Pins of the oracle's storage-precision emulation (oracle.lowprec)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import lowprec as lp
from oracle.multigrid import Hierarchy
from oracle.operators import operators
from oracle.precond import Preconditioner
from oracle.solve import build


def _all_values(fmt):
    """Every finite value of a 16-bit format, as float64, with its bit pattern."""
    bits = np.arange(1 << 16, dtype=np.uint32)
    with np.errstate(invalid="ignore"):
        if fmt == "bf16":
            vals = (bits << np.uint32(16)).view(np.float32).astype(np.float64)
        else:
            vals = bits.astype(np.uint16).view(np.float16).astype(np.float64)
    ok = np.isfinite(vals)
    return vals[ok], bits[ok]


def _nearest_even(x, fmt):
    """Brute force: the format's value nearest to x, ties to the even bit pattern."""
    vals, bits = _all_values(fmt)
    order = np.argsort(vals, kind="stable")
    vals, bits = vals[order], bits[order]
    out = np.empty_like(x)
    for n, v in enumerate(x):
        d = np.abs(vals - v)
        best = np.flatnonzero(d == d.min())
        if len(best) > 1:
            even = [i for i in best if bits[i] % 2 == 0 and vals[i] != 0.0] or list(best)
            best = even
        out[n] = vals[best[0]]
    return out


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_rounding_is_nearest_ties_to_even(fmt):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(300) * 10.0 ** rng.integers(-6, 5, 300),
                        rng.standard_normal(50) * 1e-3])
    vals, _ = _all_values(fmt)
    vals = np.unique(vals[vals > 0])
    mids = 0.5 * (vals[:-1] + vals[1:])            # exact ties between neighbours
    pick = mids[rng.integers(0, len(mids), 200)]
    pick = pick[(pick < 6.0e4) & (pick > 1e-4)]
    x = np.concatenate([x, pick, -pick]).astype(np.float32)
    got = (lp.round_bf16(x) if fmt == "bf16" else lp.round_fp16(x)).astype(np.float64)
    assert np.array_equal(got, _nearest_even(x.astype(np.float64), fmt))


@pytest.mark.parametrize("fmt,u", [("bf16", 2.0 ** -8), ("fp16", 2.0 ** -11)])
def test_row_scales_powers_of_two_and_half_ulp(fmt, u):
    rng = np.random.default_rng(2)
    n0 = 37
    x = (rng.standard_normal((20, n0)) * 10.0 ** rng.integers(-8, 8, (20, 1))).astype(np.float32)
    x[3] = 0.0
    sc, inv = lp.row_scales(x)
    m, e = np.frexp(sc.astype(np.float64))
    assert np.all(m == 0.5)                                   # exact powers of two
    assert np.all(sc * inv == 1.0)
    scaled = np.abs(x).max(axis=1) * inv
    nz = np.abs(x).max(axis=1) > 0
    assert np.all((scaled[nz] >= 2.0 ** 13) & (scaled[nz] < 2.0 ** 14))
    y = lp.store_rows(x.reshape(-1), n0, fmt).reshape(x.shape)
    assert np.all(y[3] == 0.0)
    tiny = (2.0 ** -24 if fmt == "fp16" else 0.0) * sc[:, None]      # fp16 subnormals below 2^-14
    assert np.all(np.abs(y - x) <= u * np.abs(x) + tiny)
    # storage is idempotent: stored values are representable with the same scales
    assert np.array_equal(lp.store_rows(y.reshape(-1), n0, fmt).reshape(x.shape), y)


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16"])
def test_stencil_storage_per_component(fmt):
    ns = (40, 36)
    _, K = operators(ns)
    A = sp.identity(K.shape[0], format="csr") + 0.01 * K
    h = Hierarchy(A, ns, 0.8, 2, 2)
    S = lp.stencil_of(h.A[1], h.sizes[1])
    assert (lp.matrix_of(S, h.sizes[1]) - h.A[1]).count_nonzero() == 0      # stencil <-> matrix
    St = lp.store_stencil(S, fmt)
    u = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}[fmt]
    assert np.all(np.abs(St - S) <= u * np.abs(S) * (1 + 1e-12))
    if fmt != "fp32":
        sc = lp.stencil_scales(S).astype(np.float64)
        m, _ = np.frexp(sc)
        assert np.all(m == 0.5)                                   # exact powers of two
        mx = np.abs(S).max(axis=1)
        nz = mx > 0
        # the stored maximum of every component lands in [2^13, 2^14]
        assert np.all((mx[nz] / sc[nz] >= 2.0 ** 13) & (mx[nz] / sc[nz] < 2.0 ** 14))
        assert np.all(np.abs(St).max(axis=1)[nz] / sc[nz] <= 2.0 ** 14)


@pytest.mark.parametrize("ns", [(40, 36), (64, 64), (12, 10, 14)])
def test_fp64_storage_reduces_to_the_oracle_vcycles(ns):
    _, K = operators(ns)
    h = Hierarchy(sp.identity(K.shape[0], format="csr") + 0.02 * K, ns, 0.8, 2, 2)
    b = synth.random_vector(K.shape[0], 5)
    ref = h.solve(b, 3)
    m = lp.StoredMG(h, "fp64")
    for plan in (lp.Plan(keep_x=True), lp.Plan(onchip_from=0), lp.Plan(onchip_from=1, fuse=[True] * 4),
                 lp.Plan(onchip_from=1, fuse=[False] * 4)):
        x = m.solve(b, 3, plan)
        assert np.abs(x - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("fmt,bound", [("fp32", 2e-5), ("bf16", 2e-2), ("fp16", 3e-3)])
def test_lowprec_vcycles_within_roundoff_of_fp64(fmt, bound):
    ns = (48, 40)
    _, K = operators(ns)
    h = Hierarchy(sp.identity(K.shape[0], format="csr") + 0.02 * K, ns, 0.8, 2, 2)
    b = synth.random_vector(K.shape[0], 6)
    ref = h.solve(b, 3)
    m = lp.StoredMG(h, fmt)
    for plan in (lp.Plan(keep_x=True), lp.Plan(onchip_from=1, fuse=[False] * 4)):
        x = m.solve(lp.store_rows(b, ns[0], fmt), 3, plan)
        err = np.abs(x - ref).max() / np.abs(ref).max()
        assert err <= bound
    # FP32 storage of float32 results is exact, so the memory plan cannot matter there; with
    # 16-bit storage, storing every intermediate differs from keeping them on chip
    x1 = m.solve(lp.store_rows(b, ns[0], fmt), 3, lp.Plan(keep_x=True))
    x2 = m.solve(lp.store_rows(b, ns[0], fmt), 3, lp.Plan(onchip_from=1, fuse=[False] * 4))
    if fmt == "fp32":
        assert np.array_equal(x1, x2)
    else:
        assert np.abs(x1 - x2).max() > 0.0


@pytest.mark.parametrize("ns,s", [((24, 20), 3), ((7, 6, 5), 2)])
def test_fp64_storage_reduces_to_the_oracle_preconditioner(ns, s):
    nt = 3
    op = build(ns, 1.0, nt, "radau", s)
    P = Preconditioner(op, ns, inner_maxit=3, inner_tol=1e-3, omega=0.8)
    E = lp.StoredPreconditioner(P, "fp64", "fp64", lp.Plan(onchip_from=0), lp.Plan(keep_x=True))
    r = synth.random_vector(op.n_st, 9)
    rb = r[op.n_v: op.n_v + s * op.nx]
    assert np.abs(E.pint(rb, E.plan_single) - P.pint_apply(rb)).max() <= 1e-14 * np.abs(P.pint_apply(rb)).max()
    ref_t = P.pint_apply_T(rb)
    assert np.abs(E.pint(rb, E.plan_single, transpose=True) - ref_t).max() <= 1e-14 * np.abs(ref_t).max()
    ref_i = P.inner_solve(rb)
    assert np.abs(E.inner_solve(rb, E.plan_batch) - ref_i).max() <= 1e-13 * np.abs(ref_i).max()
    ref = P.apply(r)
    assert np.abs(E.apply(r) - ref).max() <= 1e-13 * np.abs(ref).max()
    ref = P.apply_T(r)
    assert np.abs(E.apply_T(r) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("fmtP,fmtI,bound", [("fp32", "fp32", 1e-5), ("fp32", "bf16", 3e-2),
                                             ("bf16", "bf16", 3e-2), ("fp16", "fp16", 5e-3)])
def test_lowprec_preconditioner_within_roundoff_of_fp64(fmtP, fmtI, bound):
    ns, nt, s = (24, 20), 3, 3
    op = build(ns, 1.0, nt, "radau", s)
    P = Preconditioner(op, ns, inner_maxit=3, inner_tol=0.0, omega=0.8)
    E = lp.StoredPreconditioner(P, fmtP, fmtI, lp.Plan(onchip_from=0), lp.Plan(keep_x=True))
    r = synth.random_vector(op.n_st, 10)
    for got, ref in ((E.apply(r), P.apply(r)), (E.apply_T(r), P.apply_T(r))):
        assert np.linalg.norm(got - ref) <= bound * np.linalg.norm(ref)


def test_unscaled_fp16_storage_overflows_where_scaled_storage_does_not():
    """Why 16-bit rows carry a scale: a right-hand side of size 1e7 (and the stiff problem's
    K-sized intermediates, 4/h^2 ~ 2.6e5 at 256^2) exceed FP16's largest value 65504."""
    x = (1e7 * synth.random_vector(256, 8)).astype(np.float32)
    assert np.isinf(lp.round_fp16(x)).any()
    y = lp.store_rows(x, 64, "fp16")
    assert np.all(np.isfinite(y)) and np.abs(y - x).max() <= 2.0 ** -11 * np.abs(x).max()
