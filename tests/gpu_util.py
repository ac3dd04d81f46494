"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev())


def zeros(n):
    return torch.zeros(int(n), dtype=torch.float64, device=dev())


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_max(a, b):
    """max |a - b| / max |b| (element-wise comparison scaled by the reference's size)."""
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def gpu_plan(sizes, B, cluster=False, fmt="fp32"):
    """The CUDA path's multigrid memory plan for B items of a hierarchy with level sizes `sizes`
    (finest first), restated from its launch rules for the storage emulation of the oracle:
    up to 32 items of a 2D grid with a cluster plan keep all their V-cycles on chip (one
    thread-block cluster per item); otherwise the levels
    from the first one with at most 4096 (B > 1) or 1024 (B = 1) points down run as one on-chip
    V-cycle, and a level above them fuses its steps when B * points <= 2^20 and it is 2D or the
    matrix-free finest level, except a 16-bit finest level whose rows are whole 16-byte vectors
    (n0 a multiple of 8, at most 256), which streams through separate vectorised sweeps."""
    from oracle.lowprec import Plan
    if cluster and B <= 32:
        return Plan(keep_x=True)
    pts = [int(np.prod(s)) for s in sizes]
    maxp = 4096 if B > 1 else 1024
    lc = len(sizes) - 1
    for l in range(len(sizes) - 1, -1, -1):
        if pts[l] > maxp:
            break
        lc = l
    d = len(sizes[0])
    n0 = sizes[0][0]
    vec0 = fmt in ("bf16", "fp16") and n0 % 8 == 0 and n0 // 8 <= 32
    fuse = [B * pts[l] <= (1 << 20) and (d == 2 or l == 0) and not (l == 0 and vec0) for l in range(len(sizes))]
    return Plan(onchip_from=lc, fuse=fuse)


def lowprec_errors(got, ref):
    """(relative 2-norm, relative max-norm, fraction of entries differing by more than 1e-5 of
    the reference's max) of a GPU result against the storage emulation."""
    got, ref = np.asarray(got), np.asarray(ref)
    d = np.abs(got - ref)
    mx = np.abs(ref).max()
    return (float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), float(d.max() / mx),
            float(np.mean(d > 1e-5 * mx)))


def storage_ulps(got, ref, n0, fmt):
    """Largest |got - ref| per entry in units in the last place of the 16-bit format fmt at the
    stored value of ref (ref's per-row power-of-two scales, rows of n0), with a float32 noise
    floor of 2^-18 of the row's maximum added to each unit (entries near zero have units far
    below the float32 rounding-order noise of the arithmetic that produced them), and the
    fraction of entries that differ at all."""
    from oracle.lowprec import row_scales
    ref32 = np.asarray(ref, dtype=np.float32).reshape(-1, n0)
    got = np.asarray(got, dtype=np.float64).reshape(-1, n0)
    sc, inv = row_scales(ref32)
    v = np.abs(ref32.astype(np.float64) * inv[:, None])
    mant = 7 if fmt == "bf16" else 10
    tiny = 2.0 ** -14 if fmt == "fp16" else 2.0 ** -126
    e = np.floor(np.log2(np.maximum(v, tiny)))
    rowmax = np.abs(ref32.astype(np.float64)).max(axis=1, keepdims=True)
    ulp = 2.0 ** (e - mant) * sc[:, None].astype(np.float64) + 2.0 ** -18 * rowmax
    d = np.abs(got - ref32.astype(np.float64))
    return float((d / ulp).max()), float(np.mean(d > 0))
