// Geometric Galerkin multigrid for the shifted operators M + c K (Sec. 5:
// "(M + cK)^{-1} by 3 V-cycles"; the paper's closed AMG is replaced by a
// geometric V-cycle with a fixed definition):
//   coarse points = even fine indices (1-based), N_c = N / 2 per axis;
//   1D interpolation: injection at coarse points, average of the two
//   neighbours at odd points (a Dirichlet neighbour counts 0); P = tensor
//   product, R = P^T, A_c = P^T A P stored as a 3^d-point stencil per point;
//   damped-Jacobi smoothing; dense exact solve at the coarsest level.
// All kernels are row kernels: one warp per (batch item, grid row), lanes
// along x, so a row's per-row scale (16-bit storage) is one warp reduction.
#pragma once

#include "common.cuh"

namespace aao {

// Operator of one level as the kernels see it, arithmetic type A.
template <class S> struct LevelOp {
    using A = typename PT<S>::A;
    Geo g;
    int fine = 1;            // 1: matrix-free sigma*u + c*K u; 0: stored stencil
    A sigma = A(1), c = A(0);
    Faces<A> faces;          // fine level, variable kappa (nullptr = kappa 1)
    const S* sten = nullptr; // coarse: ncoef*nx, component-major
    const float* sten_sc = nullptr;  // coarse, scaled types: one scale per component
    int ncoef = 9;
};

template <class S>
__device__ __forceinline__ typename PT<S>::A sten_coef(const LevelOp<S>& op, int q, long long p) {
    typename PT<S>::A v = PT<S>::ld(op.sten[(long long)q * op.g.nx + p]);
    if constexpr (PT<S>::scaled) v *= op.sten_sc[q];
    return v;
}

// (A u)_P and the diagonal a_PP at column c of row (j,k).
template <class S, class SU>
__device__ __forceinline__ void level_apply(const LevelOp<S>& op, const View<SU>& u, long long row, int j,
                                            int k, int c, typename PT<S>::A& Au,
                                            typename PT<S>::A& diag) {
    using A = typename PT<S>::A;
    const Geo& g = op.g;
    if (op.fine) {
        Au = op.sigma * A(u.at(row, c)) + op.c * A(fd_K(u, g, op.faces, row, j, k, c));
        diag = op.sigma + op.c * fd_K_diag<A>(g, op.faces, row, j, k, c);
        return;
    }
    const long long p = row * g.n0 + c;
    A acc = A(0);
    const int zlo = g.d == 3 ? -1 : 0, zhi = g.d == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int kk = k + dz;
        if (kk < 0 || kk >= g.n2) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int jj = j + dy;
            if (jj < 0 || jj >= g.n1) continue;
            long long rr = row + dy + (long long)dz * g.n1;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                int cc = c + dx;
                if (cc < 0 || cc >= g.n0) continue;
                int q = (dx + 1) + 3 * (dy + 1) + (g.d == 3 ? 9 * (dz + 1) : 0);
                acc += sten_coef(op, q, p) * A(u.at(rr, cc));
            }
        }
    }
    Au = acc;
    diag = sten_coef(op, g.d == 3 ? 13 : 4, p);
}

// (A u)_P and a_PP for a level whose values come from a getter u(row, col)
// (used by the fused kernels, where u is itself computed on the fly).
template <class S, class G>
__device__ __forceinline__ void level_apply_g(const LevelOp<S>& op, G&& u, long long row, int j, int k, int c,
                                              typename PT<S>::A& Au, typename PT<S>::A& diag) {
    using A = typename PT<S>::A;
    const Geo& g = op.g;
    if (op.fine) {
        A uP = u(row, c);
        A uW = c > 0 ? u(row, c - 1) : A(0);
        A uE = c + 1 < g.n0 ? u(row, c + 1) : A(0);
        A uS = j > 0 ? u(row - 1, c) : A(0);
        A uN = j + 1 < g.n1 ? u(row + 1, c) : A(0);
        A uD = A(0), uU = A(0);
        if (g.d == 3) {
            uD = k > 0 ? u(row - g.n1, c) : A(0);
            uU = k + 1 < g.n2 ? u(row + g.n1, c) : A(0);
        }
        A Ku;
        const Faces<A>& f = op.faces;
        if (f.fx == nullptr) {
            Ku = A(g.hx2) * (A(2) * uP - uW - uE) + A(g.hy2) * (A(2) * uP - uS - uN);
            if (g.d == 3) Ku += A(g.hz2) * (A(2) * uP - uD - uU);
        } else {
            const long long fxi = row * (g.n0 + 1) + c;
            const long long fyi = ((long long)k * (g.n1 + 1) + j) * g.n0 + c;
            Ku = A(f.fx[fxi]) * (uP - uW) + A(f.fx[fxi + 1]) * (uP - uE) + A(f.fy[fyi]) * (uP - uS) +
                 A(f.fy[fyi + g.n0]) * (uP - uN);
            if (g.d == 3) {
                const long long fzi = ((long long)k * g.n1 + j) * g.n0 + c;
                Ku += A(f.fz[fzi]) * (uP - uD) + A(f.fz[fzi + (long long)g.n1 * g.n0]) * (uP - uU);
            }
        }
        Au = op.sigma * uP + op.c * Ku;
        diag = op.sigma + op.c * fd_K_diag<A>(g, op.faces, row, j, k, c);
        return;
    }
    const long long p = row * g.n0 + c;
    A acc = A(0);
    const int zlo = g.d == 3 ? -1 : 0, zhi = g.d == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int kk = k + dz;
        if (kk < 0 || kk >= g.n2) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            int jj = j + dy;
            if (jj < 0 || jj >= g.n1) continue;
            long long rr = row + dy + (long long)dz * g.n1;
            for (int dx = -1; dx <= 1; ++dx) {
                int cc = c + dx;
                if (cc < 0 || cc >= g.n0) continue;
                int q = (dx + 1) + 3 * (dy + 1) + (g.d == 3 ? 9 * (dz + 1) : 0);
                acc += sten_coef(op, q, p) * u(rr, cc);
            }
        }
    }
    Au = acc;
    diag = sten_coef(op, g.d == 3 ? 13 : 4, p);
}

template <class S>
__device__ __forceinline__ typename PT<S>::A level_diag(const LevelOp<S>& op, long long row, int j, int k, int c) {
    using A = typename PT<S>::A;
    if (op.fine) return op.sigma + op.c * fd_K_diag<A>(op.g, op.faces, row, j, k, c);
    return sten_coef(op, op.g.d == 3 ? 13 : 4, row * op.g.n0 + c);
}

// Two damped-Jacobi sweeps in one pass: the first sweep is recomputed at the
// point and at its stencil neighbours (x_in.d == nullptr: zero initial guess).
template <class S>
__global__ void __launch_bounds__(kPtMaxThreads) k_smooth2(LevelOp<S> op, PtMap pm, int B, const int* active,
                                                           Vec<S> xin, Vec<S> bv, Vec<S> xout,
                                                           typename PT<S>::A omega) {
    pdl_prologue();
    using A = typename PT<S>::A;
    const Geo g = op.g;
    PtPos q = pt_pos(pm, B, g.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int j, k;
    row_jk(g, row, j, k);
    View<S> bb = view_of(bv, q.b, 0, g.n0);
    const bool has = xin.d != nullptr;
    View<S> xx = has ? view_of(xin, q.b, 0, g.n0) : View<S>{nullptr, nullptr, g.n0};
    auto x1 = [&](long long rr, int cc) -> A {
        int jj, kk;
    row_jk(g, rr, jj, kk);
        if (!has) return omega * bb.at(rr, cc) / level_diag(op, rr, jj, kk, cc);
        A Au, dg;
        level_apply(op, xx, rr, jj, kk, cc, Au, dg);
        return xx.at(rr, cc) + omega * (bb.at(rr, cc) - Au) / dg;
    };
    S* out; float* osc;
    row_store_ptrs(xout, q.b, 0, row, g.n0, out, osc);
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
        A Au, dg;
        level_apply_g(op, x1, row, j, k, c, Au, dg);
        return x1(row, c) + omega * (bb.at(row, c) - Au) / dg;
    });
}

// bc = P^T (b - A x) with the fine residual computed on the fly (coarse rows;
// x.d == nullptr: x = 0, residual = b).
template <class S>
__global__ void __launch_bounds__(kPtMaxThreads) k_resid_restrict(LevelOp<S> op, Geo gc, PtMap pm, int B,
                                                                  const int* active, Vec<S> xv, Vec<S> bv,
                                                                  Vec<S> bcv) {
    pdl_prologue();
    using A = typename PT<S>::A;
    const Geo gf = op.g;
    PtPos q = pt_pos(pm, B, gc.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int J, Kc;
    row_jk(gc, row, J, Kc);
    View<S> bb = view_of(bv, q.b, 0, gf.n0);
    const bool has = xv.d != nullptr;
    View<S> xx = has ? view_of(xv, q.b, 0, gf.n0) : View<S>{nullptr, nullptr, gf.n0};
    S* out; float* osc;
    row_store_ptrs(bcv, q.b, 0, row, gc.n0, out, osc);
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int I) -> A {
        A acc = A(0);
        const int zlo = gf.d == 3 ? -1 : 0, zhi = gf.d == 3 ? 1 : 0;
        for (int dz = zlo; dz <= zhi; ++dz) {
            int fk = gf.d == 3 ? 2 * Kc + 1 + dz : 0;
            if (fk < 0 || fk >= gf.n2) continue;
            A wz = dz == 0 ? A(1) : A(0.5);
            for (int dy = -1; dy <= 1; ++dy) {
                int fj = 2 * J + 1 + dy;
                if (fj < 0 || fj >= gf.n1) continue;
                A wy = dy == 0 ? A(1) : A(0.5);
                long long frow = fj + (long long)gf.n1 * fk;
                for (int dx = -1; dx <= 1; ++dx) {
                    int fi = 2 * I + 1 + dx;
                    if (fi < 0 || fi >= gf.n0) continue;
                    A wx = dx == 0 ? A(1) : A(0.5);
                    A r = bb.at(frow, fi);
                    if (has) {
                        A Au, dg;
                        level_apply(op, xx, frow, fj, fk, fi, Au, dg);
                        r -= Au;
                    }
                    acc += wx * wy * wz * r;
                }
            }
        }
        return acc;
    });
}

// Level kinds known at compile time (fewer registers than the run-time dispatch of level_apply):
// 0 any, 1 matrix-free FD level, 2 stored 9-point (2D), 3 stored 27-point (3D),
// 4: matrix-free FD level in 2D.
inline int level_kind(int fine, int d) { return fine ? (d == 2 ? 4 : 1) : (d == 2 ? 2 : 3); }

template <int KIND, class S, class SU>
__device__ __forceinline__ void level_apply_k(const LevelOp<S>& op, const View<SU>& u, long long row, int j, int k,
                                              int c, typename PT<S>::A& Au, typename PT<S>::A& diag) {
    using A = typename PT<S>::A;
    const Geo& g = op.g;
    if constexpr (KIND == 1) {
        Au = op.sigma * A(u.at(row, c)) + op.c * A(fd_K(u, g, op.faces, row, j, k, c));
        diag = op.sigma + op.c * fd_K_diag<A>(g, op.faces, row, j, k, c);
    } else if constexpr (KIND == 4) {
        // fd_K / fd_K_diag for d = 2 (same arithmetic, 32-bit indexing within the item)
        const int r = (int)row, n0 = g.n0;
        const A uP = A(u.at(r, c));
        const A uW = c > 0 ? A(u.at(r, c - 1)) : A(0);
        const A uE = c + 1 < n0 ? A(u.at(r, c + 1)) : A(0);
        const A uS = j > 0 ? A(u.at(r - 1, c)) : A(0);
        const A uN = j + 1 < g.n1 ? A(u.at(r + 1, c)) : A(0);
        A K, kd;
        if (op.faces.fx == nullptr) {
            K = A(g.hx2) * (A(2) * uP - uW - uE) + A(g.hy2) * (A(2) * uP - uS - uN);
            kd = A(2) * A(g.hx2) + A(2) * A(g.hy2);
        } else {
            const int fxi = r * (n0 + 1) + c, fyi = j * n0 + c;
            const A fx0 = A(op.faces.fx[fxi]), fx1 = A(op.faces.fx[fxi + 1]);
            const A fy0 = A(op.faces.fy[fyi]), fy1 = A(op.faces.fy[fyi + n0]);
            K = fx0 * (uP - uW) + fx1 * (uP - uE) + fy0 * (uP - uS) + fy1 * (uP - uN);
            kd = fx0 + fx1 + fy0 + fy1;
        }
        Au = op.sigma * uP + op.c * K;
        diag = op.sigma + op.c * kd;
    } else if constexpr (KIND == 2) {
        const long long p = row * g.n0 + c;
        A acc = A(0);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int jj = j + dy;
            if (jj < 0 || jj >= g.n1) continue;
            const long long rr = row + dy;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int cc = c + dx;
                if (cc < 0 || cc >= g.n0) continue;
                acc += sten_coef(op, (dx + 1) + 3 * (dy + 1), p) * A(u.at(rr, cc));
            }
        }
        Au = acc;
        diag = sten_coef(op, 4, p);
    } else {
        level_apply(op, u, row, j, k, c, Au, diag);
    }
}

template <int KIND, class S>
__device__ __forceinline__ typename PT<S>::A level_diag_k(const LevelOp<S>& op, long long row, int j, int k, int c) {
    using A = typename PT<S>::A;
    if constexpr (KIND == 1 || KIND == 4) return op.sigma + op.c * fd_K_diag<A>(op.g, op.faces, row, j, k, c);
    else if constexpr (KIND == 2) return sten_coef(op, 4, row * op.g.n0 + c);
    else return level_diag(op, row, j, k, c);
}

// x_out = x_in + omega D^{-1} (b - A x_in); x_in.d == nullptr means x_in = 0.
template <class S, int KIND = 0>
__global__ void __launch_bounds__(kPtMaxThreads) k_smooth(LevelOp<S> op, PtMap pm, int B, const int* active, Vec<S> xin,
                                                 Vec<S> bv, Vec<S> xout, typename PT<S>::A omega) {
    pdl_prologue();
    using A = typename PT<S>::A;
    const Geo g = op.g;
    PtPos q = pt_pos(pm, B, g.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int j, k;
    row_jk(g, row, j, k);
    View<S> bb = view_of(bv, q.b, 0, g.n0);
    S* out; float* osc;
    row_store_ptrs(xout, q.b, 0, row, g.n0, out, osc);
    if (xin.d == nullptr) {
        pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
            const A dg = level_diag_k<KIND>(op, row, j, k, c);
            return omega * bb.at(row, c) / dg;
        });
    } else {
        View<S> xx = view_of(xin, q.b, 0, g.n0);
        pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
            A Au, dg;
            level_apply_k<KIND>(op, xx, row, j, k, c, Au, dg);
            return xx.at(row, c) + omega * (bb.at(row, c) - Au) / dg;
        });
    }
}

// k_smooth for unscaled storage with RPT rows per thread (rows r0, r0 + rpc, ...): all rows'
// values are computed before any store, so their loads are in flight together; fewer, longer CTAs
// for large batches.  One column per thread (n0 <= n0p).
template <class S, int KIND, int RPT>
__global__ void __launch_bounds__(kPtMaxThreads) k_smooth_rows(LevelOp<S> op, PtMap pm, int B, const int* active,
                                                               Vec<S> xin, Vec<S> bv, Vec<S> xout,
                                                               typename PT<S>::A omega) {
    pdl_prologue();
    using A = typename PT<S>::A;
    static_assert(!PT<S>::scaled, "unscaled storage only");
    const Geo g = op.g;
    const int b = blockIdx.y;
    if (b >= B || (active && !active[b])) return;
    const int c = threadIdx.x;
    if (c >= g.n0) return;
    const int r0 = blockIdx.x * pm.rpc * RPT + threadIdx.y;
    View<S> bb = view_of(bv, b, 0, g.n0);
    S* out = xout.d + (long long)b * xout.bs;
    A v[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i * pm.rpc;
        v[i] = A(0);
        if (row < g.R) {
            if (xin.d == nullptr) {
                v[i] = omega * bb.at(row, c) / level_diag_k<KIND>(op, row, row, 0, c);
            } else {
                View<S> xx = view_of(xin, b, 0, g.n0);
                A Au, dg;
                level_apply_k<KIND>(op, xx, row, row, 0, c, Au, dg);
                v[i] = xx.at(row, c) + omega * (bb.at(row, c) - Au) / dg;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i * pm.rpc;
        if (row < g.R) out[(long long)row * g.n0 + c] = PT<S>::st(v[i]);
    }
}

// ---------------------------------------------------------------------------
// Batched 2D matrix-free level (sigma I + c K, kappa = 1), unscaled storage, streaming form:
// a thread owns V consecutive columns (one 16-byte vector) of a strip of RS rows and keeps the
// rows j-1, j, j+1 of x in registers while it walks down the strip, so each point costs one
// vector load of x, one of b and one store (plus two scalar halo loads per row and two halo
// rows per strip); the next row's loads are issued before the current row is computed.
// MODE 0: damped Jacobi x + (omega / a_PP) (b - A x); MODE 1: the same from x = 0
// ((omega / a_PP) b, x is not read); MODE 2: the residual b - A x.  A x as level_apply_k<4>;
// the Jacobi weight omega / a_PP as the cluster V-cycle.  Block: 256 threads = (n0 / V)
// threads per row x strips; grid (ceil(n1 / (strips RS)), items).
// ---------------------------------------------------------------------------
template <class S> struct Vec16;
template <> struct Vec16<float> {
    using T = float4;
    static constexpr int n = 4;
};
template <> struct Vec16<double> {
    using T = double2;
    static constexpr int n = 2;
};
constexpr int kStripThreads = 256;
constexpr int kStripRows = 8;

template <class S, int MODE>
__global__ void __launch_bounds__(kStripThreads) k_strip2d(LevelOp<S> op, int B, const int* active, Vec<S> xin,
                                                           Vec<S> bv, Vec<S> out, S omega) {
    pdl_prologue();
    static_assert(!PT<S>::scaled, "unscaled storage only");
    using VT = typename Vec16<S>::T;
    constexpr int V = Vec16<S>::n;
    const Geo g = op.g;
    const int b = blockIdx.y;
    if (b >= B || (active && !active[b])) return;
    const int n0 = g.n0, n1 = g.n1;
    const int tpr = n0 / V;
    const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
    const int strips = blockDim.x / tpr;
    if (ty >= strips) return;
    const int j0 = (blockIdx.x * strips + ty) * kStripRows;
    if (j0 >= n1) return;
    const int j1 = j0 + kStripRows < n1 ? j0 + kStripRows : n1;
    const int c0 = tx * V;
    const S* X = MODE == 1 ? nullptr : xin.d + (long long)b * xin.bs;
    const S* Bp = bv.d + (long long)b * bv.bs;
    S* O = out.d + (long long)b * out.bs;
    const S hx2 = S(g.hx2), hy2 = S(g.hy2);
    const S kd = S(2) * hx2 + S(2) * hy2;
    const S wgt = omega / (op.sigma + op.c * kd);      // omega / a_PP, as the cluster V-cycle
    auto load_row = [&](int j, S* dst) {
        if (j >= 0 && j < n1) {
            VT v = *reinterpret_cast<const VT*>(X + (long long)j * n0 + c0);
            const S* q = reinterpret_cast<const S*>(&v);
#pragma unroll
            for (int t = 0; t < V; ++t) dst[t] = q[t];
        } else {
#pragma unroll
            for (int t = 0; t < V; ++t) dst[t] = S(0);
        }
    };
    auto load_b = [&](int j, S* dst) {
        VT v = *reinterpret_cast<const VT*>(Bp + (long long)j * n0 + c0);
        const S* q = reinterpret_cast<const S*>(&v);
#pragma unroll
        for (int t = 0; t < V; ++t) dst[t] = q[t];
    };
    // the loads of row j + 1 are issued before row j is computed (two rows in flight per thread)
    S sr[V], pr[V], nr[V], bq[V], nn[V], bn[V];
    S w = S(0), e = S(0), wn = S(0), en = S(0);
    load_b(j0, bq);
    if (MODE != 1) {
        load_row(j0 - 1, sr);
        load_row(j0, pr);
        load_row(j0 + 1, nr);
        w = c0 > 0 ? X[(long long)j0 * n0 + c0 - 1] : S(0);
        e = c0 + V < n0 ? X[(long long)j0 * n0 + c0 + V] : S(0);
    }
    for (int j = j0; j < j1; ++j) {
        const bool more = j + 1 < j1;
        if (more) {
            load_b(j + 1, bn);
            if (MODE != 1) {
                load_row(j + 2, nn);
                wn = c0 > 0 ? X[(long long)(j + 1) * n0 + c0 - 1] : S(0);
                en = c0 + V < n0 ? X[(long long)(j + 1) * n0 + c0 + V] : S(0);
            }
        }
        S res[V];
        if (MODE == 1) {
#pragma unroll
            for (int t = 0; t < V; ++t) res[t] = wgt * bq[t];
        } else {
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const S uP = pr[t], uW = t == 0 ? w : pr[t - 1], uE = t == V - 1 ? e : pr[t + 1];
                const S K = hx2 * (S(2) * uP - uW - uE) + hy2 * (S(2) * uP - sr[t] - nr[t]);
                const S Au = op.sigma * uP + op.c * K;
                res[t] = MODE == 0 ? uP + wgt * (bq[t] - Au) : bq[t] - Au;
            }
        }
        VT ov;
        S* oq = reinterpret_cast<S*>(&ov);
#pragma unroll
        for (int t = 0; t < V; ++t) oq[t] = res[t];
        *reinterpret_cast<VT*>(O + (long long)j * n0 + c0) = ov;
        if (more) {
#pragma unroll
            for (int t = 0; t < V; ++t) {
                bq[t] = bn[t];
                if (MODE != 1) {
                    sr[t] = pr[t];
                    pr[t] = nr[t];
                    nr[t] = nn[t];
                }
            }
            w = wn;
            e = en;
        }
    }
}

// The same streaming form for a 2D level with a stored 9-point stencil (a coarse Galerkin level;
// unscaled storage): the stencil's 9 component rows are read as 16-byte vectors beside x (the
// stencil is shared by all items, so it stays in L1/L2), the corner and side neighbours of the
// vector come from the three rows in registers plus two scalars per row.  Per point the operations
// of level_apply_k<2> in its order (neighbours beyond the grid read as zero instead of being
// skipped: the same value) and of k_smooth / k_residual: x + omega (b - A x) / a_PP.
template <class S, int MODE>
__global__ void __launch_bounds__(kStripThreads) k_strip2d_st(LevelOp<S> op, int B, const int* active, Vec<S> xin,
                                                              Vec<S> bv, Vec<S> out, S omega, int rs) {
    pdl_prologue();
    static_assert(!PT<S>::scaled, "unscaled storage only");
    using VT = typename Vec16<S>::T;
    constexpr int V = Vec16<S>::n;
    const Geo g = op.g;
    const int b = blockIdx.y;
    if (b >= B || (active && !active[b])) return;
    const int n0 = g.n0, n1 = g.n1;
    const int tpr = n0 / V;
    const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
    const int strips = blockDim.x / tpr;
    if (ty >= strips) return;
    const int j0 = (blockIdx.x * strips + ty) * rs;     // rs rows per strip (strip_st_rows)
    if (j0 >= n1) return;
    const int j1 = j0 + rs < n1 ? j0 + rs : n1;
    const int c0 = tx * V;
    const long long nx = g.nx;
    const S* X = MODE == 1 ? nullptr : xin.d + (long long)b * xin.bs;
    const S* Bp = bv.d + (long long)b * bv.bs;
    S* O = out.d + (long long)b * out.bs;
    auto vld = [&](const S* p, S* dst) {
        VT v = *reinterpret_cast<const VT*>(p);
        const S* q = reinterpret_cast<const S*>(&v);
#pragma unroll
        for (int t = 0; t < V; ++t) dst[t] = q[t];
    };
    // row j of x as V values plus the points left and right of the vector (zeros beyond the grid)
    auto load_row = [&](int j, S* dst, S& l, S& r) {
        if (j >= 0 && j < n1) {
            vld(X + (long long)j * n0 + c0, dst);
            l = c0 > 0 ? X[(long long)j * n0 + c0 - 1] : S(0);
            r = c0 + V < n0 ? X[(long long)j * n0 + c0 + V] : S(0);
        } else {
#pragma unroll
            for (int t = 0; t < V; ++t) dst[t] = S(0);
            l = r = S(0);
        }
    };
    S sr[V], pr[V], nr[V], sl = S(0), srr = S(0), pl = S(0), prr = S(0), nl = S(0), nrr = S(0);
    if (MODE != 1) {
        load_row(j0 - 1, sr, sl, srr);
        load_row(j0, pr, pl, prr);
    }
    for (int j = j0; j < j1; ++j) {
        if (MODE != 1) load_row(j + 1, nr, nl, nrr);
        const long long p = (long long)j * n0 + c0;
        S bq[V], ctr[V], res[V];
        vld(Bp + p, bq);
        vld(op.sten + 4 * nx + p, ctr);
        if (MODE == 1) {
#pragma unroll
            for (int t = 0; t < V; ++t) res[t] = omega * bq[t] / ctr[t];
        } else {
            S st[9][V];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if (k == 4) {
#pragma unroll
                    for (int t = 0; t < V; ++t) st[4][t] = ctr[t];
                } else {
                    vld(op.sten + (long long)k * nx + p, st[k]);
                }
            }
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const S s0 = t == 0 ? sl : sr[t - 1], s2 = t == V - 1 ? srr : sr[t + 1];
                const S p0 = t == 0 ? pl : pr[t - 1], p2 = t == V - 1 ? prr : pr[t + 1];
                const S n0v = t == 0 ? nl : nr[t - 1], n2 = t == V - 1 ? nrr : nr[t + 1];
                S acc = S(0);
                acc += st[0][t] * s0;
                acc += st[1][t] * sr[t];
                acc += st[2][t] * s2;
                acc += st[3][t] * p0;
                acc += st[4][t] * pr[t];
                acc += st[5][t] * p2;
                acc += st[6][t] * n0v;
                acc += st[7][t] * nr[t];
                acc += st[8][t] * n2;
                res[t] = MODE == 0 ? pr[t] + omega * (bq[t] - acc) / ctr[t] : bq[t] - acc;
            }
        }
        VT ov;
        S* oq = reinterpret_cast<S*>(&ov);
#pragma unroll
        for (int t = 0; t < V; ++t) oq[t] = res[t];
        *reinterpret_cast<VT*>(O + p) = ov;
        if (MODE != 1) {
#pragma unroll
            for (int t = 0; t < V; ++t) {
                sr[t] = pr[t];
                pr[t] = nr[t];
            }
            sl = pl;
            srr = prr;
            pl = nl;
            prr = nrr;
        }
    }
}

// Whether a level takes k_strip2d: 2D matrix-free with kappa = 1, unscaled storage, rows of whole
// 16-byte vectors that tile a 256-thread block, and 16-byte aligned rows.
template <class S>
inline bool strip_ok(const LevelOp<S>& op) {
    if constexpr (PT<S>::scaled) {
        return false;
    } else {
        constexpr int V = Vec16<S>::n;
        const int n0 = op.g.n0;
        return op.fine && op.g.d == 2 && op.faces.fx == nullptr && n0 % V == 0 && n0 / V <= kStripThreads &&
               kStripThreads % (n0 / V) == 0;
    }
}
// Whether a level takes k_strip2d_st: a 2D stored 9-point stencil, unscaled storage, rows of whole
// 16-byte vectors that tile a 256-thread block.
template <class S>
inline bool strip_st_ok(const LevelOp<S>& op) {
    if constexpr (PT<S>::scaled) {
        return false;
    } else {
        constexpr int V = Vec16<S>::n;
        const int n0 = op.g.n0;
        return !op.fine && op.g.d == 2 && op.ncoef == 9 && op.sten != nullptr && n0 % V == 0 &&
               n0 / V <= kStripThreads && kStripThreads % (n0 / V) == 0;
    }
}

// Rows per strip of k_strip2d_st: 8, halved (down to 2) while the batch gives fewer than 1024 blocks,
// so that a coarse level (few rows per item) still spreads over every SM; the shorter strips re-read
// more halo rows, from L1/L2.
template <class S>
inline int strip_st_rows(const LevelOp<S>& op, int B) {
    const int strips = kStripThreads / (op.g.n0 / Vec16<S>::n);
    int rs = kStripRows;
    while (rs > 2 && (long long)B * ((op.g.n1 + strips * rs - 1) / (strips * rs)) < 1024) rs /= 2;
    return rs;
}
template <class S>
inline dim3 strip_st_grid(const LevelOp<S>& op, int B, int rs) {
    const int strips = kStripThreads / (op.g.n0 / Vec16<S>::n);
    return dim3((unsigned)((op.g.n1 + strips * rs - 1) / (strips * rs)), (unsigned)B, 1);
}

template <class S>
inline dim3 strip_grid(const LevelOp<S>& op, int B) {
    const int tpr = op.g.n0 / Vec16<S>::n;
    const int rows_per_block = (kStripThreads / tpr) * kStripRows;
    return dim3((unsigned)((op.g.n1 + rows_per_block - 1) / rows_per_block), (unsigned)B, 1);
}

// ---------------------------------------------------------------------------
// Finest matrix-free level (sigma I + c K, kappa = 1, 2D or 3D) in 16-bit storage with per-row
// scales: a thread owns 8 consecutive columns of a row (one 16-byte vector), the threads of a row
// form a group of gs lanes within one warp (gs = the power of two >= n0 / 8), so the row's scale
// is a shuffle reduction over the group and no block barrier is needed.  MODE 0: damped Jacobi
// x + omega (b - A x) / a_PP; MODE 1: from x = 0; MODE 2: residual b - A x.  Same arithmetic as
// level_apply_k and the same scale rule as pt_store.  Block 256 threads (256 / gs rows); grid
// (ceil(R / rows per block), items).
// ---------------------------------------------------------------------------
constexpr int kVecThreads = 256;

template <class S>
__device__ __forceinline__ void vec8_load(const S* p, float sc, float* out) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const S* q = reinterpret_cast<const S*>(&v);
#pragma unroll
    for (int t = 0; t < 8; ++t) out[t] = PT<S>::ld(q[t]) * sc;
}

template <class S, int MODE>
__global__ void __launch_bounds__(kVecThreads) k_vec16(LevelOp<S> op, int gs, int B, const int* active, Vec<S> xin,
                                                       Vec<S> bv, Vec<S> out, float omega) {
    pdl_prologue();
    static_assert(PT<S>::scaled, "16-bit storage only");
    const Geo g = op.g;
    const int b = blockIdx.y;
    if (b >= B || (active && !active[b])) return;
    const int n0 = g.n0, tpr = n0 / 8;
    const int lane = threadIdx.x & 31, grp = lane / gs, gl = lane - grp * gs;
    const int rows_per_warp = 32 / gs;
    const long long row = ((long long)blockIdx.x * (kVecThreads / 32) + (threadIdx.x >> 5)) * rows_per_warp + grp;
    const bool valid = row < g.R && gl < tpr;       // every lane of a row's group takes part in its reduction
    int j = 0, k = 0;
    if (row < g.R) row_jk(g, row, j, k);
    const int c0 = gl * 8;
    const long long base = (long long)b * bv.bs;    // the same item stride for x, b and out
    const S* X = MODE == 1 ? nullptr : xin.d + (long long)b * xin.bs;
    const float* XS = MODE == 1 ? nullptr : xin.sc + (long long)b * xin.bs / n0;
    const S* Bd = bv.d + base;
    const float* BS = bv.sc + base / n0;
    float res[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) res[t] = 0.f;
    if (valid) {
        const float hx2 = float(g.hx2), hy2 = float(g.hy2), hz2 = float(g.hz2);
        float kd = 2.f * hx2 + 2.f * hy2;
        if (g.d == 3) kd += 2.f * hz2;
        const float dg = float(op.sigma) + float(op.c) * kd;
        float bq[8];
        vec8_load(Bd + row * n0 + c0, BS[row], bq);
        if (MODE == 1) {
#pragma unroll
            for (int t = 0; t < 8; ++t) res[t] = omega * bq[t] / dg;
        } else {
            float P[8], Sv[8], Nv[8], Dv[8], Uv[8];
            vec8_load(X + row * n0 + c0, XS[row], P);
            if (j > 0) vec8_load(X + (row - 1) * n0 + c0, XS[row - 1], Sv);
            else for (int t = 0; t < 8; ++t) Sv[t] = 0.f;
            if (j + 1 < g.n1) vec8_load(X + (row + 1) * n0 + c0, XS[row + 1], Nv);
            else for (int t = 0; t < 8; ++t) Nv[t] = 0.f;
            if (g.d == 3) {
                if (k > 0) vec8_load(X + (row - g.n1) * n0 + c0, XS[row - g.n1], Dv);
                else for (int t = 0; t < 8; ++t) Dv[t] = 0.f;
                if (k + 1 < g.n2) vec8_load(X + (row + g.n1) * n0 + c0, XS[row + g.n1], Uv);
                else for (int t = 0; t < 8; ++t) Uv[t] = 0.f;
            }
            const float w = c0 > 0 ? PT<S>::ld(X[row * n0 + c0 - 1]) * XS[row] : 0.f;
            const float e = c0 + 8 < n0 ? PT<S>::ld(X[row * n0 + c0 + 8]) * XS[row] : 0.f;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const float uP = P[t], uW = t == 0 ? w : P[t - 1], uE = t == 7 ? e : P[t + 1];
                float K = hx2 * (2.f * uP - uW - uE) + hy2 * (2.f * uP - Sv[t] - Nv[t]);
                if (g.d == 3) K += hz2 * (2.f * uP - Dv[t] - Uv[t]);
                const float Au = float(op.sigma) * uP + float(op.c) * K;
                res[t] = MODE == 0 ? uP + omega * (bq[t] - Au) / dg : bq[t] - Au;
            }
        }
    }
    // the row's power-of-two scale: maximum over the row's group of lanes
    float m = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) m = fmaxf(m, fabsf(res[t]));
    for (int o = gs >> 1; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int ex = 0;
    float sc = 1.f, inv = 1.f;
    if (m > 0.f && m <= 3.0e38f) {
        frexpf(m, &ex);
        sc = ldexpf(1.f, ex - 14);
        inv = ldexpf(1.f, 14 - ex);
    }
    if (valid) {
        uint4 ov;
        S* oq = reinterpret_cast<S*>(&ov);
#pragma unroll
        for (int t = 0; t < 8; ++t) oq[t] = PT<S>::st(res[t] * inv);
        *reinterpret_cast<uint4*>(out.d + (long long)b * out.bs + row * n0 + c0) = ov;
        if (gl == 0) out.sc[(long long)b * out.bs / n0 + row] = sc;
    }
}

// Whether a level takes k_vec16: the matrix-free finest level with kappa = 1, 16-bit storage,
// rows of whole 16-byte vectors with at most 32 vectors per row.
template <class S>
inline bool vec16_ok(const LevelOp<S>& op) {
    if constexpr (!PT<S>::scaled) {
        return false;
    } else {
        const int n0 = op.g.n0;
        return op.fine && op.faces.fx == nullptr && n0 % 8 == 0 && n0 / 8 <= 32;
    }
}
inline int vec16_group(int n0) {
    int gs = 1;
    while (gs < n0 / 8) gs <<= 1;
    return gs;
}
template <class S>
inline dim3 vec16_grid(const LevelOp<S>& op, int B) {
    const int rows_per_block = (kVecThreads / 32) * (32 / vec16_group(op.g.n0));
    return dim3((unsigned)((op.g.R + rows_per_block - 1) / rows_per_block), (unsigned)B, 1);
}

// r = b - A x for unscaled storage, RPT rows per thread (as k_smooth_rows).
template <class S, int KIND, int RPT>
__global__ void __launch_bounds__(kPtMaxThreads) k_residual_rows(LevelOp<S> op, PtMap pm, int B, const int* active,
                                                                 Vec<S> xv, Vec<S> bv, Vec<S> rv) {
    pdl_prologue();
    using A = typename PT<S>::A;
    static_assert(!PT<S>::scaled, "unscaled storage only");
    const Geo g = op.g;
    const int b = blockIdx.y;
    if (b >= B || (active && !active[b])) return;
    const int c = threadIdx.x;
    if (c >= g.n0) return;
    const int r0 = blockIdx.x * pm.rpc * RPT + threadIdx.y;
    View<S> xx = view_of(xv, b, 0, g.n0);
    View<S> bb = view_of(bv, b, 0, g.n0);
    S* out = rv.d + (long long)b * rv.bs;
    A v[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i * pm.rpc;
        v[i] = A(0);
        if (row < g.R) {
            A Au, dg;
            level_apply_k<KIND>(op, xx, row, row, 0, c, Au, dg);
            v[i] = bb.at(row, c) - Au;
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i * pm.rpc;
        if (row < g.R) out[(long long)row * g.n0 + c] = PT<S>::st(v[i]);
    }
}

// r = b - A x
template <class S, int KIND = 0>
__global__ void __launch_bounds__(kPtMaxThreads) k_residual(LevelOp<S> op, PtMap pm, int B, const int* active, Vec<S> xv,
                                                   Vec<S> bv, Vec<S> rv) {
    pdl_prologue();
    using A = typename PT<S>::A;
    const Geo g = op.g;
    PtPos q = pt_pos(pm, B, g.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int j, k;
    row_jk(g, row, j, k);
    View<S> xx = view_of(xv, q.b, 0, g.n0);
    View<S> bb = view_of(bv, q.b, 0, g.n0);
    S* out; float* osc;
    row_store_ptrs(rv, q.b, 0, row, g.n0, out, osc);
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
        A Au, dg;
        level_apply_k<KIND>(op, xx, row, j, k, c, Au, dg);
        return bb.at(row, c) - Au;
    });
}

// bc = P^T r  (coarse row kernel; pm maps the coarse rows)
template <class S>
__global__ void __launch_bounds__(kPtMaxThreads) k_restrict(Geo gf, Geo gc, PtMap pm, int B, const int* active, Vec<S> rv,
                                                   Vec<S> bcv) {
    pdl_prologue();
    using A = typename PT<S>::A;
    PtPos q = pt_pos(pm, B, gc.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int J, Kc;
    row_jk(gc, row, J, Kc);
    View<S> rr = view_of(rv, q.b, 0, gf.n0);
    S* out; float* osc;
    row_store_ptrs(bcv, q.b, 0, row, gc.n0, out, osc);
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int I) -> A {
        A acc = A(0);
        const int zlo = gf.d == 3 ? -1 : 0, zhi = gf.d == 3 ? 1 : 0;
        for (int dz = zlo; dz <= zhi; ++dz) {
            int fk = gf.d == 3 ? 2 * Kc + 1 + dz : 0;
            if (fk < 0 || fk >= gf.n2) continue;
            A wz = dz == 0 ? A(1) : A(0.5);
            for (int dy = -1; dy <= 1; ++dy) {
                int fj = 2 * J + 1 + dy;
                if (fj < 0 || fj >= gf.n1) continue;
                A wy = dy == 0 ? A(1) : A(0.5);
                long long frow = fj + (long long)gf.n1 * fk;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    int fi = 2 * I + 1 + dx;
                    if (fi < 0 || fi >= gf.n0) continue;
                    A wx = dx == 0 ? A(1) : A(0.5);
                    acc += wx * wy * wz * rr.at(frow, fi);
                }
            }
        }
        return acc;
    });
}

// 1D interpolation stencil of fine 0-based index F: up to two coarse indices.
__device__ __forceinline__ int interp_1d(int F, int nc, int* J, float* wt) {
    int g = F + 1;  // 1-based
    if ((g & 1) == 0) {
        J[0] = g / 2 - 1;
        wt[0] = 1.f;
        return 1;
    }
    int m = 0;
    int j1 = (g - 1) / 2 - 1, j2 = (g + 1) / 2 - 1;
    if (j1 >= 0 && j1 < nc) { J[m] = j1; wt[m] = 0.5f; ++m; }
    if (j2 >= 0 && j2 < nc) { J[m] = j2; wt[m] = 0.5f; ++m; }
    return m;
}

// x_out = x_in + P xc  (fine row kernel); x_in.d == nullptr means 0.
template <class S>
__global__ void __launch_bounds__(kPtMaxThreads) k_prolong_add(Geo gf, Geo gc, PtMap pm, int B, const int* active,
                                                      Vec<S> xcv, Vec<S> xin, Vec<S> xout) {
    pdl_prologue();
    using A = typename PT<S>::A;
    PtPos q = pt_pos(pm, B, gf.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int j, k;
    row_jk(gf, row, j, k);
    View<S> xc = view_of(xcv, q.b, 0, gc.n0);
    const bool has_in = xin.d != nullptr;
    View<S> xi = has_in ? view_of(xin, q.b, 0, gf.n0) : View<S>{nullptr, nullptr, gf.n0};
    int Jy[2], Jz[2] = {0, 0};
    float wy[2], wz[2] = {1.f, 0.f};
    int my = interp_1d(j, gc.n1, Jy, wy);
    int mz = gf.d == 3 ? interp_1d(k, gc.n2, Jz, wz) : 1;
    S* out; float* osc;
    row_store_ptrs(xout, q.b, 0, row, gf.n0, out, osc);
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
        int Jx[2];
        float wx[2];
        int mx = interp_1d(c, gc.n0, Jx, wx);
        A acc = has_in ? xi.at(row, c) : A(0);
        for (int a = 0; a < mz; ++a)
            for (int bq = 0; bq < my; ++bq) {
                long long crow = Jy[bq] + (long long)gc.n1 * Jz[a];
                A wyz = A(wy[bq]) * A(wz[a]);
                for (int e = 0; e < mx; ++e) acc += wyz * A(wx[e]) * xc.at(crow, Jx[e]);
            }
        return acc;
    });
}

// k_prolong_add in 2D for unscaled storage, RPT rows per thread (as k_smooth_rows).
template <class S, int RPT>
__global__ void __launch_bounds__(kPtMaxThreads) k_prolong_add_rows(Geo gf, Geo gc, PtMap pm, int B, const int* active,
                                                                    Vec<S> xcv, Vec<S> xin, Vec<S> xout) {
    pdl_prologue();
    using A = typename PT<S>::A;
    static_assert(!PT<S>::scaled, "unscaled storage only");
    const int b = blockIdx.y;
    if (b >= B || (active && !active[b])) return;
    const int c = threadIdx.x;
    if (c >= gf.n0) return;
    const int r0 = blockIdx.x * pm.rpc * RPT + threadIdx.y;
    View<S> xc = view_of(xcv, b, 0, gc.n0);
    const bool has_in = xin.d != nullptr;
    View<S> xi = has_in ? view_of(xin, b, 0, gf.n0) : View<S>{nullptr, nullptr, gf.n0};
    S* out = xout.d + (long long)b * xout.bs;
    int Jx[2];
    float wx[2];
    const int mx = interp_1d(c, gc.n0, Jx, wx);
    A v[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i * pm.rpc;
        v[i] = A(0);
        if (row < gf.R) {
            int Jy[2];
            float wy[2];
            const int my = interp_1d(row, gc.n1, Jy, wy);
            A acc = has_in ? xi.at(row, c) : A(0);
            for (int bq = 0; bq < my; ++bq) {
                const A wyz = A(wy[bq]) * A(1.f);
                for (int e = 0; e < mx; ++e) acc += wyz * A(wx[e]) * xc.at(Jy[bq], Jx[e]);
            }
            v[i] = acc;
        }
    }
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i * pm.rpc;
        if (row < gf.R) out[(long long)row * gf.n0 + c] = PT<S>::st(v[i]);
    }
}

// x_out = xp + omega D^{-1} (b - A xp) with xp = x_in + P xc computed on the fly at
// the point and its stencil neighbours (prolongation fused with one sweep).
template <class S>
__global__ void __launch_bounds__(kPtMaxThreads) k_prolong_smooth(LevelOp<S> op, Geo gc, PtMap pm, int B,
                                                                  const int* active, Vec<S> xcv, Vec<S> xin,
                                                                  Vec<S> bv, Vec<S> xout, typename PT<S>::A omega) {
    pdl_prologue();
    using A = typename PT<S>::A;
    const Geo gf = op.g;
    PtPos q = pt_pos(pm, B, gf.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int j, k;
    row_jk(gf, row, j, k);
    View<S> xc = view_of(xcv, q.b, 0, gc.n0);
    View<S> bb = view_of(bv, q.b, 0, gf.n0);
    const bool has = xin.d != nullptr;
    View<S> xi = has ? view_of(xin, q.b, 0, gf.n0) : View<S>{nullptr, nullptr, gf.n0};
    auto xp = [&](long long rr, int cc) -> A {
        int jj, kk;
    row_jk(gf, rr, jj, kk);
        int Jx[2], Jy[2], Jz[2] = {0, 0};
        float wx[2], wy[2], wz[2] = {1.f, 0.f};
        int mx = interp_1d(cc, gc.n0, Jx, wx);
        int my = interp_1d(jj, gc.n1, Jy, wy);
        int mz = gf.d == 3 ? interp_1d(kk, gc.n2, Jz, wz) : 1;
        A acc = has ? xi.at(rr, cc) : A(0);
        for (int a = 0; a < mz; ++a)
            for (int bq = 0; bq < my; ++bq) {
                long long crow = Jy[bq] + (long long)gc.n1 * Jz[a];
                A wyz = A(wy[bq]) * A(wz[a]);
                for (int e = 0; e < mx; ++e) acc += wyz * A(wx[e]) * xc.at(crow, Jx[e]);
            }
        return acc;
    };
    S* out; float* osc;
    row_store_ptrs(xout, q.b, 0, row, gf.n0, out, osc);
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
        A Au, dg;
        level_apply_g(op, xp, row, j, k, c, Au, dg);
        return xp(row, c) + omega * (bb.at(row, c) - Au) / dg;
    });
}

// x = Dinv b at the coarsest level (Dinv dense, nc x nc, row-major, arithmetic type).
template <class S>
__global__ void __launch_bounds__(kPtMaxThreads) k_coarse_solve(Geo g, PtMap pm, int B, const int* active,
                                                       const typename PT<S>::A* Dinv, Vec<S> bv, Vec<S> xv) {
    pdl_prologue();
    using A = typename PT<S>::A;
    PtPos q = pt_pos(pm, B, g.R, active);
    if constexpr (!PT<S>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    View<S> bb = view_of(bv, q.b, 0, g.n0);
    S* out; float* osc;
    row_store_ptrs(xv, q.b, 0, row, g.n0, out, osc);
    const int nc = (int)g.nx;
    pt_store<S>(out, osc, pm, q.c0, q.valid, [&](int c) -> A {
        long long p = row * g.n0 + c;
        A acc = A(0);
        for (int qq = 0; qq < nc; ++qq) acc += Dinv[p * nc + qq] * bb.at(qq / g.n0, qq % g.n0);
        return acc;
    });
}

// ---------------------------------------------------------------------------
// Set-up (FP64): Galerkin coarse stencil A_c = P^T A P, one thread per coarse
// point.  The fine operator is either matrix-free FD (sigma I + c K) or a
// stored FP64 3^d stencil.
// ---------------------------------------------------------------------------
struct FineDesc {
    Geo g;
    int fine;
    double sigma, c;
    Faces<double> faces;
    const double* sten;
};

__device__ __forceinline__ int fine_row_entries(const FineDesc& fd, int fi, int fj, int fk, int* gi, int* gj,
                                                int* gk, double* val) {
    const Geo& g = fd.g;
    long long row = fj + (long long)g.n1 * fk;
    int m = 0;
    if (fd.fine) {
        // diagonal and the 2d face neighbours
        double dg;
        if (fd.faces.fx == nullptr) {
            dg = 2 * g.hx2 + 2 * g.hy2 + (g.d == 3 ? 2 * g.hz2 : 0.0);
        } else {
            long long fxi = row * (g.n0 + 1) + fi;
            long long fyi = ((long long)fk * (g.n1 + 1) + fj) * g.n0 + fi;
            dg = fd.faces.fx[fxi] + fd.faces.fx[fxi + 1] + fd.faces.fy[fyi] + fd.faces.fy[fyi + g.n0];
            if (g.d == 3) {
                long long fzi = ((long long)fk * g.n1 + fj) * g.n0 + fi;
                dg += fd.faces.fz[fzi] + fd.faces.fz[fzi + (long long)g.n1 * g.n0];
            }
        }
        gi[m] = fi; gj[m] = fj; gk[m] = fk; val[m] = fd.sigma + fd.c * dg; ++m;
        for (int a = 0; a < g.d; ++a)
            for (int sg = -1; sg <= 1; sg += 2) {
                int ii = fi + (a == 0 ? sg : 0), jj = fj + (a == 1 ? sg : 0), kk = fk + (a == 2 ? sg : 0);
                if (ii < 0 || ii >= g.n0 || jj < 0 || jj >= g.n1 || kk < 0 || kk >= g.n2) continue;
                double face;
                if (fd.faces.fx == nullptr) {
                    face = a == 0 ? g.hx2 : (a == 1 ? g.hy2 : g.hz2);
                } else if (a == 0) {
                    face = fd.faces.fx[row * (g.n0 + 1) + fi + (sg > 0 ? 1 : 0)];
                } else if (a == 1) {
                    face = fd.faces.fy[((long long)fk * (g.n1 + 1) + fj + (sg > 0 ? 1 : 0)) * g.n0 + fi];
                } else {
                    face = fd.faces.fz[((long long)(fk + (sg > 0 ? 1 : 0)) * g.n1 + fj) * g.n0 + fi];
                }
                gi[m] = ii; gj[m] = jj; gk[m] = kk; val[m] = -fd.c * face; ++m;
            }
        return m;
    }
    long long p = row * g.n0 + fi;
    const int zlo = g.d == 3 ? -1 : 0, zhi = g.d == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int ii = fi + dx, jj = fj + dy, kk = fk + dz;
                if (ii < 0 || ii >= g.n0 || jj < 0 || jj >= g.n1 || kk < 0 || kk >= g.n2) continue;
                int q = (dx + 1) + 3 * (dy + 1) + (g.d == 3 ? 9 * (dz + 1) : 0);
                double v = fd.sten[(long long)q * g.nx + p];
                if (v == 0.0) continue;
                gi[m] = ii; gj[m] = jj; gk[m] = kk; val[m] = v; ++m;
            }
    return m;
}

static __global__ void k_galerkin(FineDesc fd, Geo gc, double* out) {
    pdl_prologue();
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= gc.nx) return;
    const Geo& gf = fd.g;
    const int ncoef = gc.d == 3 ? 27 : 9;
    int I = (int)(p % gc.n0), J = (int)((p / gc.n0) % gc.n1), Kc = (int)(p / ((long long)gc.n0 * gc.n1));
    double acc[27];
    for (int q = 0; q < 27; ++q) acc[q] = 0.0;
    const int zlo = gf.d == 3 ? -1 : 0, zhi = gf.d == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int fk = gf.d == 3 ? 2 * Kc + 1 + dz : 0;
        if (fk < 0 || fk >= gf.n2) continue;
        double wz = dz == 0 ? 1.0 : 0.5;
        for (int dy = -1; dy <= 1; ++dy) {
            int fj = 2 * J + 1 + dy;
            if (fj < 0 || fj >= gf.n1) continue;
            double wy = dy == 0 ? 1.0 : 0.5;
            for (int dx = -1; dx <= 1; ++dx) {
                int fi = 2 * I + 1 + dx;
                if (fi < 0 || fi >= gf.n0) continue;
                double wf = (dx == 0 ? 1.0 : 0.5) * wy * wz;   // P[f, I]
                int gi[27], gj[27], gk[27];
                double val[27];
                int m = fine_row_entries(fd, fi, fj, fk, gi, gj, gk, val);
                for (int e = 0; e < m; ++e) {
                    int Jx[2], Jy[2], Jz[2] = {0, 0};
                    float wx[2], wy2[2], wz2[2] = {1.f, 0.f};
                    int mx = interp_1d(gi[e], gc.n0, Jx, wx);
                    int my = interp_1d(gj[e], gc.n1, Jy, wy2);
                    int mz = gc.d == 3 ? interp_1d(gk[e], gc.n2, Jz, wz2) : 1;
                    for (int a = 0; a < mz; ++a)
                        for (int bq = 0; bq < my; ++bq)
                            for (int cq = 0; cq < mx; ++cq) {
                                int ox = Jx[cq] - I, oy = Jy[bq] - J, oz = gc.d == 3 ? Jz[a] - Kc : 0;
                                int q = (ox + 1) + 3 * (oy + 1) + (gc.d == 3 ? 9 * (oz + 1) : 0);
                                acc[q] += wf * val[e] * (double)wx[cq] * (double)wy2[bq] * (double)wz2[a];
                            }
                }
            }
        }
    }
    for (int q = 0; q < ncoef; ++q) out[(long long)q * gc.nx + p] = acc[q];
}

// Q1: the fine-level operator M + c K as a stored FP64 3^d-point stencil.
static __global__ void k_q1_stencil(Geo g, Q1<double> q, double c, double* out) {
    pdl_prologue();
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.nx) return;
    const int zlo = g.d == 3 ? -1 : 0, zhi = g.d == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const double mx = q.m[0][dx + 1], my = q.m[1][dy + 1], mz = g.d == 3 ? q.m[2][dz + 1] : 1.0;
                const double kx = q.k[0][dx + 1], ky = q.k[1][dy + 1], kz = g.d == 3 ? q.k[2][dz + 1] : 0.0;
                double kc = kx * my * mz + mx * ky * mz;
                if (g.d == 3) kc += mx * my * kz;
                int qi = (dx + 1) + 3 * (dy + 1) + (g.d == 3 ? 9 * (dz + 1) : 0);
                out[(long long)qi * g.nx + p] = mx * my * mz + c * kc;
            }
}

// Dense matrix of the coarsest level from its FP64 description (fine or stencil).
static __global__ void k_dense_level(FineDesc fd, double* Adense) {
    pdl_prologue();
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const Geo& g = fd.g;
    if (p >= g.nx) return;
    int fi = (int)(p % g.n0), fj = (int)((p / g.n0) % g.n1), fk = (int)(p / ((long long)g.n0 * g.n1));
    int gi[27], gj[27], gk[27];
    double val[27];
    int m = fine_row_entries(fd, fi, fj, fk, gi, gj, gk, val);
    for (long long q = 0; q < g.nx; ++q) Adense[p * g.nx + q] = 0.0;
    for (int e = 0; e < m; ++e) {
        long long q = gi[e] + (long long)g.n0 * (gj[e] + (long long)g.n1 * gk[e]);
        Adense[p * g.nx + q] += val[e];
    }
}

// In-place Gauss--Jordan inverse (SPD input, no pivoting needed), one block.
static __global__ void __launch_bounds__(1024) k_gauss_jordan(double* A, double* Inv, int n, int* fail) {
    pdl_prologue();
    // one CTA; warps take rows, lanes take columns; the scaled pivot rows live in shared memory
    __shared__ double prow[kMaxCoarsest], pinvrow[kMaxCoarsest];
    __shared__ double piv;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = w; i < n; i += nw)
        for (int j = lane; j < n; j += 32) Inv[i * n + j] = i == j ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            piv = A[k * n + k];
            if (!(piv > 0.0)) *fail = 1;
        }
        __syncthreads();
        const double pinv = 1.0 / piv;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double a = A[k * n + j] * pinv, v = Inv[k * n + j] * pinv;
            A[k * n + j] = a;
            Inv[k * n + j] = v;
            prow[j] = a;
            pinvrow[j] = v;
        }
        __syncthreads();
        for (int i = w; i < n; i += nw) {
            if (i == k) continue;
            const double f = A[i * n + k];
            for (int j = lane; j < n; j += 32) {
                if (j != k) A[i * n + j] -= f * prow[j];
                Inv[i * n + j] -= f * pinvrow[j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (i != k) A[i * n + k] = 0.0;
        __syncthreads();
    }
}

// Per-component max |coef| (one block per component) and conversion to S.
static __global__ void k_stencil_absmax(const double* sten, long long nx, float* cmax) {
    pdl_prologue();
    int q = blockIdx.x;
    double m = 0.0;
    for (long long p = threadIdx.x; p < nx; p += blockDim.x) m = fmax(m, fabs(sten[(long long)q * nx + p]));
    __shared__ double sh[kBlock];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double mm = sh[0];
        float sc = 1.f;
        if (mm > 0.0) {
            int e;
            frexp(mm, &e);
            sc = ldexpf(1.f, e - 14);
        }
        cmax[q] = sc;
    }
}

template <class S>
__global__ void k_stencil_convert(const double* sten, long long nx, int ncoef, const float* sc, S* out) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ncoef) return;
    int q = (int)(i / nx);
    double v = sten[i];
    if constexpr (PT<S>::scaled) v /= (double)sc[q];
    out[i] = PT<S>::st((typename PT<S>::A)v);
}

template <class A>
__global__ void k_convert_dense(const double* in, A* out, long long n) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (A)in[i];
}

}  // namespace aao

namespace aao {

// ---------------------------------------------------------------------------
// Fused V-cycle tail: levels lc..L-1 of one batch item in one CTA, every level
// held on chip (x and b per level, arithmetic type A), Jacobi sweeps staged in
// registers, residual recomputed inside the restriction.  One launch replaces
// the ~7 launches per level of the level-by-level path.  Vectors that stay on
// chip are not rounded to the 16-bit storage format (that format is for data
// that travels through HBM).
// ---------------------------------------------------------------------------
constexpr int kTailPmax = 4;    // points per thread at level lc (kTailMaxPoints / 1024)
constexpr int kTailMaxPoints = 4096;         // batched V-cycles
constexpr int kTailMaxPointsSingle = 1024;   // single-item V-cycles (the Schur sweep)
constexpr long long kFuseMaxPoints = 1 << 20;   // fuse sweeps below this many points per launch

template <class SI> struct TailCtx {
    using A = typename PT<SI>::A;
    int lc, L;
    LevelOp<SI> op[kMaxLevels];
    int off[kMaxLevels];        // smem offset (A elements) of X_l; B_l and R_l follow
    int vec_bytes;              // bytes of all X_l, B_l
    int stage_from;             // levels >= stage_from (and >= 1) read their stencil from smem
    int sten_off[kMaxLevels];   // byte offset of a staged stencil (after the vectors)
    const A* Dinv;
    A omega;
    int nu1, nu2;
};

// The operator of tail level l, reading a staged stencil from shared memory.
template <class SI>
__device__ __forceinline__ LevelOp<SI> tail_op(const TailCtx<SI>& t, int l, const unsigned char* smem) {
    LevelOp<SI> op = t.op[l];
    if (l >= 1 && l >= t.stage_from) op.sten = reinterpret_cast<const SI*>(smem + t.sten_off[l]);
    return op;
}

// Damped-Jacobi sweeps of tail level l, ping-ponging between its two on-chip x
// buffers (one barrier per sweep); cur selects the buffer holding x.
template <class SI>
__device__ __forceinline__ void tail_smooth(const TailCtx<SI>& t, int l, typename PT<SI>::A* sm, int sweeps,
                                            bool zero_first, unsigned& curbits) {
    int cur = (curbits >> l) & 1u;
    using A = typename PT<SI>::A;
    const LevelOp<SI> op = tail_op(t, l, reinterpret_cast<const unsigned char*>(sm));
    const Geo& g = op.g;
    A* X0 = sm + t.off[l];
    const A* Bv = X0 + 2 * g.nx;
    const int nt = blockDim.x;
    for (int sw = 0; sw < sweeps; ++sw) {
        const bool zero = zero_first && sw == 0;
        const A* Xc = X0 + (long long)cur * g.nx;
        A* Xn = X0 + (long long)(1 - cur) * g.nx;
        View<A> xv{Xc, nullptr, g.n0};
        for (int p = threadIdx.x; p < g.nx; p += nt) {
            int c = p % g.n0;
            long long row = p / g.n0;
            int j, k;
    row_jk(g, row, j, k);
            if (zero) {
                Xn[p] = t.omega * Bv[p] / level_diag(op, row, j, k, c);
            } else {
                A Au, dg;
                level_apply(op, xv, row, j, k, c, Au, dg);
                Xn[p] = Xc[p] + t.omega * (Bv[p] - Au) / dg;
            }
        }
        cur = 1 - cur;
        __syncthreads();
    }
    curbits = (curbits & ~(1u << l)) | ((unsigned)cur << l);
}

template <class SI>
__global__ void __launch_bounds__(1024) k_vcycle_tail(TailCtx<SI> t, int B, const int* active, Vec<SI> bv,
                                                      Vec<SI> xin, Vec<SI> xout) {
    pdl_prologue();
    using A = typename PT<SI>::A;
    extern __shared__ __align__(16) unsigned char tail_smem[];
    A* sm = reinterpret_cast<A*>(tail_smem);
    const int b = blockIdx.x;
    if (b >= B || (active && !active[b])) return;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int lc = t.lc, L = t.L;
    // per level: X0, X1 (x ping-pong; the free one holds the residual), B
    unsigned cur = 0u;      // bit l: which of level l's two x buffers holds the iterate
    // copy the coarse stencils of levels >= stage_from into shared memory
    for (int l = t.stage_from; l < L; ++l) {
        if (l < 1) continue;
        const long long n = (long long)t.op[l].ncoef * t.op[l].g.nx;
        SI* dst = reinterpret_cast<SI*>(tail_smem + t.sten_off[l]);
        for (long long i = tid; i < n; i += nt) dst[i] = t.op[l].sten[i];
    }
    {
        const Geo& g = t.op[lc].g;
        A* X = sm + t.off[lc];
        A* Bv = X + 2 * g.nx;
        View<SI> bs = view_of(bv, b, 0, g.n0);
        const bool has = xin.d != nullptr;
        View<SI> xs = has ? view_of(xin, b, 0, g.n0) : View<SI>{nullptr, nullptr, g.n0};
        for (int p = tid; p < g.nx; p += nt) {
            int c = p % g.n0, row = p / g.n0;
            Bv[p] = bs.at(row, c);
            X[p] = has ? xs.at(row, c) : A(0);
        }
    }
    __syncthreads();
    bool xzero = xin.d == nullptr;
    for (int l = lc; l < L - 1; ++l) {
        const LevelOp<SI> op = tail_op(t, l, tail_smem);
        const Geo& gf = op.g;
        const Geo& gc = t.op[l + 1].g;
        if (t.nu1 > 0) {
            tail_smooth(t, l, sm, t.nu1, xzero, cur);
            xzero = false;
        }
        A* X0 = sm + t.off[l];
        const A* Xf = X0 + (long long)((cur >> (l)) & 1u) * gf.nx;
        A* Rf = X0 + (long long)(1 - ((cur >> (l)) & 1u)) * gf.nx;   // the free x buffer holds the residual
        const A* Bv = X0 + 2 * gf.nx;
        A* Xc = sm + t.off[l + 1];
        A* Bc = Xc + 2 * gc.nx;
        if (xzero) {
            for (int p = tid; p < gf.nx; p += nt) Rf[p] = Bv[p];
        } else {
            View<A> xv{Xf, nullptr, gf.n0};
            for (int p = tid; p < gf.nx; p += nt) {
                int c = p % gf.n0;
                long long row = p / gf.n0;
                int j, k;
    row_jk(gf, row, j, k);
                A Au, dg;
                level_apply(op, xv, row, j, k, c, Au, dg);
                Rf[p] = Bv[p] - Au;
            }
        }
        __syncthreads();
        for (int P = tid; P < gc.nx; P += nt) {
            int I = P % gc.n0;
            long long crow = P / gc.n0;
            int J, Kc;
    row_jk(gc, crow, J, Kc);
            A acc = A(0);
            const int zlo = gf.d == 3 ? -1 : 0, zhi = gf.d == 3 ? 1 : 0;
            for (int dz = zlo; dz <= zhi; ++dz) {
                int fk = gf.d == 3 ? 2 * Kc + 1 + dz : 0;
                if (fk < 0 || fk >= gf.n2) continue;
                A wz = dz == 0 ? A(1) : A(0.5);
                for (int dy = -1; dy <= 1; ++dy) {
                    int fj = 2 * J + 1 + dy;
                    if (fj < 0 || fj >= gf.n1) continue;
                    A wy = dy == 0 ? A(1) : A(0.5);
                    long long frow = fj + (long long)gf.n1 * fk;
                    for (int dx = -1; dx <= 1; ++dx) {
                        int fi = 2 * I + 1 + dx;
                        if (fi < 0 || fi >= gf.n0) continue;
                        A wx = dx == 0 ? A(1) : A(0.5);
                        acc += wx * wy * wz * Rf[frow * gf.n0 + fi];
                    }
                }
            }
            Bc[P] = acc;
            Xc[P] = A(0);      // coarse levels start from zero (buffer 0)
        }
        __syncthreads();
        xzero = true;
    }
    {
        const Geo& g = t.op[L - 1].g;
        A* X = sm + t.off[L - 1] + (long long)((cur >> (L - 1)) & 1u) * g.nx;
        const A* Bv = sm + t.off[L - 1] + 2 * g.nx;
        const int nc = (int)g.nx;
        for (int p = tid; p < nc; p += nt) {
            A acc = A(0);
            for (int q = 0; q < nc; ++q) acc += t.Dinv[(long long)p * nc + q] * Bv[q];
            X[p] = acc;
        }
    }
    __syncthreads();
    for (int l = L - 2; l >= lc; --l) {
        const Geo& gf = t.op[l].g;
        const Geo& gc = t.op[l + 1].g;
        A* X = sm + t.off[l] + (long long)((cur >> (l)) & 1u) * gf.nx;
        const A* Xc = sm + t.off[l + 1] + (long long)((cur >> (l + 1)) & 1u) * gc.nx;
        for (int p = tid; p < gf.nx; p += nt) {
            int c = p % gf.n0;
            long long row = p / gf.n0;
            int j, k;
    row_jk(gf, row, j, k);
            int Jx[2], Jy[2], Jz[2] = {0, 0};
            float wx[2], wy[2], wz[2] = {1.f, 0.f};
            int mx = interp_1d(c, gc.n0, Jx, wx);
            int my = interp_1d(j, gc.n1, Jy, wy);
            int mz = gf.d == 3 ? interp_1d(k, gc.n2, Jz, wz) : 1;
            A acc = X[p];
            for (int a = 0; a < mz; ++a)
                for (int q = 0; q < my; ++q)
                    for (int e = 0; e < mx; ++e)
                        acc += A(wz[a]) * A(wy[q]) * A(wx[e]) * Xc[(Jz[a] * (long long)gc.n1 + Jy[q]) * gc.n0 + Jx[e]];
            X[p] = acc;
        }
        __syncthreads();
        if (t.nu2 > 0) tail_smooth(t, l, sm, t.nu2, false, cur);
    }
    // write level lc
    {
        const Geo& g = t.op[lc].g;
        const A* X = sm + t.off[lc] + (long long)((cur >> (lc)) & 1u) * g.nx;
        const int w = tid >> 5, lane = tid & 31, nw = nt >> 5;
        for (long long row = w; row < g.R; row += nw) {
            SI* o;
            float* osc;
            row_store_ptrs(xout, b, 0, row, g.n0, o, osc);
            row_store<SI>(o, osc, g.n0, lane, [&](int c) -> A { return X[row * g.n0 + c]; });
        }
    }
}

// ---------------------------------------------------------------------------
// 2D specialisation of the fused tail: a 32 x 32 thread block maps (column,
// row) directly, stencils are the unrolled 9-point (stored) or 5-point
// (matrix-free fine level) forms.  Same levels, buffers and arithmetic as
// k_vcycle_tail; only the indexing work per point is smaller.
// ---------------------------------------------------------------------------
template <class SI>
__device__ __forceinline__ typename PT<SI>::A tail2d_apply(const LevelOp<SI>& op, const typename PT<SI>::A* X, int c,
                                                           int j, typename PT<SI>::A& diag) {
    using A = typename PT<SI>::A;
    const Geo& g = op.g;
    const int n0 = g.n0, n1 = g.n1;
    if (op.fine) {
        A Au, dg;
        View<A> xv{X, nullptr, n0};
        level_apply(op, xv, j, j, 0, c, Au, dg);
        diag = dg;
        return Au;
    }
    const long long p = (long long)j * n0 + c;
    A acc = A(0);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int jj = j + dy;
        if (jj < 0 || jj >= n1) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int cc = c + dx;
            if (cc < 0 || cc >= n0) continue;
            acc += sten_coef(op, (dx + 1) + 3 * (dy + 1), p) * X[jj * n0 + cc];
        }
    }
    diag = sten_coef(op, 4, p);
    return acc;
}

template <class SI>
__device__ __forceinline__ void tail2d_smooth(const TailCtx<SI>& t, int l, typename PT<SI>::A* sm, int sweeps,
                                              bool zero_first, unsigned& curbits) {
    int cur = (curbits >> l) & 1u;
    using A = typename PT<SI>::A;
    const LevelOp<SI> op = tail_op(t, l, reinterpret_cast<const unsigned char*>(sm));
    const Geo& g = op.g;
    A* X0 = sm + t.off[l];
    const A* Bv = X0 + 2 * g.nx;
    for (int sw = 0; sw < sweeps; ++sw) {
        const bool zero = zero_first && sw == 0;
        const A* Xc = X0 + (long long)cur * g.nx;
        A* Xn = X0 + (long long)(1 - cur) * g.nx;
        for (int j = threadIdx.y; j < g.n1; j += blockDim.y)
            for (int c = threadIdx.x; c < g.n0; c += blockDim.x) {
                const int p = j * g.n0 + c;
                if (zero) {
                    Xn[p] = t.omega * Bv[p] / level_diag(op, j, j, 0, c);
                } else {
                    A dg;
                    const A Au = tail2d_apply(op, Xc, c, j, dg);
                    Xn[p] = Xc[p] + t.omega * (Bv[p] - Au) / dg;
                }
            }
        cur = 1 - cur;
        __syncthreads();
    }
    curbits = (curbits & ~(1u << l)) | ((unsigned)cur << l);
}

template <class SI>
__global__ void __launch_bounds__(1024) k_vcycle_tail_2d(TailCtx<SI> t, int B, const int* active, Vec<SI> bv,
                                                         Vec<SI> xin, Vec<SI> xout) {
    pdl_prologue();
    using A = typename PT<SI>::A;
    extern __shared__ __align__(16) unsigned char tail_smem[];
    A* sm = reinterpret_cast<A*>(tail_smem);
    const int b = blockIdx.x;
    if (b >= B || (active && !active[b])) return;
    const int tx = threadIdx.x, ty = threadIdx.y, bx = blockDim.x, by = blockDim.y;
    const int tid = ty * bx + tx, nt = bx * by;
    const int lc = t.lc, L = t.L;
    unsigned cur = 0u;      // bit l: which of level l's two x buffers holds the iterate
    for (int l = t.stage_from; l < L; ++l) {
        if (l < 1) continue;
        const int n = t.op[l].ncoef * (int)t.op[l].g.nx;
        SI* dst = reinterpret_cast<SI*>(tail_smem + t.sten_off[l]);
        for (int i = tid; i < n; i += nt) dst[i] = t.op[l].sten[i];
    }
    {
        const Geo& g = t.op[lc].g;
        A* X = sm + t.off[lc];
        A* Bv = X + 2 * g.nx;
        View<SI> bs = view_of(bv, b, 0, g.n0);
        const bool has = xin.d != nullptr;
        View<SI> xs = has ? view_of(xin, b, 0, g.n0) : View<SI>{nullptr, nullptr, g.n0};
        for (int j = ty; j < g.n1; j += by)
            for (int c = tx; c < g.n0; c += bx) {
                const int p = j * g.n0 + c;
                Bv[p] = bs.at(j, c);
                X[p] = has ? xs.at(j, c) : A(0);
            }
    }
    __syncthreads();
    bool xzero = xin.d == nullptr;
    for (int l = lc; l < L - 1; ++l) {
        const LevelOp<SI> op = tail_op(t, l, tail_smem);
        const Geo& gf = op.g;
        const Geo& gc = t.op[l + 1].g;
        if (t.nu1 > 0) {
            tail2d_smooth(t, l, sm, t.nu1, xzero, cur);
            xzero = false;
        }
        A* X0 = sm + t.off[l];
        const A* Xf = X0 + (long long)((cur >> (l)) & 1u) * gf.nx;
        A* Rf = X0 + (long long)(1 - ((cur >> (l)) & 1u)) * gf.nx;
        const A* Bv = X0 + 2 * gf.nx;
        for (int j = ty; j < gf.n1; j += by)
            for (int c = tx; c < gf.n0; c += bx) {
                const int p = j * gf.n0 + c;
                if (xzero) {
                    Rf[p] = Bv[p];
                } else {
                    A dg;
                    Rf[p] = Bv[p] - tail2d_apply(op, Xf, c, j, dg);
                }
            }
        __syncthreads();
        A* Xc = sm + t.off[l + 1];
        A* Bc = Xc + 2 * gc.nx;
        for (int J = ty; J < gc.n1; J += by)
            for (int I = tx; I < gc.n0; I += bx) {
                A acc = A(0);
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    const int fj = 2 * J + 1 + dy;
                    if (fj < 0 || fj >= gf.n1) continue;
                    const A wy = dy == 0 ? A(1) : A(0.5);
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int fi = 2 * I + 1 + dx;
                        if (fi < 0 || fi >= gf.n0) continue;
                        const A wx = dx == 0 ? A(1) : A(0.5);
                        acc += wx * wy * Rf[fj * gf.n0 + fi];
                    }
                }
                Bc[J * gc.n0 + I] = acc;
                Xc[J * gc.n0 + I] = A(0);
            }
        __syncthreads();
        xzero = true;
    }
    {
        const Geo& g = t.op[L - 1].g;
        A* X = sm + t.off[L - 1] + (long long)((cur >> (L - 1)) & 1u) * g.nx;
        const A* Bv = sm + t.off[L - 1] + 2 * g.nx;
        const int nc = (int)g.nx;
        for (int p = tid; p < nc; p += nt) {
            A acc = A(0);
            for (int q = 0; q < nc; ++q) acc += t.Dinv[(long long)p * nc + q] * Bv[q];
            X[p] = acc;
        }
    }
    __syncthreads();
    for (int l = L - 2; l >= lc; --l) {
        const Geo& gf = t.op[l].g;
        const Geo& gc = t.op[l + 1].g;
        A* X = sm + t.off[l] + (long long)((cur >> (l)) & 1u) * gf.nx;
        const A* Xc = sm + t.off[l + 1] + (long long)((cur >> (l + 1)) & 1u) * gc.nx;
        for (int j = ty; j < gf.n1; j += by) {
            int Jy[2];
            float wy[2];
            const int my = interp_1d(j, gc.n1, Jy, wy);
            for (int c = tx; c < gf.n0; c += bx) {
                int Jx[2];
                float wx[2];
                const int mx = interp_1d(c, gc.n0, Jx, wx);
                A acc = X[j * gf.n0 + c];
                for (int q = 0; q < my; ++q)
                    for (int e = 0; e < mx; ++e) acc += A(wy[q]) * A(wx[e]) * Xc[Jy[q] * gc.n0 + Jx[e]];
                X[j * gf.n0 + c] = acc;
            }
        }
        __syncthreads();
        if (t.nu2 > 0) tail2d_smooth(t, l, sm, t.nu2, false, cur);
    }
    {
        const Geo& g = t.op[lc].g;
        const A* X = sm + t.off[lc] + (long long)((cur >> (lc)) & 1u) * g.nx;
        const int w = tid >> 5, lane = tid & 31, nw = nt >> 5;
        for (long long row = w; row < g.R; row += nw) {
            SI* o;
            float* osc;
            row_store_ptrs(xout, b, 0, row, g.n0, o, osc);
            row_store<SI>(o, osc, g.n0, lane, [&](int c) -> A { return X[row * g.n0 + c]; });
        }
    }
}

}  // namespace aao
