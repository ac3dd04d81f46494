// Cluster-resident multigrid for one 2D item (the Schur sweep's shifted
// solves (M + c_i K) x = b, Sec. 5: three V-cycles per stage solve).
//
// The V-cycles of one shifted solve are a chain of ~30 dependent grid-wide
// steps per cycle; as separate launches each step costs a launch latency.
// Here one thread-block cluster (up to 16 CTAs, one per SM) runs all cycles:
//   * every level above the coarsest is split by grid rows over the CTAs; a
//     CTA keeps its rows of x (two ping-pong buffers), b, the stored stencil
//     and the Jacobi weights in shared memory;
//   * x / b rows are stored with a zero column on each side and a ghost row
//     above and below the CTA's range, so stencils, restriction and
//     interpolation read without bounds tests (the zeros stand for the
//     Dirichlet boundary and add exact zeros);
//   * a step that writes a CTA's first or last row also stores that row into
//     the neighbouring CTA's ghost row (distributed shared memory, generic
//     addresses from `mapa`), so after the cluster barrier that ends the step
//     every read is local;
//   * the level-l partition follows the finest one: coarse row J belongs to
//     the CTA owning fine row 2J+1, so restriction and interpolation only ever
//     touch one row beyond a CTA's range;
//   * the coarsest level (at most a few hundred unknowns) is held whole by
//     every CTA: each CTA restricts its right-hand side from all CTAs'
//     residual rows, applies its own slice of rows of the dense inverse
//     (staged once per launch) and gathers the other slices after a cluster
//     barrier;
//   * the Jacobi weights omega / a_PP are staged once per launch, so a sweep
//     is x + w (b - A x) without a division.
// Operator applications, residuals, restriction and interpolation follow the
// level kernels in mg.cuh (same formulas and summation order); intermediate
// vectors stay on chip in the arithmetic type.
#pragma once

#include <type_traits>

#include "mg.cuh"

namespace aao {

constexpr int kClMax = 16;            // CTAs per cluster (16 needs the non-portable size)
constexpr int kClThreads = 512;
constexpr int kClMaxBatch = 32;       // batches of at most this many items run one cluster per item
constexpr int kClBatch8 = 8;          // batches of at least this many items take the 8-CTA plan
constexpr int kClPad = 4;             // columns before a row's first point (column -1 is the last of them) and
                                      // after its last (column n0 the first): rows start 16-byte aligned

template <class SI> struct ClCtx {
    using A = typename PT<SI>::A;
    int C, L, T;                          // cluster size, levels, T = L-1 (the replicated coarsest level)
    int cycles, nu1, nu2;
    A omega;
    A sigma, c;                           // level 0 (FD): sigma I + c K
    int fine0, has_faces;
    Geo g[kMaxLevels];
    unsigned magic[kMaxLevels];           // ceil(2^32 / n0_l): p / n0_l = umulhi(p, magic) for p*n0_l < 2^32
    int rlo[kMaxLevels][kClMax + 1];      // distributed level l: CTA r owns rows [rlo[l][r], rlo[l][r+1])
    int maxr[kMaxLevels];                 // rows per CTA in the shared-memory layout (n1 for l >= T)
    int off[kMaxLevels];                  // A-element offset of level l's X0 | X1 | B, each (maxr+2) x (n0+2)
    int soff[kMaxLevels];                 // A-element offset of level l's staged stencil (9 x maxr*n0; -1: none)
    int woff[kMaxLevels];                 // A-element offset of omega / a_PP (maxr*n0; -1: coarsest)
    int fxoff, fyoff;                     // level 0 faces: maxr rows of n0+1 | maxr+1 rows of n0
    int cs[kClMax + 1];                   // coarsest rows [cs[r], cs[r+1]) of A_c^{-1} b are computed by CTA r
    int dinv_off;                         // A-element offset of this CTA's rows of A_c^{-1} (max rows * nc)
    int rowtab_off;                       // A-element offset (8-byte aligned) of the row table of level T-1
    const A* fx;
    const A* fy;
    const SI* sten[kMaxLevels];
    const float* sten_sc[kMaxLevels];
    const A* Dinv;
    // lean plans (a cluster of 8 for batches, where the full layout does not fit shared memory):
    int sten_global[kMaxLevels];          // 1: level l's stencil is read from global memory (L2), not staged
    int dinv_global;                      // 1: the rows of A_c^{-1} are read from global memory
    int w0_const;                         // 1: level 0's omega / a_PP is one scalar (FD, kappa = 1)
    int vec[kMaxLevels];                  // 1: level l's sweeps and residual take 16-byte vectors of points
    unsigned magicv[kMaxLevels];          // ceil(2^32 / (n0_l / points per vector))
};

// This CTA's share of a distributed level.
template <class A> struct ClLev {
    int a, nr;                // own rows [a, a + nr)
    A* pu[3];                 // ghost row below the range of the previous non-empty CTA (buffers X0, X1, B;
                              // first interior column), or nullptr
    A* pd[3];                 // ghost row above the range of the next non-empty CTA
};

// One level as a step sees it (built once per launch in shared memory; a step copies it to
// registers only in warps that have points of the level).
template <class A> struct ClL {
    int n0, n1, nr, a, ld, xs, cs;
    unsigned magic;
    int vec;                  // sweeps and residual by 16-byte vectors of points (cl_step_v)
    unsigned magicv;
    A* X;                     // buffer 0 at (row -1, column -1); buffer k at X + k*xs; (lr, c) at (lr+1)*ld + c+1
    const A* S;               // stored stencil (component stride cs = maxr*n0); nullptr: FD level 0 (or Sg)
    const void* Sg;           // stencil in global memory in the storage type (16-bit: times Ssc[k]), read by
    const float* Ssc;         //   the vector steps only; nullptr: S
    const A* W;               // omega / a_PP (index lr*n0 + c); nullptr: the scalar w0
    A w0;
    A *pu0, *pu1, *pu2;       // neighbours' ghost rows (see ClLev)
    A *pd0, *pd1, *pd2;
    A sigma, c, hx2, hy2;
    const A* fx;              // staged faces of the FD level (nullptr: kappa = 1)
    const A* fy;
    __device__ __forceinline__ A* pu(int k) const { return k == 0 ? pu0 : (k == 1 ? pu1 : pu2); }
    __device__ __forceinline__ A* pd(int k) const { return k == 0 ? pd0 : (k == 1 ? pd1 : pd2); }
    __device__ __forceinline__ A* el(int k, int lr, int col) const {
        return X + k * xs + (lr + 1) * ld + col + kClPad;
    }
    // store v at (lr, c) of buffer k and mirror the CTA's first / last row into the neighbours' ghost rows
    __device__ __forceinline__ void put(int k, int lr, int col, A v) const {
        *el(k, lr, col) = v;
        if (lr == 0) {
            A* q = pu(k);
            if (q) q[col] = v;
        }
        if (lr == nr - 1) {
            A* q = pd(k);
            if (q) q[col] = v;
        }
    }
};

template <class SI> struct ClShared {
    ClCtx<SI> t;
    ClLev<typename PT<SI>::A> lv[kMaxLevels];
    ClL<typename PT<SI>::A> lev[kMaxLevels];
    typename PT<SI>::A w0;    // level 0's omega / a_PP where it is one scalar (w0_const)
    int rank;
};

__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Index of this CTA's cluster in the grid: the batch item the cluster solves.
__device__ __forceinline__ int cl_item() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return (int)r;
}

__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Barrier after a step: the cluster for distributed levels, the CTA for replicated ones.
__device__ __forceinline__ void cl_step_sync(bool dist) {
    if (dist) cl_sync();
    else __syncthreads();
}

// Generic address of the same shared-memory location in CTA `rank` of the cluster.
template <class T> __device__ __forceinline__ T* cl_map(T* p, unsigned rank) {
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
    return reinterpret_cast<T*>(out);
}

__device__ __forceinline__ int cl_div(int p, unsigned magic) { return (int)__umulhi((unsigned)p, magic); }

template <class SI>
__device__ __forceinline__ ClL<typename PT<SI>::A> cl_level(const ClShared<SI>& S, typename PT<SI>::A* sm, int l) {
    using A = typename PT<SI>::A;
    const ClCtx<SI>& t = S.t;
    ClL<A> v;
    v.n0 = t.g[l].n0;
    v.n1 = t.g[l].n1;
    v.ld = v.n0 + 2 * kClPad;
    v.xs = (t.maxr[l] + 2) * v.ld;
    v.cs = t.maxr[l] * v.n0;
    v.magic = t.magic[l];
    v.vec = t.vec[l];
    v.magicv = t.magicv[l];
    const bool dist = l < t.T;
    v.a = dist ? S.lv[l].a : 0;
    v.nr = dist ? S.lv[l].nr : v.n1;
    v.X = sm + t.off[l];
    v.Sg = nullptr;
    v.Ssc = nullptr;
    if ((l == 0 && t.fine0) || (t.soff[l] < 0 && !t.sten_global[l])) {
        v.S = nullptr;
    } else if (t.sten_global[l]) {
        // the level's stencil in global memory: component stride n_x, rows from this CTA's first
        v.cs = (int)t.g[l].nx;
        if constexpr (std::is_same<SI, A>::value) {
            v.S = reinterpret_cast<const A*>(t.sten[l]) + (long long)v.a * v.n0;
        } else {
            v.S = nullptr;
            v.Sg = t.sten[l] + (long long)v.a * v.n0;
            v.Ssc = t.sten_sc[l];
        }
    } else {
        v.S = sm + t.soff[l];
    }
    v.W = t.woff[l] < 0 ? nullptr : sm + t.woff[l];
    v.w0 = S.w0;
    v.pu0 = dist ? S.lv[l].pu[0] : nullptr;
    v.pu1 = dist ? S.lv[l].pu[1] : nullptr;
    v.pu2 = dist ? S.lv[l].pu[2] : nullptr;
    v.pd0 = dist ? S.lv[l].pd[0] : nullptr;
    v.pd1 = dist ? S.lv[l].pd[1] : nullptr;
    v.pd2 = dist ? S.lv[l].pd[2] : nullptr;
    v.sigma = t.sigma;
    v.c = t.c;
    v.hx2 = A(t.g[0].hx2);
    v.hy2 = A(t.g[0].hy2);
    v.fx = t.has_faces ? sm + t.fxoff : nullptr;
    v.fy = t.has_faces ? sm + t.fyoff : nullptr;
    return v;
}

// (A x)_P at own point p = (lr, c); xm points at x(lr, c) in the padded layout.
template <class A>
__device__ __forceinline__ A cl_apply(const ClL<A>& v, int p, int lr, int c, const A* xm) {
    const int ld = v.ld;
    if (v.S == nullptr) {
        const A uP = xm[0], uW = xm[-1], uE = xm[1], uS = xm[-ld], uN = xm[ld];
        A K;
        if (v.fx == nullptr) {
            K = v.hx2 * (A(2) * uP - uW - uE) + v.hy2 * (A(2) * uP - uS - uN);
        } else {
            const A* fxr = v.fx + lr * (v.n0 + 1);
            const A* fyr = v.fy + lr * v.n0;
            K = fxr[c] * (uP - uW) + fxr[c + 1] * (uP - uE) + fyr[c] * (uP - uS) + fyr[c + v.n0] * (uP - uN);
        }
        return v.sigma * uP + v.c * K;
    }
    const A* Sp = v.S + p;
    const int cs = v.cs;
    A acc = A(0);
    acc += Sp[0 * cs] * xm[-ld - 1];
    acc += Sp[1 * cs] * xm[-ld];
    acc += Sp[2 * cs] * xm[-ld + 1];
    acc += Sp[3 * cs] * xm[-1];
    acc += Sp[4 * cs] * xm[0];
    acc += Sp[5 * cs] * xm[1];
    acc += Sp[6 * cs] * xm[ld - 1];
    acc += Sp[7 * cs] * xm[ld];
    acc += Sp[8 * cs] * xm[ld + 1];
    return acc;
}

// Damped Jacobi into buffer 1-kin: zero ? w b : x + w (b - A x), x = buffer kin.
template <class A>
__device__ __forceinline__ void cl_sweep(const ClL<A>& vin, int kin, bool zero, int tid, int nthr) {
    if (tid >= vin.nr * vin.n0) return;
    const ClL<A> v = vin;
    const int n0 = v.n0;
    const int np = v.nr * n0;
    for (int p = tid; p < np; p += nthr) {
        const int lr = cl_div(p, v.magic);
        const int c = p - lr * n0;
        const A bp = *v.el(2, lr, c);
        A val;
        const A wp = v.W ? v.W[p] : v.w0;
        if (zero) {
            val = wp * bp;
        } else {
            const A* xm = v.el(kin, lr, c);
            val = xm[0] + wp * (bp - cl_apply(v, p, lr, c, xm));
        }
        v.put(1 - kin, lr, c, val);
    }
}

// Residual b - A x of buffer kin into buffer 1 - kin.
template <class A>
__device__ __forceinline__ void cl_residual(const ClL<A>& vin, int kin, int tid, int nthr) {
    if (tid >= vin.nr * vin.n0) return;
    const ClL<A> v = vin;
    const int n0 = v.n0;
    const int np = v.nr * n0;
    for (int p = tid; p < np; p += nthr) {
        const int lr = cl_div(p, v.magic);
        const int c = p - lr * n0;
        const A* xm = v.el(kin, lr, c);
        v.put(1 - kin, lr, c, *v.el(2, lr, c) - cl_apply(v, p, lr, c, xm));
    }
}

// The points of a CTA's rows as 16-byte vectors (4 FP32 or 2 FP64 consecutive points of a row, rows
// 16-byte aligned by kClPad): one vector load per neighbouring row, scalar loads of the two points
// beside the vector, one vector store.  MODE 0: damped Jacobi into buffer 1 - kin; MODE 1: the same
// from x = 0 (w b); MODE 2: the residual b - A x into buffer 1 - kin.  Per point the operations of
// cl_sweep / cl_residual / cl_apply in the same order: the same values.  Levels planned with
// `vec`: n0 a multiple of the vector width, and a 9-point stored stencil or the FD level with
// kappa = 1.
template <class A> struct ClVec;
template <> struct ClVec<float> {
    using T = float4;
    static constexpr int n = 4;
};
template <> struct ClVec<double> {
    using T = double2;
    static constexpr int n = 2;
};

template <class A>
__device__ __forceinline__ void cl_vload(const A* p, A* out) {
    using VT = typename ClVec<A>::T;
    const VT v = *reinterpret_cast<const VT*>(p);
    const A* q = reinterpret_cast<const A*>(&v);
#pragma unroll
    for (int t = 0; t < ClVec<A>::n; ++t) out[t] = q[t];
}

template <class A>
__device__ __forceinline__ void cl_vstore(A* p, const A* in) {
    using VT = typename ClVec<A>::T;
    VT v;
    A* q = reinterpret_cast<A*>(&v);
#pragma unroll
    for (int t = 0; t < ClVec<A>::n; ++t) q[t] = in[t];
    *reinterpret_cast<VT*>(p) = v;
}

template <int MODE, class SI, class A>
__device__ __forceinline__ void cl_step_v(const ClL<A>& vin, int kin, int tid, int nthr) {
    constexpr int VN = ClVec<A>::n;
    const int nv = vin.n0 / VN;
    if (tid >= vin.nr * nv) return;
    const ClL<A> v = vin;
    const int np = v.nr * nv, ld = v.ld, kout = 1 - kin;
    for (int q = tid; q < np; q += nthr) {
        const int lr = cl_div(q, v.magicv);
        const int c = (q - lr * nv) * VN;
        const int p = lr * v.n0 + c;
        A b[VN], w[VN], out[VN];
        cl_vload(v.el(2, lr, c), b);
        if (MODE != 2) {
            if (v.W) {
                cl_vload(v.W + p, w);
            } else {
#pragma unroll
                for (int t = 0; t < VN; ++t) w[t] = v.w0;
            }
        }
        if (MODE == 1) {
#pragma unroll
            for (int t = 0; t < VN; ++t) out[t] = w[t] * b[t];
        } else {
            const A* xm = v.el(kin, lr, c);
            A xc[VN], xs[VN], xn[VN];
            cl_vload(xm, xc);
            cl_vload(xm - ld, xs);
            cl_vload(xm + ld, xn);
            const A xl = xm[-1], xr = xm[VN];
            A Au[VN];
            if (v.S == nullptr && v.Sg == nullptr) {
#pragma unroll
                for (int t = 0; t < VN; ++t) {
                    const A uP = xc[t], uW = t == 0 ? xl : xc[t - 1], uE = t == VN - 1 ? xr : xc[t + 1];
                    const A K = v.hx2 * (A(2) * uP - uW - uE) + v.hy2 * (A(2) * uP - xs[t] - xn[t]);
                    Au[t] = v.sigma * uP + v.c * K;
                }
            } else {
                const A sl = xm[-ld - 1], sr = xm[-ld + VN], nl = xm[ld - 1], nrt = xm[ld + VN];
                A S[9][VN];
                if constexpr (!std::is_same<SI, A>::value) {
                    if (v.Sg) {
                        // 16-bit storage in global memory: VN values (8 bytes) per component, times its scale
                        const SI* g = reinterpret_cast<const SI*>(v.Sg) + p;
#pragma unroll
                        for (int k = 0; k < 9; ++k) {
                            const uint2 raw = *reinterpret_cast<const uint2*>(g + (long long)k * v.cs);
                            const SI* e = reinterpret_cast<const SI*>(&raw);
#pragma unroll
                            for (int t = 0; t < VN; ++t) S[k][t] = PT<SI>::ld(e[t]) * v.Ssc[k];
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 9; ++k) cl_vload(v.S + (long long)k * v.cs + p, S[k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 9; ++k) cl_vload(v.S + (long long)k * v.cs + p, S[k]);
                }
#pragma unroll
                for (int t = 0; t < VN; ++t) {
                    const A sW = t == 0 ? sl : xs[t - 1], sE = t == VN - 1 ? sr : xs[t + 1];
                    const A uW = t == 0 ? xl : xc[t - 1], uE = t == VN - 1 ? xr : xc[t + 1];
                    const A nW = t == 0 ? nl : xn[t - 1], nE = t == VN - 1 ? nrt : xn[t + 1];
                    A acc = A(0);
                    acc += S[0][t] * sW;
                    acc += S[1][t] * xs[t];
                    acc += S[2][t] * sE;
                    acc += S[3][t] * uW;
                    acc += S[4][t] * xc[t];
                    acc += S[5][t] * uE;
                    acc += S[6][t] * nW;
                    acc += S[7][t] * xn[t];
                    acc += S[8][t] * nE;
                    Au[t] = acc;
                }
            }
#pragma unroll
            for (int t = 0; t < VN; ++t) out[t] = MODE == 0 ? xc[t] + w[t] * (b[t] - Au[t]) : b[t] - Au[t];
        }
        cl_vstore(v.el(kout, lr, c), out);
        if (lr == 0) {
            A* u = v.pu(kout);
            if (u) cl_vstore(u + c, out);
        }
        if (lr == v.nr - 1) {
            A* d = v.pd(kout);
            if (d) cl_vstore(d + c, out);
        }
    }
}

// Sweep or residual of one level: vectors where planned, else point by point.
template <class SI, class A>
__device__ __forceinline__ void cl_sweep_any(const ClL<A>& v, int kin, bool zero, int tid, int nthr) {
    if (v.vec) {
        if (zero) cl_step_v<1, SI>(v, kin, tid, nthr);
        else cl_step_v<0, SI>(v, kin, tid, nthr);
    } else {
        cl_sweep(v, kin, zero, tid, nthr);
    }
}

template <class SI, class A>
__device__ __forceinline__ void cl_residual_any(const ClL<A>& v, int kin, int tid, int nthr) {
    if (v.vec) cl_step_v<2, SI>(v, kin, tid, nthr);
    else cl_residual(v, kin, tid, nthr);
}

// b_c = P^T r (r = buffer kr of the fine level f) on the coarse rows this CTA computes.
// any_row: the coarse level is the replicated coarsest; fine rows come from rowtab (row i of
// buffer 0, first interior column, in the CTA that owns it).
template <class A>
__device__ __forceinline__ void cl_restrict(const ClL<A>& fin, const ClL<A>& cvin, int kr, bool any_row,
                                            const A* const* rowtab, int tid, int nthr) {
    if (tid >= cvin.nr * cvin.n0) return;
    const ClL<A> f = fin, cv = cvin;
    const int n0c = cv.n0;
    const int np = cv.nr * n0c;
    for (int p = tid; p < np; p += nthr) {
        const int lr = cl_div(p, cv.magic);
        const int I = p - lr * n0c;
        const int J = cv.a + lr;
        A acc = A(0);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int fj = 2 * J + 1 + dy;
            const A wy = dy == 0 ? A(1) : A(0.5);
            const A* row;
            if (any_row) {
                if (fj < 0 || fj >= f.n1) continue;
                row = rowtab[fj] + kr * f.xs;
            } else {
                row = f.el(kr, fj - f.a, 0);          // own or ghost row (zero beyond the boundary)
            }
            const int fi = 2 * I + 1;
            acc += A(0.5) * wy * row[fi - 1];
            acc += A(1) * wy * row[fi];
            acc += A(0.5) * wy * row[fi + 1];        // the zero column when fi + 1 == n0
        }
        cv.put(2, lr, I, acc);
    }
}

// 1D interpolation of fine index F: injection from coarse j0, or the average of j0 and j1
// (index -1 or nc: the zero ghost row / column at the boundary).
__device__ __forceinline__ void cl_interp(int F, int& j0, int& j1, bool& inj) {
    const int g = F + 1;                 // 1-based; coarse j sits at fine 2(j+1)
    inj = (g & 1) == 0;
    if (inj) {
        j0 = g / 2 - 1;
        j1 = j0;
    } else {
        j0 = (g - 1) / 2 - 1;
        j1 = (g + 1) / 2 - 1;
    }
}

// x_f (buffer kx) += P x_c (buffer kc) on the fine rows this CTA computes.
template <class A>
__device__ __forceinline__ void cl_prolong(const ClL<A>& fin, const ClL<A>& cvin, int kx, int kc, int tid, int nthr) {
    if (tid >= fin.nr * fin.n0) return;
    const ClL<A> f = fin, cv = cvin;
    const int n0 = f.n0;
    const int np = f.nr * n0;
    for (int p = tid; p < np; p += nthr) {
        const int lr = cl_div(p, f.magic);
        const int c = p - lr * n0;
        int y0, y1, x0, x1;
        bool yi, xi;
        cl_interp(f.a + lr, y0, y1, yi);
        cl_interp(c, x0, x1, xi);
        // injection in a direction: one coarse index, the second term gets weight 0
        const A wy = yi ? A(1) : A(0.5), wx = xi ? A(1) : A(0.5);
        const A w00 = wy * wx, w01 = xi ? A(0) : w00, w10 = yi ? A(0) : w00, w11 = (xi || yi) ? A(0) : w00;
        const A* r0 = cv.el(kc, y0 - cv.a, 0);
        const A* r1 = cv.el(kc, y1 - cv.a, 0);
        A acc = *f.el(kx, lr, c);
        acc += w00 * r0[x0];
        acc += w01 * r0[x1];
        acc += w10 * r1[x0];
        acc += w11 * r1[x1];
        f.put(kx, lr, c, acc);
    }
}

// xh = x_f (buffer kx) + P x_c (buffer kc) into buffer kout for this CTA's rows and its two ghost
// rows (rows outside the grid stay zero): the first post-smoothing sweep then reads xh without a
// cluster barrier, because each CTA computes its own ghost rows from its ghost rows of x_f and x_c.
// With kout == kx every element is read and written by the same thread.
template <class A>
__device__ __forceinline__ void cl_prolong_ext(const ClL<A>& fin, const ClL<A>& cvin, int kx, int kc, int kout,
                                               int tid, int nthr) {
    if (fin.nr == 0 || tid >= (fin.nr + 2) * fin.n0) return;
    const ClL<A> f = fin, cv = cvin;
    const int n0 = f.n0;
    const int np = f.nr > 0 ? (f.nr + 2) * n0 : 0;
    for (int p = tid; p < np; p += nthr) {
        const int lr = cl_div(p, f.magic) - 1;
        const int c = p - (lr + 1) * n0;
        const int F = f.a + lr;
        if (F < 0 || F >= f.n1) continue;
        int y0, y1, x0, x1;
        bool yi, xi;
        cl_interp(F, y0, y1, yi);
        cl_interp(c, x0, x1, xi);
        const A wy = yi ? A(1) : A(0.5), wx = xi ? A(1) : A(0.5);
        const A w00 = wy * wx, w01 = xi ? A(0) : w00, w10 = yi ? A(0) : w00, w11 = (xi || yi) ? A(0) : w00;
        const A* r0 = cv.el(kc, y0 - cv.a, 0);
        const A* r1 = cv.el(kc, y1 - cv.a, 0);
        A acc = *f.el(kx, lr, c);
        acc += w00 * r0[x0];
        acc += w01 * r0[x1];
        acc += w10 * r1[x0];
        acc += w11 * r1[x1];
        *f.el(kout, lr, c) = acc;
    }
}

// cl_prolong_ext with 16-byte vectors of fine points (fine n0 a multiple of the vector width): one
// vector load and store of x_f, the three coarse values beside each vector from each coarse row;
// per point the operations of cl_prolong_ext in the same order.
template <class A>
__device__ __forceinline__ void cl_prolong_ext_v(const ClL<A>& fin, const ClL<A>& cvin, int kx, int kc, int kout,
                                                 int tid, int nthr) {
    constexpr int VN = ClVec<A>::n;
    const int nv = fin.n0 / VN;
    if (fin.nr == 0 || tid >= (fin.nr + 2) * nv) return;
    const ClL<A> f = fin, cv = cvin;
    const int np = (f.nr + 2) * nv;
    for (int q = tid; q < np; q += nthr) {
        const int lr = cl_div(q, f.magicv) - 1;
        const int c = (q - (lr + 1) * nv) * VN;
        const int F = f.a + lr;
        if (F < 0 || F >= f.n1) continue;
        int y0, y1;
        bool yi;
        cl_interp(F, y0, y1, yi);
        const A wy = yi ? A(1) : A(0.5);
        const A* r0 = cv.el(kc, y0 - cv.a, 0);
        const A* r1 = cv.el(kc, y1 - cv.a, 0);
        A xv[VN], out[VN];
        cl_vload(f.el(kx, lr, c), xv);
#pragma unroll
        for (int t = 0; t < VN; ++t) {
            int x0, x1;
            bool xi;
            cl_interp(c + t, x0, x1, xi);
            const A wx = xi ? A(1) : A(0.5);
            const A w00 = wy * wx, w01 = xi ? A(0) : w00, w10 = yi ? A(0) : w00, w11 = (xi || yi) ? A(0) : w00;
            A acc = xv[t];
            acc += w00 * r0[x0];
            acc += w01 * r0[x1];
            acc += w10 * r1[x0];
            acc += w11 * r1[x1];
            out[t] = acc;
        }
        cl_vstore(f.el(kout, lr, c), out);
    }
}

// cl_restrict from a distributed fine level into a distributed coarse one with 16-byte vectors of
// coarse points: each fine row contributes two vector loads and one scalar; per point the operations
// of cl_restrict in the same order.  Both levels' n0 must be multiples of the vector width (the fine
// rows are read as vectors: with an odd fine n0 the row stride n0 + 2 kClPad is odd).
template <class A>
__device__ __forceinline__ void cl_restrict_v(const ClL<A>& fin, const ClL<A>& cvin, int kr, int tid, int nthr) {
    constexpr int VN = ClVec<A>::n;
    const int nv = cvin.n0 / VN;
    if (tid >= cvin.nr * nv) return;
    const ClL<A> f = fin, cv = cvin;
    const int np = cv.nr * nv;
    for (int q = tid; q < np; q += nthr) {
        const int lr = cl_div(q, cv.magicv);
        const int I0 = (q - lr * nv) * VN;
        const int J = cv.a + lr;
        A acc[VN];
#pragma unroll
        for (int t = 0; t < VN; ++t) acc[t] = A(0);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int fj = 2 * J + 1 + dy;
            const A wy = dy == 0 ? A(1) : A(0.5);
            const A* row = f.el(kr, fj - f.a, 0) + 2 * I0;     // own or ghost row (zero beyond the boundary)
            A fv[2 * VN + 1];
            cl_vload(row, fv);
            cl_vload(row + VN, fv + VN);
            fv[2 * VN] = row[2 * VN];                          // the zero column when 2 (I0 + VN) == n0
#pragma unroll
            for (int t = 0; t < VN; ++t) {
                acc[t] += A(0.5) * wy * fv[2 * t];
                acc[t] += A(1) * wy * fv[2 * t + 1];
                acc[t] += A(0.5) * wy * fv[2 * t + 2];
            }
        }
        cl_vstore(cv.el(2, lr, I0), acc);
        if (lr == 0) {
            A* u = cv.pu(2);
            if (u) cl_vstore(u + I0, acc);
        }
        if (lr == cv.nr - 1) {
            A* d = cv.pd(2);
            if (d) cl_vstore(d + I0, acc);
        }
    }
}

// Asynchronous copy of 4 bytes global -> shared (no register round trip).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}

// Asynchronous copy of 16 bytes global -> shared (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}

// n floats global -> shared: 16-byte copies where both ends are 16-byte aligned and n is a multiple
// of 4, else 4-byte copies.
__device__ __forceinline__ void cl_copy_async(float* dst, const float* src, int n, int tid, int nthr) {
    if (((reinterpret_cast<unsigned long long>(dst) | reinterpret_cast<unsigned long long>(src)) & 15ULL) == 0 &&
        (n & 3) == 0) {
        for (int p = tid * 4; p < n; p += nthr * 4) cp_async16(dst + p, src + p);
    } else {
        for (int p = tid; p < n; p += nthr) cp_async4(dst + p, src + p);
    }
}

// Staging for FP32 storage: every copy (b with ghost rows, faces, this CTA's stencil rows and rows
// of the coarsest inverse) is issued asynchronously before one wait; the Jacobi weights follow
// from the staged data.  Same values as the register path.
template <class SI>
__device__ __forceinline__ void cl_stage_async(const ClCtx<SI>& t, int rank, int L, int T, float* sm, const Vec<SI>& bv,
                                               int item, int tid, int nthr) {
    const Geo& g = t.g[0];
    const int a = t.rlo[0][rank], nr = t.rlo[0][rank + 1] - a;
    const int ld0 = g.n0 + 2 * kClPad, xs0 = (t.maxr[0] + 2) * ld0;
    float* B0 = sm + t.off[0] + 2 * xs0;
    const float* bsrc = reinterpret_cast<const float*>(bv.d) + (long long)item * bv.bs;
    const bool b16 = (g.n0 & 3) == 0 && (reinterpret_cast<unsigned long long>(bsrc) & 15ULL) == 0;
    if (nr > 0 && b16) {
        // rows of 16-byte vectors (padded shared rows start aligned)
        const int nv = g.n0 / 4, nb0 = (nr + 2) * nv;
        for (int q = tid; q < nb0; q += nthr) {
            const int lr = cl_div(q, t.magicv[0]) - 1;
            const int row = a + lr, c = (q - (lr + 1) * nv) * 4;
            float* d = B0 + (lr + 1) * ld0 + c + kClPad;
            if (row >= 0 && row < g.n1) cp_async16(d, bsrc + (long long)row * g.n0 + c);
            else *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else if (nr > 0) {
        const int nb0 = (nr + 2) * g.n0;
        for (int p = tid; p < nb0; p += nthr) {
            const int lr = cl_div(p, t.magic[0]) - 1;
            const int row = a + lr, c = p - (lr + 1) * g.n0;
            if (row >= 0 && row < g.n1) cp_async4(B0 + (lr + 1) * ld0 + c + kClPad, bsrc + (long long)row * g.n0 + c);
            else B0[(lr + 1) * ld0 + c + kClPad] = 0.f;
        }
    }
    const int w = g.n0 + 1;
    if (t.fine0 && t.has_faces) {
        const int nfx = nr * w, nfy = (nr + 1) * g.n0;
        const float* fx = reinterpret_cast<const float*>(t.fx) + (long long)a * w;
        const float* fy = reinterpret_cast<const float*>(t.fy) + (long long)a * g.n0;
        for (int p = tid; p < nfx; p += nthr) cp_async4(sm + t.fxoff + p, fx + p);
        for (int p = tid; p < nfy; p += nthr) cp_async4(sm + t.fyoff + p, fy + p);
    }
    for (int l = t.fine0 ? 1 : 0; l < L - 1; ++l) {
        if (t.sten_global[l]) continue;
        const Geo& gl = t.g[l];
        const bool dist = l < T;
        const int al = dist ? t.rlo[l][rank] : 0;
        const int npl = dist ? (t.rlo[l][rank + 1] - al) * gl.n0 : (int)gl.nx;
        const int cs = t.maxr[l] * gl.n0;
        const float* src = reinterpret_cast<const float*>(t.sten[l]) + (long long)al * gl.n0;
        for (int q = 0; q < 9; ++q) cl_copy_async(sm + t.soff[l] + q * cs, src + (long long)q * gl.nx, npl, tid, nthr);
    }
    if (!t.dinv_global) {
        const int nc = (int)t.g[L - 1].nx;
        const int n = (t.cs[rank + 1] - t.cs[rank]) * nc;
        const float* src = reinterpret_cast<const float*>(t.Dinv) + (long long)t.cs[rank] * nc;
        cl_copy_async(sm + t.dinv_off, src, n, tid, nthr);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // Jacobi weights omega / a_PP from the staged faces / stencil centres
    if (t.fine0 && !t.w0_const) {
        const int np0 = nr * g.n0;
        for (int p = tid; p < np0; p += nthr) {
            float kd;
            if (t.has_faces) {
                const int lr = cl_div(p, t.magic[0]);
                const int c = p - lr * g.n0;
                const float* fxr = sm + t.fxoff + lr * w;
                const float* fyr = sm + t.fyoff + lr * g.n0;
                kd = fxr[c] + fxr[c + 1] + fyr[c] + fyr[c + g.n0];
            } else {
                kd = 2.f * (float)g.hx2 + 2.f * (float)g.hy2;
            }
            sm[t.woff[0] + p] = t.omega / (t.sigma + t.c * kd);
        }
    }
    for (int l = t.fine0 ? 1 : 0; l < L - 1; ++l) {
        const Geo& gl = t.g[l];
        const bool dist = l < T;
        const int al = dist ? t.rlo[l][rank] : 0;
        const int npl = dist ? (t.rlo[l][rank + 1] - al) * gl.n0 : (int)gl.nx;
        const int cs = t.maxr[l] * gl.n0;
        if (t.sten_global[l]) {
            const float* ctr = reinterpret_cast<const float*>(t.sten[l]) + 4 * gl.nx + (long long)al * gl.n0;
            for (int p = tid; p < npl; p += nthr) sm[t.woff[l] + p] = t.omega / ctr[p];
        } else {
            for (int p = tid; p < npl; p += nthr) sm[t.woff[l] + p] = t.omega / sm[t.soff[l] + 4 * cs + p];
        }
    }
}

// All mg_cycles V-cycles of (M + c K) x = b, b and x in global memory: cluster k of the grid solves
// batch item k (grid = C x items CTAs; clusters never wait on one another).
template <class SI>
__global__ void __launch_bounds__(kClThreads, 1) k_cluster_mg(const ClCtx<SI>* __restrict__ ctx, const int* active,
                                                              Vec<SI> bv, Vec<SI> xout) {
    pdl_prologue();
    using A = typename PT<SI>::A;
    __shared__ ClShared<SI> S;
    extern __shared__ __align__(16) unsigned char cl_smem[];
    A* sm = reinterpret_cast<A*>(cl_smem);
    const int item = cl_item();               // one cluster per batch item
    if (active && !active[item]) return;      // the same decision in every CTA of the cluster
    const int tid = threadIdx.x, nthr = blockDim.x;
    {
        const int* src = reinterpret_cast<const int*>(ctx);
        int* dst = reinterpret_cast<int*>(&S.t);
        for (int i = tid; i < (int)(sizeof(ClCtx<SI>) / sizeof(int)); i += nthr) dst[i] = src[i];
    }
    __syncthreads();
    const ClCtx<SI>& t = S.t;
    const int rank = (int)cl_rank();
    const int L = t.L, T = t.T;
    if (tid == 0) S.rank = rank;
    // zero the padding columns and ghost rows of every x / b buffer (interiors are written before
    // they are read; the zeros stand for the Dirichlet boundary)
    for (int l = 0; l < L; ++l) {
        const int ld = t.g[l].n0 + 2 * kClPad, rows = t.maxr[l] + 2, xs = rows * ld;
        const int nrl = l < T ? t.rlo[l][rank + 1] - t.rlo[l][rank] : t.g[l].n1;   // this CTA's rows
        A* base = sm + t.off[l];
        const int nedge = 2 * ld + 2 * rows;          // ghost rows -1 and nrl, two padding columns
        for (int i = tid; i < 3 * nedge; i += nthr) {
            const int k = i / nedge, e = i - k * nedge;
            int idx;
            if (e < ld) idx = e;                                  // ghost row -1
            else if (e < 2 * ld) idx = (nrl + 1) * ld + e - ld;   // ghost row nrl
            else if (e < 2 * ld + rows) idx = (e - 2 * ld) * ld + kClPad - 1;          // column -1
            else idx = (e - 2 * ld - rows) * ld + kClPad + t.g[l].n0;                 // column n0
            base[k * xs + idx] = A(0);
        }
    }
    if (tid < T) {
        const int l = tid;
        ClLev<A>& v = S.lv[l];
        v.a = t.rlo[l][rank];
        v.nr = t.rlo[l][rank + 1] - v.a;
        int pr = rank - 1;
        while (pr >= 0 && t.rlo[l][pr + 1] == t.rlo[l][pr]) --pr;
        int nx = rank + 1;
        while (nx < t.C && t.rlo[l][nx + 1] == t.rlo[l][nx]) ++nx;
        const int ld = t.g[l].n0 + 2 * kClPad, xs = (t.maxr[l] + 2) * ld;
        for (int k = 0; k < 3; ++k) {
            v.pu[k] = nullptr;
            v.pd[k] = nullptr;
            if (v.nr > 0 && v.a > 0 && pr >= 0) {
                const int cnt = t.rlo[l][pr + 1] - t.rlo[l][pr];     // its ghost row below is row cnt
                v.pu[k] = cl_map(sm + t.off[l] + k * xs + (cnt + 1) * ld + kClPad, (unsigned)pr);
            }
            if (v.nr > 0 && v.a + v.nr < t.g[l].n1 && nx < t.C)
                v.pd[k] = cl_map(sm + t.off[l] + k * xs + kClPad, (unsigned)nx);     // its ghost row -1
        }
    }
    // row table of level T-1 (the restriction into the coarsest level reads every row of it)
    const A** rowtab = reinterpret_cast<const A**>(sm + t.rowtab_off);
    {
        const int l = T - 1;
        const int ld = t.g[l].n0 + 2 * kClPad;
        for (int i = tid; i < t.g[l].n1; i += nthr) {
            int r = 0;
            while (r + 1 < t.C && t.rlo[l][r + 1] <= i) ++r;
            A* q = sm + t.off[l] + (i - t.rlo[l][r] + 1) * ld + kClPad;
            rowtab[i] = r == rank ? q : cl_map(q, (unsigned)r);
        }
    }
    if (tid == 0 && t.w0_const) {
        // the formula of the staged weights (FD, kappa = 1: the same at every point)
        const Geo& g = t.g[0];
        const A kd = A(2) * A(g.hx2) + A(2) * A(g.hy2);
        S.w0 = t.omega / (t.sigma + t.c * kd);
    }
    __syncthreads();
    if (tid < L) S.lev[tid] = cl_level(S, sm, tid);
    if constexpr (std::is_same<SI, float>::value && std::is_same<typename PT<SI>::A, float>::value) {
        cl_stage_async(t, rank, L, T, sm, bv, item, tid, nthr);
    } else {
        // ---- stage b, faces, stencils, Jacobi weights and this CTA's rows of the coarsest inverse
        // (loads from global memory are issued in groups before the shared-memory stores)
        {
            constexpr int U = 4;
            const Geo& g = t.g[0];
            const int a = t.rlo[0][rank], nr = t.rlo[0][rank + 1] - a;
            const int np0 = nr * g.n0, ld0 = g.n0 + 2 * kClPad, xs0 = (t.maxr[0] + 2) * ld0;
            View<SI> bs = view_of(bv, item, 0, g.n0);
            A* B0 = sm + t.off[0] + 2 * xs0;
            // rows a-1 .. a+nr of b (the ghost rows too: the residual of a zero guess is b)
            const int nb0 = nr > 0 ? (nr + 2) * g.n0 : 0;
            for (int p0 = tid; p0 < nb0; p0 += U * nthr) {
                A v[U];
    #pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * nthr;
                    const int lr = cl_div(p, t.magic[0]) - 1;
                    const int row = a + lr;
                    v[u] = p < nb0 && row >= 0 && row < g.n1 ? bs.at(row, p - (lr + 1) * g.n0) : A(0);
                }
    #pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = p0 + u * nthr;
                    const int lr = cl_div(p, t.magic[0]) - 1;
                    if (p < nb0) B0[(lr + 1) * ld0 + p - (lr + 1) * g.n0 + kClPad] = v[u];
                }
            }
            if (t.fine0 && !t.w0_const) {
                const int w = g.n0 + 1;
                if (t.has_faces) {
                    const int nfx = nr * w, nfy = (nr + 1) * g.n0;
                    const A* fx = t.fx + (long long)a * w;
                    const A* fy = t.fy + (long long)a * g.n0;
                    for (int p0 = tid; p0 < nfx; p0 += U * nthr) {
                        A v[U];
    #pragma unroll
                        for (int u = 0; u < U; ++u) v[u] = p0 + u * nthr < nfx ? fx[p0 + u * nthr] : A(0);
    #pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (p0 + u * nthr < nfx) sm[t.fxoff + p0 + u * nthr] = v[u];
                    }
                    for (int p0 = tid; p0 < nfy; p0 += U * nthr) {
                        A v[U];
    #pragma unroll
                        for (int u = 0; u < U; ++u) v[u] = p0 + u * nthr < nfy ? fy[p0 + u * nthr] : A(0);
    #pragma unroll
                        for (int u = 0; u < U; ++u)
                            if (p0 + u * nthr < nfy) sm[t.fyoff + p0 + u * nthr] = v[u];
                    }
                }
                for (int p0 = tid; p0 < np0; p0 += U * nthr) {
                    A kd[U];
    #pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int p = p0 + u * nthr;
                        const int lr = cl_div(p, t.magic[0]);
                        const int c = p - lr * g.n0;
                        if (t.has_faces && p < np0) {
                            const long long fxi = (long long)(a + lr) * w + c, fyi = (long long)(a + lr) * g.n0 + c;
                            kd[u] = t.fx[fxi] + t.fx[fxi + 1] + t.fy[fyi] + t.fy[fyi + g.n0];
                        } else {
                            kd[u] = A(2) * A(g.hx2) + A(2) * A(g.hy2);
                        }
                    }
    #pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (p0 + u * nthr < np0) sm[t.woff[0] + p0 + u * nthr] = t.omega / (t.sigma + t.c * kd[u]);
                }
            }
            for (int l = t.fine0 ? 1 : 0; l < L - 1; ++l) {
                const Geo& gl = t.g[l];
                const bool dist = l < T;
                const int al = dist ? t.rlo[l][rank] : 0;
                const int npl = dist ? (t.rlo[l][rank + 1] - al) * gl.n0 : (int)gl.nx;
                const int cs = t.maxr[l] * gl.n0;
                const SI* src = t.sten[l] + (long long)al * gl.n0;
                if (t.sten_global[l]) {
                    // read in place by the vector steps: only the Jacobi weights are staged
                    for (int p = tid; p < npl; p += nthr) {
                        A ctr = PT<SI>::ld(src[4 * gl.nx + p]);
                        if constexpr (PT<SI>::scaled) ctr *= t.sten_sc[l][4];
                        sm[t.woff[l] + p] = t.omega / ctr;
                    }
                    continue;
                }
                for (int p = tid; p < npl; p += nthr) {
                    A v[9];
    #pragma unroll
                    for (int q = 0; q < 9; ++q) v[q] = PT<SI>::ld(src[(long long)q * gl.nx + p]);
    #pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        if constexpr (PT<SI>::scaled) v[q] *= t.sten_sc[l][q];
                        sm[t.soff[l] + q * cs + p] = v[q];
                    }
                    sm[t.woff[l] + p] = t.omega / v[4];
                }
            }
            if (!t.dinv_global) {
                const int nc = (int)t.g[L - 1].nx;
                const int n = (t.cs[rank + 1] - t.cs[rank]) * nc;
                const A* src = t.Dinv + (long long)t.cs[rank] * nc;
                for (int p0 = tid; p0 < n; p0 += U * nthr) {
                    A v[U];
    #pragma unroll
                    for (int u = 0; u < U; ++u) v[u] = p0 + u * nthr < n ? src[p0 + u * nthr] : A(0);
    #pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (p0 + u * nthr < n) sm[t.dinv_off + p0 + u * nthr] = v[u];
                }
            }
        }
    }
    __syncthreads();
    cl_sync();     // every CTA of the cluster is resident and staged before any remote access
    unsigned cur = 0u;       // bit l: buffer of level l holding the iterate
    for (int cyc = 0; cyc < t.cycles; ++cyc) {
        bool zero = cyc == 0;
        // ---- down: distributed levels (l < T) step with cluster barriers, replicated ones with
        // block barriers
        for (int l = 0; l < L - 1; ++l) {
            const bool dist = l < T;
            const ClL<A>& f = S.lev[l];
            int k = (cur >> l) & 1u;
            for (int sw = 0; sw < t.nu1; ++sw) {
                cl_sweep_any<SI>(f, k, zero && sw == 0, tid, nthr);
                k ^= 1;
                cl_step_sync(dist);
            }
            int kr;
            if (zero && t.nu1 == 0) {
                // x = 0: the residual is b; clear x (own and ghost rows) for the interpolation later
                kr = 2;
                const int nz = f.nr > 0 ? (f.nr + 2) * f.n0 : 0;
                for (int p = tid; p < nz; p += nthr) {
                    const int lr = cl_div(p, f.magic) - 1;
                    *f.el(k, lr, p - (lr + 1) * f.n0) = A(0);
                }
                cl_step_sync(dist);                       // b rows were written by this level's restriction
            } else {
                cl_residual_any<SI>(f, k, tid, nthr);
                kr = k ^ 1;
                cl_step_sync(dist);
            }
            cur = (cur & ~(1u << l)) | ((unsigned)k << l);
            const ClL<A>& cv = S.lev[l + 1];
            // vector restriction: coarse points in vectors and the fine rows 16-byte aligned too
            if (dist && l + 1 < T && cv.vec && f.n0 % ClVec<A>::n == 0) cl_restrict_v(f, cv, kr, tid, nthr);
            else cl_restrict(f, cv, kr, dist && l + 1 >= T, rowtab, tid, nthr);
            __syncthreads();
            zero = true;
        }
        // ---- coarsest level, held whole by every CTA: x = A_c^{-1} b, this CTA's rows one warp
        // per row, then the other CTAs' rows gathered after a cluster barrier
        {
            const int l = L - 1;
            const ClL<A> v = S.lev[l];
            const int nc = v.n0 * v.n1;
            const int k = (cur >> l) & 1u;
            A* bvec = v.X + (1 - k) * v.xs;           // b of the coarsest level, unpadded copy
            for (int p = tid; p < nc; p += nthr) {
                const int lr = cl_div(p, v.magic);
                bvec[p] = *v.el(2, lr, p - lr * v.n0);
            }
            __syncthreads();
            const A* Di = t.dinv_global ? t.Dinv + (long long)t.cs[rank] * nc : sm + t.dinv_off;
            const int lo = t.cs[rank], hi = t.cs[rank + 1];
            const int w = tid >> 5, lane = tid & 31, nw = nthr >> 5;
            for (int p = lo + w; p < hi; p += nw) {
                const A* row = Di + (p - lo) * nc;
                A acc = A(0);
                for (int q = lane; q < nc; q += kWarp) acc += row[q] * bvec[q];
                acc = warp_sum(acc);
                if (lane == 0) {
                    const int lr = cl_div(p, v.magic);
                    *v.el(k, lr, p - lr * v.n0) = acc;
                }
            }
            cl_sync();
            for (int p = tid; p < nc; p += nthr) {
                if (p >= lo && p < hi) continue;
                int r = 0;
                while (r + 1 < t.C && t.cs[r + 1] <= p) ++r;
                const int lr = cl_div(p, v.magic);
                A* q = v.el(k, lr, p - lr * v.n0);
                *q = *cl_map(q, (unsigned)r);
            }
            __syncthreads();
        }
        // ---- up
        for (int l = L - 2; l >= 0; --l) {
            const bool dist = l < T;
            const ClL<A>& f = S.lev[l];
            const ClL<A>& cv = S.lev[l + 1];
            int k = (cur >> l) & 1u;
            const int kc = (cur >> (l + 1)) & 1u;
            if (t.nu2 > 0) {
                // x += P x_c in place on own and ghost rows (no remote store: every CTA computes its
                // ghost rows itself), then the first sweep into the other buffer; a neighbour's
                // stores of that sweep land in a buffer nobody reads during this step
                if (f.vec) cl_prolong_ext_v(f, cv, k, kc, k, tid, nthr);
                else cl_prolong_ext(f, cv, k, kc, k, tid, nthr);
                __syncthreads();
                for (int sw = 0; sw < t.nu2; ++sw) {
                    cl_sweep_any<SI>(f, k, false, tid, nthr);
                    k ^= 1;
                    cl_step_sync(dist);
                }
            } else {
                cl_prolong(f, cv, k, kc, tid, nthr);
                cl_step_sync(dist);
            }
            cur = (cur & ~(1u << l)) | ((unsigned)k << l);
        }
    }
    // ---- write this CTA's rows of x_0
    {
        const ClL<A> v = S.lev[0];
        const int k = cur & 1u;
        if constexpr (PT<SI>::scaled) {
            const int w = tid >> 5, lane = tid & 31, nw = nthr >> 5;
            for (int lr = w; lr < v.nr; lr += nw) {
                SI* o;
                float* osc;
                row_store_ptrs(xout, item, 0, v.a + lr, v.n0, o, osc);
                const A* X = v.el(k, lr, 0);
                row_store<SI>(o, osc, v.n0, lane, [&](int c) -> A { return X[c]; });
            }
        } else {
            SI* o = xout.d + (long long)item * xout.bs + (long long)v.a * v.n0;
            for (int p = tid; p < v.nr * v.n0; p += nthr) {
                const int lr = cl_div(p, v.magic);
                o[p] = PT<SI>::st(*v.el(k, lr, p - lr * v.n0));
            }
        }
    }
}

}  // namespace aao
