// Row kernels of the Krylov and stage pieces:
//   * batched reductions (norms, modified Gram--Schmidt steps) with a
//     deterministic last-block finish, one result per batch item;
//   * Givens update and Hessenberg back-substitution per batch item;
//   * basis writes, Z y combinations;
//   * Theta_hat application (Eq. discretized_system_stages) and the Rana
//     stage-sweep right-hand side;
//   * the Schur forward / backward substitution steps (Eq. AppSchur);
//   * the FP64 all-at-once matvec and its transpose (Eq. system_all_at_once_RK).
#pragma once

#include "common.cuh"

namespace aao {

// ---------------------------------------------------------------------------
// Reductions: grid (nchunk, B), block kBlock.  Every batch item b spans `rows`
// rows of n0 values; block x of item b takes rows x*8+w, x*8+w + nchunk*8, ...
// Partial sums are double; the last block of item b (arrival counter) adds
// them in chunk order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
struct Red {
    double* partials;     // B * nchunk
    unsigned int* count;  // B, zero between launches
    int nchunk;
};

__device__ __forceinline__ void block_finish(double v, int b, const Red& red, double* out, int do_sqrt) {
    __shared__ double sh[kWarpsPerBlock];
    __shared__ bool last;
    v = warp_sum(v);
    int w = threadIdx.x >> 5;
    if (lane_id() == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kWarpsPerBlock; ++i) t += sh[i];
        red.partials[(long long)b * red.nchunk + blockIdx.x] = t;
        __threadfence();
        unsigned int prev = atomicAdd(&red.count[b], 1u);
        last = (prev == (unsigned int)red.nchunk - 1);
    }
    __syncthreads();
    if (last) {            // the whole block sums the partials (fixed order: strided, warp, then warps)
        __threadfence();
        double t = 0.0;
        const volatile double* p = red.partials + (long long)b * red.nchunk;
        for (int i = threadIdx.x; i < red.nchunk; i += blockDim.x) t += p[i];
        t = warp_sum(t);
        if (lane_id() == 0) sh[w] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < kWarpsPerBlock; ++i) s += sh[i];
            *out = do_sqrt ? sqrt(s) : s;
            red.count[b] = 0;
        }
    }
}

// ||src_b|| for an unscaled source (double or float), rows of n0.  Work is
// split in 32-column segments (one per warp iteration) so that a single item
// still spreads over many warps.
template <class SR>
__global__ void __launch_bounds__(kBlock) k_norm(int n0, long long rows, int B, const int* active,
                                                 const SR* src, long long bs, Red red, double* out,
                                                 long long ostride) {
    pdl_prologue();
    int b = blockIdx.y;
    if (active && !active[b]) return;
    const SR* x = src + (long long)b * bs;
    const int w = threadIdx.x >> 5, lane = lane_id();
    const unsigned spr = (n0 + kWarp - 1) / kWarp;
    const unsigned nseg = (unsigned)(rows * spr);   // < 2^32 segments (checked on the host)
    SR acc = SR(0);
    for (unsigned g = blockIdx.x * kWarpsPerBlock + w; g < nseg; g += red.nchunk * kWarpsPerBlock) {
        const unsigned r = g / spr;
        int c = (int)(g - r * spr) * kWarp + lane;
        if (c < n0) {
            SR v = x[(long long)r * n0 + c];
            acc += v * v;
        }
    }
    block_finish((double)acc, b, red, out + (long long)b * ostride, 1);
}

// One modified Gram--Schmidt step on w (arithmetic type A, unscaled):
//   if Vp: w -= hp[b] * Vp;   then   out[b] = Vn . w   (or ||w|| when Vn is null).
template <class SV, class A>
__global__ void __launch_bounds__(kBlock) k_mgs(int n0, long long rows, int B, const int* active, A* wv,
                                                long long wbs, Vec<SV> Vp, const double* hp, Vec<SV> Vn,
                                                long long hstride, Red red, double* out) {
    pdl_prologue();
    int b = blockIdx.y;
    if (active && !active[b]) return;
    A* w = wv + (long long)b * wbs;
    const bool upd = Vp.d != nullptr, dot = Vn.d != nullptr;
    View<SV> vp = upd ? view_of(Vp, b, 0, n0) : View<SV>{nullptr, nullptr, n0};
    View<SV> vn = dot ? view_of(Vn, b, 0, n0) : View<SV>{nullptr, nullptr, n0};
    A h = upd ? (A)hp[(long long)b * hstride] : A(0);
    const int wi = threadIdx.x >> 5, lane = lane_id();
    const unsigned spr = (n0 + kWarp - 1) / kWarp;
    const unsigned nseg = (unsigned)(rows * spr);   // < 2^32 segments (checked on the host)
    A acc = A(0);
    for (unsigned g = blockIdx.x * kWarpsPerBlock + wi; g < nseg; g += red.nchunk * kWarpsPerBlock) {
        const unsigned r = g / spr;
        int c = (int)(g - r * spr) * kWarp + lane;
        if (c < n0) {
            long long i = (long long)r * n0 + c;
            A x = w[i];
            if (upd) {
                x -= h * vp.at(r, c);
                w[i] = x;
            }
            acc += dot ? vn.at(r, c) * x : x * x;
        }
    }
    block_finish((double)acc, b, red, out + (long long)b * hstride, dot ? 0 : 1);
}

// out_b = src_b / denom[b * dstride]  (any storage); inactive items skipped.
template <class SO, class SR>
__global__ void __launch_bounds__(kPtMaxThreads) k_scale_store(PtMap pm, int rows, int B, const int* active, const SR* src,
                                                      long long sbs, const double* denom, long long dstride,
                                                      Vec<SO> out) {
    pdl_prologue();
    using A = typename PT<SO>::A;
    PtPos q = pt_pos(pm, B, rows, active);
    if constexpr (!PT<SO>::scaled) {
        if (!q.valid) return;
    }
    const int n0 = pm.n0;
    const SR* x = src + (long long)q.b * sbs + q.row * n0;
    // the reciprocal in the arithmetic type: an FP64 division per thread is slow on this GPU
    A inv = (denom && q.valid) ? A(1) / A(denom[(long long)q.b * dstride]) : A(1);
    SO* o; float* osc;
    row_store_ptrs(out, q.b, 0, q.row, n0, o, osc);
    pt_store<SO>(o, osc, pm, q.c0, q.valid, [&](int c) -> A { return A(x[c]) * inv; });
}

// Read a stored vector back into an unscaled array.
template <class S, class SO>
__global__ void __launch_bounds__(kPtMaxThreads) k_load(PtMap pm, int rows, int B, Vec<S> in, SO* out, long long obs) {
    pdl_prologue();
    PtPos q = pt_pos(pm, B, rows, nullptr);
    if (!q.valid) return;
    const int n0 = pm.n0;
    View<S> v = view_of(in, q.b, 0, n0);
    SO* o = out + (long long)q.b * obs + q.row * n0;
    for (int c = q.c0; c < n0; c += pm.n0p) o[c] = (SO)v.at(q.row, c);
}

// ---------------------------------------------------------------------------
// Givens update of column k of every item's Hessenberg matrix (Algorithm 1's
// least-squares problem).  H[b] is (kmax+1) x kmax row-major, stride hs.
// done[b] is set when |g_{k+1}| <= tol*beta_ref[b], h_{k+1,k} == 0 or k == kmax-1.
// ---------------------------------------------------------------------------
static __global__ void k_givens(int B, int k, int kmax, double* H, long long hs, double* cs, double* sn, double* g,
                         const double* beta_ref, double tol, int* active, int* its, int* nonfinite,
                         double* resid_out) {
    pdl_prologue();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || !active[b]) return;
    double* h = H + (long long)b * hs;
    double* c_ = cs + (long long)b * kmax;
    double* s_ = sn + (long long)b * kmax;
    double* g_ = g + (long long)b * (kmax + 1);
    for (int i = 0; i < k; ++i) {
        double a = h[i * kmax + k], bb = h[(i + 1) * kmax + k];
        h[i * kmax + k] = c_[i] * a + s_[i] * bb;
        h[(i + 1) * kmax + k] = -s_[i] * a + c_[i] * bb;
    }
    double a = h[k * kmax + k], hk1 = h[(k + 1) * kmax + k];
    double den = hypot(a, hk1);
    double cc = 1.0, ss = 0.0;
    if (den != 0.0) {
        cc = a / den;
        ss = hk1 / den;
    }
    c_[k] = cc;
    s_[k] = ss;
    h[k * kmax + k] = den;
    g_[k + 1] = -ss * g_[k];
    g_[k] = cc * g_[k];
    // keep the unrotated h_{k+1,k} for the basis write (denominator)
    h[(k + 1) * kmax + k] = hk1;
    double res = fabs(g_[k + 1]);
    if (resid_out) resid_out[b] = res;
    its[b] = k + 1;
    if (!isfinite(res) || !isfinite(den)) {
        atomicExch(nonfinite, 1);
        active[b] = 0;
        return;
    }
    if (res <= tol * beta_ref[b] || hk1 == 0.0 || k == kmax - 1) active[b] = 0;
}

// Start of a batched inner solve: items with beta == 0 are done at once (z = 0).
static __global__ void k_inner_init(int B, int kmax, const double* beta, int* active, int* its, double* g, int* nonfinite) {
    pdl_prologue();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double bt = beta[b];
    if (!isfinite(bt)) atomicExch(nonfinite, 1);
    active[b] = (bt > 0.0 && isfinite(bt)) ? 1 : 0;
    its[b] = 0;
    for (int i = 0; i <= kmax; ++i) g[(long long)b * (kmax + 1) + i] = i == 0 ? bt : 0.0;
}

static __global__ void k_count_its(int B, const int* its, long long* count) {
    pdl_prologue();
    __shared__ long long sh[128];
    long long t = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) t += its[b];
    sh[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) a += sh[i];
        *count += a;
    }
}

// y = R^{-1} g (R the rotated upper triangle, its[b] columns), per item.
static __global__ void k_hess_solve(int B, int kmax, const double* H, long long hs, const double* g, const int* its,
                             double* y, int* breakdown) {
    pdl_prologue();
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double* h = H + (long long)b * hs;
    const double* g_ = g + (long long)b * (kmax + 1);
    double* y_ = y + (long long)b * kmax;
    int m = its[b];
    for (int i = m - 1; i >= 0; --i) {
        double t = g_[i];
        for (int j = i + 1; j < m; ++j) t -= h[i * kmax + j] * y_[j];
        double d = h[i * kmax + i];
        if (d == 0.0) {
            atomicExch(breakdown, 1);
            y_[i] = 0.0;
        } else {
            y_[i] = t / d;
        }
    }
    for (int i = m; i < kmax; ++i) y_[i] = 0.0;
}

// out_b (+)= sum_{k < its[b]} y[b][k] Z_k,b ; Z_k at Z0 shifted by k*zstride elements.
template <class SZ, class SO>
__global__ void __launch_bounds__(kPtMaxThreads) k_combine(PtMap pm, int rows, int B, Vec<SZ> Z0, long long zstride,
                                                  const double* y, int kmax, const int* its, SO* out, long long obs,
                                                  int accumulate) {
    pdl_prologue();
    PtPos q = pt_pos(pm, B, rows, nullptr);
    if (!q.valid) return;
    using A = typename PT<SZ>::A;
    const int n0 = pm.n0;
    const int m = its ? its[q.b] : kmax;
    SO* o = out + (long long)q.b * obs + q.row * n0;
    for (int c = q.c0; c < n0; c += pm.n0p) {
        A acc = accumulate ? A(o[c]) : A(0);
        for (int k = 0; k < m; ++k) {
            Vec<SZ> Zk = Z0;
            Zk.d += k * zstride;
            if constexpr (PT<SZ>::scaled) Zk.sc += (k * zstride) / n0;
            View<SZ> z = view_of(Zk, q.b, 0, n0);
            acc += (A)y[(long long)q.b * kmax + k] * z.at(q.row, c);
        }
        o[c] = (SO)acc;
    }
}

// ---------------------------------------------------------------------------
// Theta_hat z (Eq. discretized_system_stages with M = I):
//   w_i = z_i + tau sum_j coef[i*s + j] K z_j,  coef = A_RK (or A_RK^T).
// One warp per (item, spatial row); every stage of the row at once.
// ---------------------------------------------------------------------------
template <class SZ, class A>
__global__ void __launch_bounds__(kPtMaxThreads) k_theta(Geo g, PtMap pm, int B, const int* active, Vec<SZ> Z, A* wv,
                                                long long wbs, int s, const double* coef, A tau, SpaceOp<A> sop) {
    pdl_prologue();
    // tau a_ij in the arithmetic type, once per block (the products the per-point sum uses)
    __shared__ A tc[kMaxS * kMaxS];
    for (int t = threadIdx.y * blockDim.x + threadIdx.x; t < s * s; t += blockDim.x * blockDim.y)
        tc[t] = tau * (A)coef[t];
    __syncthreads();
    PtPos q = pt_pos(pm, B, g.R, active);
    if (!q.valid) return;
    const long long row = q.row;
    int j, k;
    row_jk(g, row, j, k);
    A* out = wv + (long long)q.b * wbs + row * g.n0;
    for (int c = q.c0; c < g.n0; c += pm.n0p) {
        A kz[kMaxS];
        for (int i = 0; i < s; ++i) {
            View<SZ> zi = view_of(Z, q.b, (long long)i * g.nx, g.n0);
            kz[i] = (A)op_K(zi, g, sop, row, j, k, c);
        }
        for (int i = 0; i < s; ++i) {
            View<SZ> zi = view_of(Z, q.b, (long long)i * g.nx, g.n0);
            A acc = (A)op_M(zi, g, sop, row, j, k, c);
            for (int jj = 0; jj < s; ++jj) acc += tc[i * s + jj] * kz[jj];
            out[(long long)i * g.nx + c] = acc;
        }
    }
}

// Rana stage-sweep right-hand side: out = V_stage - tau sum_j coef[j] K Z_j.
template <class SV, class SZ>
__global__ void __launch_bounds__(kPtMaxThreads) k_rana_rhs(Geo g, PtMap pm, int B, const int* active, Vec<SV> V, int stage,
                                                   Vec<SZ> Z, int s, const double* coef, typename PT<SZ>::A tau,
                                                   SpaceOp<typename PT<SZ>::A> sop, Vec<SZ> out) {
    pdl_prologue();
    using A = typename PT<SZ>::A;
    PtPos q = pt_pos(pm, B, g.R, active);
    if constexpr (!PT<SZ>::scaled) {
        if (!q.valid) return;
    }
    const long long row = q.row;
    int j, k;
    row_jk(g, row, j, k);
    View<SV> v = view_of(V, q.b, (long long)stage * g.nx, g.n0);
    SZ* o; float* osc;
    row_store_ptrs(out, q.b, 0, row, g.n0, o, osc);
    if (g.d == 2 && !sop.q1) {
        // fd_K for d = 2 with 32-bit indexing within the item (same arithmetic)
        const int r = (int)row, n0 = g.n0;
        pt_store<SZ>(o, osc, pm, q.c0, q.valid, [&](int c) -> A {
            A acc = (A)v.at(row, c);
            for (int jj = 0; jj < s; ++jj) {
                const double cf = coef[jj];
                if (cf != 0.0) {
                    View<SZ> zj = view_of(Z, q.b, (long long)jj * g.nx, n0);
                    const A uP = zj.at(r, c);
                    const A uW = c > 0 ? zj.at(r, c - 1) : A(0);
                    const A uE = c + 1 < n0 ? zj.at(r, c + 1) : A(0);
                    const A uS = j > 0 ? zj.at(r - 1, c) : A(0);
                    const A uN = j + 1 < g.n1 ? zj.at(r + 1, c) : A(0);
                    A K;
                    if (sop.faces.fx == nullptr) {
                        K = A(g.hx2) * (A(2) * uP - uW - uE) + A(g.hy2) * (A(2) * uP - uS - uN);
                    } else {
                        const int fxi = r * (n0 + 1) + c, fyi = j * n0 + c;
                        K = A(sop.faces.fx[fxi]) * (uP - uW) + A(sop.faces.fx[fxi + 1]) * (uP - uE) +
                            A(sop.faces.fy[fyi]) * (uP - uS) + A(sop.faces.fy[fyi + n0]) * (uP - uN);
                    }
                    acc -= tau * (A)cf * K;
                }
            }
            return acc;
        });
        return;
    }
    pt_store<SZ>(o, osc, pm, q.c0, q.valid, [&](int c) -> A {
        A acc = (A)v.at(row, c);
        for (int jj = 0; jj < s; ++jj) {
            const double cf = coef[jj];
            if (cf != 0.0) {
                View<SZ> zj = view_of(Z, q.b, (long long)jj * g.nx, g.n0);
                acc -= tau * (A)cf * (A)op_K(zj, g, sop, row, j, k, c);
            }
        }
        return acc;
    });
}

// ---------------------------------------------------------------------------
// Schur substitution pieces (Eq. AppSchur, FD: M = I).  The recurrence runs
// in arithmetic type A; z_v lives in the FP64 output vector.
// ---------------------------------------------------------------------------
// w_0 = r_{v,0}; w_{n+1} = r_{v,n+1} + tau sum_i b_i zV_{n,i};  z_{v,0} = w_0.
template <class A>
__global__ void k_schur_g(long long nx, int nt, int s, const double* r, const double* zV, const double* bw,
                          double tau, A* wbuf, double* zv0) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)(nt + 1) * nx;
    if (i >= tot) return;
    long long n = i / nx, p = i % nx;
    A v;
    if (n == 0) {
        v = (A)r[p];
        zv0[p] = (double)v;
    } else {
        A acc = A(0);
        const double* z = zV + (n - 1) * s * nx + p;
        for (int q = 0; q < s; ++q) acc += (A)bw[q] * (A)z[(long long)q * nx];
        v = (A)r[i] + (A)tau * acc;
    }
    wbuf[i] = v;
}

// Per-step state of the Schur substitution, in device memory so that one
// captured step can be replayed for every n: z (output vector), r (input
// vector) and the step index n.
struct StepPtrs {
    double* z;
    const double* r;
    int n;
};

static __global__ void k_step_set(StepPtrs* sp, double* z, const double* r, int n) {
    pdl_prologue();
    sp->z = z;
    sp->r = r;
    sp->n = n;
}

static __global__ void k_step_add(StepPtrs* sp, int d) {
    pdl_prologue(); sp->n += d; }

// t_i = K z_{v,n} for every stage i (the e (x) K z_{v,n} right-hand side).
template <class A>
__global__ void __launch_bounds__(kBlock) k_schur_rhs(Geo g, int s, const StepPtrs* sp, A* t, SpaceOp<A> sop) {
    pdl_prologue();
    long long row = gwarp();
    if (row >= g.R) return;
    int j, k;
    row_jk(g, row, j, k);
    View<double> z{sp->z + (long long)sp->n * g.nx, nullptr, g.n0};
    for (int c = lane_id(); c < g.n0; c += kWarp) {
        A v = (A)op_K(z, g, sop, row, j, k, c);
        for (int i = 0; i < s; ++i) t[(long long)i * g.nx + row * g.n0 + c] = v;
    }
}

// z_{v,n+1} = w_{n+1} + z_{v,n} - tau sum_i b_i q_i,  q = sum_k y_k Z_k (item 0).
template <class SZ, class A>
__global__ void __launch_bounds__(kBlock) k_schur_update(Geo g, int s, const A* wbuf, const StepPtrs* sp,
                                                         Vec<SZ> Z0, long long zstride, const double* y,
                                                         int kmax, const int* its, const double* bw,
                                                         double tau) {
    pdl_prologue();
    long long row = gwarp();
    if (row >= g.R) return;
    const int n = sp->n;
    const A* wn1 = wbuf + (long long)(n + 1) * g.nx;
    const double* zvn = sp->z + (long long)n * g.nx;
    double* zvn1 = sp->z + (long long)(n + 1) * g.nx;
    int m = its[0];
    A coef[kMaxInner * kMaxS];
    for (int k = 0; k < m; ++k)
        for (int i = 0; i < s; ++i) coef[k * s + i] = (A)(tau * bw[i] * y[k]);
    for (int c = lane_id(); c < g.n0; c += kWarp) {
        long long p = row * g.n0 + c;
        A acc = wn1[p] + (A)zvn[p];
        for (int k = 0; k < m; ++k) {
            Vec<SZ> Zk = Z0;
            Zk.d += k * zstride;
            if constexpr (PT<SZ>::scaled) Zk.sc += (k * zstride) / g.n0;
            for (int i = 0; i < s; ++i) {
                View<SZ> z = view_of(Zk, 0, (long long)i * g.nx, g.n0);
                acc -= coef[k * s + i] * z.at(row, c);
            }
        }
        zvn1[p] = (double)acc;
    }
}

// Transposed substitution: t_i = b_i u_{n+1}.
template <class A>
__global__ void k_schurT_rhs(long long nx, int s, const StepPtrs* sp, const double* bw, A* t) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)s * nx) return;
    int q = (int)(i / nx);
    t[i] = (A)bw[q] * (A)sp->z[(long long)(sp->n + 1) * nx + i % nx];
}

// u_n = r_{v,n} + u_{n+1} - tau sum_i K q_i   (q flat, s*nx, type A).
template <class A>
__global__ void __launch_bounds__(kBlock) k_schurT_update(Geo g, int s, const StepPtrs* sp, const A* q,
                                                          double tau, SpaceOp<A> sop) {
    pdl_prologue();
    long long row = gwarp();
    if (row >= g.R) return;
    int j, k;
    row_jk(g, row, j, k);
    const int n = sp->n;
    const double* rvn = sp->r + (long long)n * g.nx;
    const double* un1 = sp->z + (long long)(n + 1) * g.nx;
    double* un = sp->z + (long long)n * g.nx;
    View<A> qs[kMaxS];
    for (int i = 0; i < s; ++i) qs[i] = View<A>{q + (long long)i * g.nx, nullptr, g.n0};
    for (int c = lane_id(); c < g.n0; c += kWarp) {
        long long p = row * g.n0 + c;
        A acc = A(0);
        for (int i = 0; i < s; ++i) acc += (A)op_K(qs[i], g, sop, row, j, k, c);
        un[p] = (double)((A)rvn[p] + (A)un1[p] - (A)tau * acc);
    }
}

// ---------------------------------------------------------------------------
// Batched steps of the Schur recurrence (two-level MGRIT, the parallel form of
// S_tilde in Sec. 5): B items of one step at once, item b at time index
// n_b = sp->n + b * stride (forward; transposed: n_b = sp->n - b * stride), the
// items' inner solves batched (blockIdx.y = item).  With `res` set, a step writes
// the C-point residual w_{n+1} + Phi(z_n) - z_{n+1} of item b into block b + 1 of
// res (transposed: block nres - 1 - b) instead of updating the recurrence.
// ---------------------------------------------------------------------------
template <class A>
__global__ void __launch_bounds__(kBlock) k_schur_rhs_b(Geo g, int s, const StepPtrs* sp, int stride, A* t,
                                                        SpaceOp<A> sop) {
    pdl_prologue();
    long long row = gwarp();
    if (row >= g.R) return;
    const int b = blockIdx.y;
    int j, k;
    row_jk(g, row, j, k);
    View<double> z{sp->z + (long long)(sp->n + b * stride) * g.nx, nullptr, g.n0};
    A* tb = t + (long long)b * s * g.nx;
    for (int c = lane_id(); c < g.n0; c += kWarp) {
        A v = (A)op_K(z, g, sop, row, j, k, c);
        for (int i = 0; i < s; ++i) tb[(long long)i * g.nx + row * g.n0 + c] = v;
    }
}

template <class SZ, class A>
__global__ void __launch_bounds__(kBlock) k_schur_update_b(Geo g, int s, const A* wbuf, const StepPtrs* sp,
                                                           int stride, Vec<SZ> Z0, long long zstride,
                                                           const double* y, int kmax, const int* its,
                                                           const double* bw, double tau, A* res) {
    pdl_prologue();
    long long row = gwarp();
    if (row >= g.R) return;
    const int b = blockIdx.y;
    const int n = sp->n + b * stride;
    const A* wn1 = wbuf + (long long)(n + 1) * g.nx;
    const double* zvn = sp->z + (long long)n * g.nx;
    double* zvn1 = sp->z + (long long)(n + 1) * g.nx;
    const int m = its[b];
    A coef[kMaxInner * kMaxS];
    for (int k = 0; k < m; ++k)
        for (int i = 0; i < s; ++i) coef[k * s + i] = (A)(tau * bw[i] * y[(long long)b * kmax + k]);
    for (int c = lane_id(); c < g.n0; c += kWarp) {
        long long p = row * g.n0 + c;
        A acc = wn1[p] + (A)zvn[p];
        for (int k = 0; k < m; ++k) {
            Vec<SZ> Zk = Z0;
            Zk.d += k * zstride;
            if constexpr (PT<SZ>::scaled) Zk.sc += (k * zstride) / g.n0;
            for (int i = 0; i < s; ++i) {
                View<SZ> z = view_of(Zk, b, (long long)i * g.nx, g.n0);
                acc -= coef[k * s + i] * z.at(row, c);
            }
        }
        if (res) res[(long long)(b + 1) * g.nx + p] = acc - (A)zvn1[p];
        else zvn1[p] = (double)acc;
    }
}

// Transposed: t_{b,i} = b_i u_{n_b + 1}.
template <class A>
__global__ void k_schurT_rhs_b(long long nx, int s, const StepPtrs* sp, int stride, const double* bw, A* t) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)s * nx) return;
    const int b = blockIdx.y;
    int q = (int)(i / nx);
    t[(long long)b * s * nx + i] =
        (A)bw[q] * (A)sp->z[(long long)(sp->n - b * stride + 1) * nx + i % nx];
}

// Transposed: u_{n_b} = r_{v,n_b} + u_{n_b+1} - tau sum_i K q_{b,i}  (or its C-point residual).
template <class A>
__global__ void __launch_bounds__(kBlock) k_schurT_update_b(Geo g, int s, const StepPtrs* sp, int stride,
                                                            const A* q, double tau, SpaceOp<A> sop, double* res,
                                                            int nres) {
    pdl_prologue();
    long long row = gwarp();
    if (row >= g.R) return;
    const int b = blockIdx.y;
    int j, k;
    row_jk(g, row, j, k);
    const int n = sp->n - b * stride;
    const double* rvn = sp->r + (long long)n * g.nx;
    const double* un1 = sp->z + (long long)(n + 1) * g.nx;
    double* un = sp->z + (long long)n * g.nx;
    View<A> qs[kMaxS];
    for (int i = 0; i < s; ++i) qs[i] = View<A>{q + ((long long)b * s + i) * g.nx, nullptr, g.n0};
    for (int c = lane_id(); c < g.n0; c += kWarp) {
        long long p = row * g.n0 + c;
        A acc = A(0);
        for (int i = 0; i < s; ++i) acc += (A)op_K(qs[i], g, sop, row, j, k, c);
        const A v = (A)rvn[p] + (A)un1[p] - (A)tau * acc;
        if (res) res[(long long)(nres - 1 - b) * g.nx + p] = (double)(v - (A)un[p]);
        else un[p] = (double)v;
    }
}

// MGRIT C-points: z_{z0 + zdir c m} (+)= e_{e0 + edir c} for c = 1..nc (e == nullptr: set to zero).
static __global__ void k_mgrit_cpoints(double* z, const double* e, long long nx, int nc, int m, int z0, int zdir,
                                       int e0, int edir) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nc * nx) return;
    const int c = (int)(i / nx) + 1;
    const long long p = i % nx;
    double* zp = z + (long long)(z0 + zdir * c * m) * nx + p;
    if (e) *zp += e[(long long)(e0 + edir * c) * nx + p];
    else *zp = 0.0;
}

// t_{n,i} = r_{V,n,i} + tau b_i z_{v,n+1}  (all n at once, type A).
template <class A>
__global__ void k_schurT_vrhs(long long nx, int nt, int s, const double* rV, const double* zv, const double* bw,
                              double tau, A* t) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)nt * s * nx;
    if (i >= tot) return;
    long long n = i / ((long long)s * nx);
    int q = (int)((i / nx) % s);
    long long p = i % nx;
    t[i] = (A)rV[i] + (A)tau * (A)bw[q] * (A)zv[(n + 1) * nx + p];
}

template <class SI, class SO>
__global__ void k_convert(const SI* in, SO* out, long long n) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (SO)in[i];
}

struct Tab {
    int s;
    double A[kMaxS * kMaxS];
    double b[kMaxS];
};

// ---------------------------------------------------------------------------
// Q1 pieces of the Schur substitution: M applied inside the right-hand sides,
// and M^{-1} by Chebyshev semi-iteration with Jacobi splitting (Sec. 5: 20
// steps), batched over blocks of n_x values.
// ---------------------------------------------------------------------------
// g_0 = r_{v,0};  g_{n+1} = r_{v,n+1} + tau M (sum_i b_i zV_{n,i})   (point-mapped over (nt+1) blocks)
template <class A>
__global__ void __launch_bounds__(kPtMaxThreads) k_schur_g_q1(Geo g, PtMap pm, int nt, int s, const double* r,
                                                              const double* zV, const double* bw, double tau,
                                                              Q1<A> q, A* wbuf) {
    pdl_prologue();
    PtPos p = pt_pos(pm, nt + 1, g.R, nullptr);
    if (!p.valid) return;
    const long long row = p.row;
    int j, k;
    row_jk(g, row, j, k);
    const int n = p.b;
    for (int c = p.c0; c < g.n0; c += pm.n0p) {
        const long long idx = (long long)n * g.nx + row * g.n0 + c;
        if (n == 0) {
            wbuf[idx] = (A)r[idx];
            continue;
        }
        A acc = A(0);
        for (int i = 0; i < s; ++i) {
            View<double> zi{zV + ((long long)(n - 1) * s + i) * g.nx, nullptr, g.n0};
            acc += (A)bw[i] * (A)q1_apply(zi, g, q, row, j, k, c, 1.0, 0.0);
        }
        wbuf[idx] = (A)r[idx] + (A)tau * acc;
    }
}

// Chebyshev set-up: x = 0, r = g, d = D^{-1} g / theta  (flat, n values)
template <class A>
__global__ void k_cheb_init(long long n, const A* g, A dinv_theta, A* x, A* r, A* d) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = A(0);
    r[i] = g[i];
    d[i] = dinv_theta * g[i];
}

// x += d;  r -= M d   (B blocks of n_x)
template <class A>
__global__ void __launch_bounds__(kPtMaxThreads) k_cheb_a(Geo g, PtMap pm, int B, Q1<A> q, const A* d, A* x, A* r) {
    pdl_prologue();
    PtPos p = pt_pos(pm, B, g.R, nullptr);
    if (!p.valid) return;
    const long long row = p.row;
    int j, k;
    row_jk(g, row, j, k);
    View<A> dv{d + (long long)p.b * g.nx, nullptr, g.n0};
    for (int c = p.c0; c < g.n0; c += pm.n0p) {
        const long long idx = (long long)p.b * g.nx + row * g.n0 + c;
        x[idx] += d[idx];
        r[idx] -= q1_apply(dv, g, q, row, j, k, c, A(1), A(0));
    }
}

// d = c1 d + c2 D^{-1} r
template <class A>
__global__ void k_cheb_b(long long n, A c1, A c2dinv, const A* r, A* d) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    d[i] = c1 * d[i] + c2dinv * r[i];
}

// t_{n,i} = r_{V,n,i} + tau b_i (M z_{v,n+1})_  (Q1, point-mapped over nt blocks)
template <class A>
__global__ void __launch_bounds__(kPtMaxThreads) k_schurT_vrhs_q1(Geo g, PtMap pm, int nt, int s, const double* rV,
                                                                  const double* zv, const double* bw, double tau,
                                                                  Q1<A> q, A* t) {
    pdl_prologue();
    PtPos p = pt_pos(pm, nt, g.R, nullptr);
    if (!p.valid) return;
    const long long row = p.row;
    int j, k;
    row_jk(g, row, j, k);
    const int n = p.b;
    View<double> zn{zv + (long long)(n + 1) * g.nx, nullptr, g.n0};
    for (int c = p.c0; c < g.n0; c += pm.n0p) {
        A mz = (A)q1_apply(zn, g, q, row, j, k, c, 1.0, 0.0);
        for (int i = 0; i < s; ++i) {
            const long long idx = ((long long)n * s + i) * g.nx + row * g.n0 + c;
            t[idx] = (A)rV[idx] + (A)tau * (A)bw[i] * mz;
        }
    }
}

// FP64 all-at-once matvec for Q1 (M and K both 3^d-point), same row structure
// as k_matvec; transposes use M^T = M, K^T = K.
static __global__ void __launch_bounds__(kBlock) k_matvec_q1(Geo g, int nt, Tab tab, double tau, Q1<double> q,
                                                             const double* x, double* y, const double* rhs,
                                                             int transpose) {
    pdl_prologue();
    long long w = gwarp();
    if (w >= (long long)(nt + 1) * g.R) return;
    int n = (int)(w / g.R);
    long long row = w % g.R;
    int j, k;
    row_jk(g, row, j, k);
    const int s = tab.s;
    const long long nx = g.nx;
    const long long voff = (long long)(nt + 1) * nx;
    const int lane = lane_id();
    if (n == nt) {   // y_{v,0} = M v_0 (forward) or y_{v,nt} = M l_{v,nt} (transpose)
        long long base = transpose ? (long long)nt * nx : 0;
        View<double> v{x + base, nullptr, g.n0};
        for (int c = lane; c < g.n0; c += kWarp) {
            long long p = base + row * g.n0 + c;
            double a = q1_apply(v, g, q, row, j, k, c, 1.0, 0.0);
            y[p] = rhs ? rhs[p] - a : a;
        }
        return;
    }
    View<double> vn{x + (long long)n * nx, nullptr, g.n0};
    View<double> vn1{x + (long long)(n + 1) * nx, nullptr, g.n0};
    View<double> Vs[kMaxS];
    for (int i = 0; i < s; ++i) Vs[i] = View<double>{x + voff + ((long long)n * s + i) * nx, nullptr, g.n0};
    for (int c = lane; c < g.n0; c += kWarp) {
        long long p = row * g.n0 + c;
        double KV[kMaxS], MV[kMaxS];
        for (int i = 0; i < s; ++i) {
            KV[i] = q1_apply(Vs[i], g, q, row, j, k, c, 0.0, 1.0);
            MV[i] = q1_apply(Vs[i], g, q, row, j, k, c, 1.0, 0.0);
        }
        if (!transpose) {
            double acc = q1_apply(vn1, g, q, row, j, k, c, 1.0, 0.0) - q1_apply(vn, g, q, row, j, k, c, 1.0, 0.0);
            for (int i = 0; i < s; ++i) acc -= tau * tab.b[i] * MV[i];
            long long yi = (long long)(n + 1) * nx + p;
            y[yi] = rhs ? rhs[yi] - acc : acc;
            double Kv = q1_apply(vn, g, q, row, j, k, c, 0.0, 1.0);
            for (int i = 0; i < s; ++i) {
                double a = MV[i] + Kv;
                for (int qq = 0; qq < s; ++qq) a += tau * tab.A[i * s + qq] * KV[qq];
                long long yv = voff + ((long long)n * s + i) * nx + p;
                y[yv] = rhs ? rhs[yv] - a : a;
            }
        } else {
            double Mln1 = q1_apply(vn1, g, q, row, j, k, c, 1.0, 0.0);
            double acc = q1_apply(vn, g, q, row, j, k, c, 1.0, 0.0) - Mln1;
            for (int i = 0; i < s; ++i) acc += KV[i];
            long long yi = (long long)n * nx + p;
            y[yi] = rhs ? rhs[yi] - acc : acc;
            for (int i = 0; i < s; ++i) {
                double a = MV[i] - tau * tab.b[i] * Mln1;
                for (int qq = 0; qq < s; ++qq) a += tau * tab.A[qq * s + i] * KV[qq];
                long long yv = voff + ((long long)n * s + i) * nx + p;
                y[yv] = rhs ? rhs[yv] - a : a;
            }
        }
    }
}

// rhs = [M u0 ; 0 ; M f_{n,i}] for Q1 (point-mapped over nt*s + 2 blocks: block 0 = v_0,
// block 1 = the zero v blocks, blocks >= 2 the stage blocks)
static __global__ void __launch_bounds__(kPtMaxThreads) k_rhs_q1(Geo g, PtMap pm, int nt, int s, const double* f,
                                                                 int f_time_dep, const double* u0, Q1<double> q,
                                                                 double* out) {
    pdl_prologue();
    const int nblk = nt * s + 2;
    PtPos p = pt_pos(pm, nblk, g.R, nullptr);
    if (!p.valid) return;
    const long long row = p.row, nx = g.nx;
    int j, k;
    row_jk(g, row, j, k);
    for (int c = p.c0; c < g.n0; c += pm.n0p) {
        const long long pi = row * g.n0 + c;
        if (p.b == 0) {
            View<double> u{u0, nullptr, g.n0};
            out[pi] = q1_apply(u, g, q, row, j, k, c, 1.0, 0.0);
        } else if (p.b == 1) {
            for (int n = 1; n <= nt; ++n) out[(long long)n * nx + pi] = 0.0;
        } else {
            const long long blk = p.b - 2;
            View<double> u{f_time_dep ? f + blk * nx : f, nullptr, g.n0};
            out[(long long)(nt + 1) * nx + blk * nx + pi] = q1_apply(u, g, q, row, j, k, c, 1.0, 0.0);
        }
    }
}

// gf = M sum_{n,i} lambda_{V,n,i}  (Q1; the plain sum is formed by k_grad_f first, in place)
static __global__ void __launch_bounds__(kPtMaxThreads) k_apply_M_q1(Geo g, PtMap pm, Q1<double> q, const double* in,
                                                                     double* out) {
    pdl_prologue();
    PtPos p = pt_pos(pm, 1, g.R, nullptr);
    if (!p.valid) return;
    int j, k;
    row_jk(g, p.row, j, k);
    View<double> u{in, nullptr, g.n0};
    for (int c = p.c0; c < g.n0; c += pm.n0p) out[p.row * g.n0 + c] = q1_apply(u, g, q, p.row, j, k, c, 1.0, 0.0);
}

// ---------------------------------------------------------------------------
// FP64 all-at-once matvec (FD, M = I), one warp per (time block n, row):
//   y_{v,0}   = v_0
//   y_{v,n+1} = v_{n+1} - v_n - tau sum_i b_i V_{n,i}
//   y_{V,n,i} = V_{n,i} + K v_n + tau sum_j a_ij K V_{n,j}
// and its transpose
//   y_{v,n}   = l_{v,n} - l_{v,n+1} + sum_i K l_{V,n,i}   (n < nt),  y_{v,nt} = l_{v,nt}
//   y_{V,n,i} = l_{V,n,i} - tau b_i l_{v,n+1} + tau sum_j a_ji K l_{V,n,j}.
// rhs != nullptr gives y = rhs - (A x).  Warps with n == nt handle block v_0 / v_nt.
// skip != nullptr: the launch does nothing when *skip is nonzero (the relaxed outer product kept
// its FP32 result, k_relax_decide).
// ---------------------------------------------------------------------------

static __global__ void __launch_bounds__(kBlock) k_matvec(Geo g, int nt, Tab tab, double tau, Faces<double> faces,
                                                   const double* x, double* y, const double* rhs, int transpose,
                                                   const int* skip) {
    pdl_prologue();
    if (skip && *skip) return;
    long long w = gwarp();
    if (w >= (long long)(nt + 1) * g.R) return;
    int n = (int)(w / g.R);
    long long row = w % g.R;
    int j, k;
    row_jk(g, row, j, k);
    const int s = tab.s;
    const long long nx = g.nx;
    const long long voff = (long long)(nt + 1) * nx;
    const int lane = lane_id();
    if (n == nt) {   // y_{v,0} (forward) or y_{v,nt} (transpose)
        long long base = (transpose ? (long long)nt * nx : 0) + row * g.n0;
        for (int c = lane; c < g.n0; c += kWarp) {
            double v = x[base + c];
            y[base + c] = rhs ? rhs[base + c] - v : v;
        }
        return;
    }
    View<double> vn{x + (long long)n * nx, nullptr, g.n0};
    View<double> Vs[kMaxS];
    for (int i = 0; i < s; ++i) Vs[i] = View<double>{x + voff + ((long long)n * s + i) * nx, nullptr, g.n0};
    for (int c = lane; c < g.n0; c += kWarp) {
        long long p = row * g.n0 + c;
        double KV[kMaxS];
        for (int i = 0; i < s; ++i) KV[i] = fd_K(Vs[i], g, faces, row, j, k, c);
        if (!transpose) {
            double Kv = fd_K(vn, g, faces, row, j, k, c);
            double acc = x[(long long)(n + 1) * nx + p] - x[(long long)n * nx + p];
            for (int i = 0; i < s; ++i) acc -= tau * tab.b[i] * Vs[i].at(row, c);
            long long yi = (long long)(n + 1) * nx + p;
            y[yi] = rhs ? rhs[yi] - acc : acc;
            for (int i = 0; i < s; ++i) {
                double a = Vs[i].at(row, c) + Kv;
                for (int q = 0; q < s; ++q) a += tau * tab.A[i * s + q] * KV[q];
                long long yv = voff + ((long long)n * s + i) * nx + p;
                y[yv] = rhs ? rhs[yv] - a : a;
            }
        } else {
            double ln1 = x[(long long)(n + 1) * nx + p];
            double acc = x[(long long)n * nx + p] - ln1;
            for (int i = 0; i < s; ++i) acc += KV[i];
            long long yi = (long long)n * nx + p;
            y[yi] = rhs ? rhs[yi] - acc : acc;
            for (int i = 0; i < s; ++i) {
                double a = Vs[i].at(row, c) - tau * tab.b[i] * ln1;
                for (int q = 0; q < s; ++q) a += tau * tab.A[q * s + i] * KV[q];
                long long yv = voff + ((long long)n * s + i) * nx + p;
                y[yv] = rhs ? rhs[yv] - a : a;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Relaxed outer product (aao_options.relax_matvec): y = A x (or A^T x) evaluated in FP32 -- x and
// every coefficient rounded to FP32, every operation in FP32, y stored in FP64 -- beside the
// absolute expression |A||x| (the same linear expression tree with every coefficient and input
// replaced by its absolute value, so no cancellation).  Every output is a linear expression tree
// in the inputs, so fl(y) = sum_t c_t x_t (1 + theta_t) with |theta_t| <= gamma_d, d the number
// of roundings on the longest path from an input to the output (Higham, Accuracy and Stability of
// Numerical Algorithms, Lemma 3.1), and |fl(y) - y| <= gamma_d |A||x| entry by entry.  Counted
// on the stage row with faces in 3D: input 1, difference 1, face product 1, the six-term stencil
// sum 5, the product with the rounded tau a_ij 1 + 2, the stage sum s + 1: s + 12 <= 20 for
// s <= 8; kRelaxDepth = 32 over-counts it.  Each block writes the sum of squares of its outputs'
// absolute expressions to part[blockIdx.x]; absy != nullptr also receives them entry by entry.
// ---------------------------------------------------------------------------
constexpr int kRelaxDepth = 32;

struct K32 {
    float v, a;    // (K u)_P in FP32 and its absolute expression
};

__device__ __forceinline__ K32 fd_K32(const double* u, const Geo& g, const Faces<double>& f, long long row, int j,
                                      int k, int c) {
    auto at = [&](long long r, int cc) -> float { return (float)u[r * g.n0 + cc]; };
    const float uP = at(row, c);
    const float uW = c > 0 ? at(row, c - 1) : 0.f;
    const float uE = c + 1 < g.n0 ? at(row, c + 1) : 0.f;
    const float uS = j > 0 ? at(row - 1, c) : 0.f;
    const float uN = j + 1 < g.n1 ? at(row + 1, c) : 0.f;
    const float aP = fabsf(uP), aW = fabsf(uW), aE = fabsf(uE), aS = fabsf(uS), aN = fabsf(uN);
    K32 o;
    if (f.fx == nullptr) {
        const float hx2 = (float)g.hx2, hy2 = (float)g.hy2;
        o.v = hx2 * (2.f * uP - uW - uE) + hy2 * (2.f * uP - uS - uN);
        o.a = hx2 * (2.f * aP + aW + aE) + hy2 * (2.f * aP + aS + aN);
        if (g.d == 3) {
            const float hz2 = (float)g.hz2;
            const float uD = k > 0 ? at(row - g.n1, c) : 0.f;
            const float uU = k + 1 < g.n2 ? at(row + g.n1, c) : 0.f;
            o.v += hz2 * (2.f * uP - uD - uU);
            o.a += hz2 * (2.f * aP + fabsf(uD) + fabsf(uU));
        }
    } else {
        const long long fxi = row * (g.n0 + 1) + c;
        const long long fyi = ((long long)k * (g.n1 + 1) + j) * g.n0 + c;
        const float fW = (float)f.fx[fxi], fE = (float)f.fx[fxi + 1], fS = (float)f.fy[fyi],
                    fN = (float)f.fy[fyi + g.n0];
        o.v = fW * (uP - uW) + fE * (uP - uE) + fS * (uP - uS) + fN * (uP - uN);
        o.a = fW * (aP + aW) + fE * (aP + aE) + fS * (aP + aS) + fN * (aP + aN);
        if (g.d == 3) {
            const float uD = k > 0 ? at(row - g.n1, c) : 0.f;
            const float uU = k + 1 < g.n2 ? at(row + g.n1, c) : 0.f;
            const long long fzi = ((long long)k * g.n1 + j) * g.n0 + c;
            const float fD = (float)f.fz[fzi], fU = (float)f.fz[fzi + (long long)g.n1 * g.n0];
            o.v += fD * (uP - uD) + fU * (uP - uU);
            o.a += fD * (aP + fabsf(uD)) + fU * (aP + fabsf(uU));
        }
    }
    return o;
}

static __global__ void __launch_bounds__(kBlock) k_matvec32(Geo g, int nt, Tab tab, double tau, Faces<double> faces,
                                                     const double* x, double* y, int transpose, double* part,
                                                     double* absy) {
    pdl_prologue();
    __shared__ double wsum[kBlock / kWarp];
    const long long w = gwarp();
    const int lane = lane_id();
    double sq = 0.0;          // sum of squares of this lane's absolute expressions
    if (w < (long long)(nt + 1) * g.R) {
        const int n = (int)(w / g.R);
        const long long row = w % g.R;
        int j, k;
        row_jk(g, row, j, k);
        const int s = tab.s;
        const long long nx = g.nx;
        const long long voff = (long long)(nt + 1) * nx;
        if (n == nt) {   // y_{v,0} (forward) or y_{v,nt} (transpose)
            const long long base = (transpose ? (long long)nt * nx : 0) + row * g.n0;
            for (int c = lane; c < g.n0; c += kWarp) {
                const float v = (float)x[base + c];
                y[base + c] = (double)v;
                if (absy) absy[base + c] = (double)fabsf(v);
                sq += (double)v * (double)v;
            }
        } else {
            float tA[kMaxS * kMaxS], tb[kMaxS];
            for (int i = 0; i < s * s; ++i) tA[i] = (float)(tau * tab.A[i]);
            for (int i = 0; i < s; ++i) tb[i] = (float)(tau * tab.b[i]);
            const double* xv = x + (long long)n * nx;
            for (int c = lane; c < g.n0; c += kWarp) {
                const long long p = row * g.n0 + c;
                K32 KV[kMaxS];
                float Vi[kMaxS];
                for (int i = 0; i < s; ++i) {
                    const double* xs = x + voff + ((long long)n * s + i) * nx;
                    KV[i] = fd_K32(xs, g, faces, row, j, k, c);
                    Vi[i] = (float)xs[p];
                }
                const float xn1 = (float)x[(long long)(n + 1) * nx + p], xn = (float)xv[p];
                if (!transpose) {
                    const K32 Kv = fd_K32(xv, g, faces, row, j, k, c);
                    float acc = xn1 - xn, abs_ = fabsf(xn1) + fabsf(xn);
                    for (int i = 0; i < s; ++i) {
                        acc -= tb[i] * Vi[i];
                        abs_ += fabsf(tb[i]) * fabsf(Vi[i]);
                    }
                    y[(long long)(n + 1) * nx + p] = (double)acc;
                    if (absy) absy[(long long)(n + 1) * nx + p] = (double)abs_;
                    sq += (double)abs_ * (double)abs_;
                    for (int i = 0; i < s; ++i) {
                        float a = Vi[i] + Kv.v, aa = fabsf(Vi[i]) + Kv.a;
                        for (int q = 0; q < s; ++q) {
                            a += tA[i * s + q] * KV[q].v;
                            aa += fabsf(tA[i * s + q]) * KV[q].a;
                        }
                        y[voff + ((long long)n * s + i) * nx + p] = (double)a;
                        if (absy) absy[voff + ((long long)n * s + i) * nx + p] = (double)aa;
                        sq += (double)aa * (double)aa;
                    }
                } else {
                    float acc = xn - xn1, abs_ = fabsf(xn) + fabsf(xn1);
                    for (int i = 0; i < s; ++i) {
                        acc += KV[i].v;
                        abs_ += KV[i].a;
                    }
                    y[(long long)n * nx + p] = (double)acc;
                    if (absy) absy[(long long)n * nx + p] = (double)abs_;
                    sq += (double)abs_ * (double)abs_;
                    for (int i = 0; i < s; ++i) {
                        float a = Vi[i] - tb[i] * xn1, aa = fabsf(Vi[i]) + fabsf(tb[i]) * fabsf(xn1);
                        for (int q = 0; q < s; ++q) {
                            a += tA[q * s + i] * KV[q].v;
                            aa += fabsf(tA[q * s + i]) * KV[q].a;
                        }
                        y[voff + ((long long)n * s + i) * nx + p] = (double)a;
                        if (absy) absy[voff + ((long long)n * s + i) * nx + p] = (double)aa;
                        sq += (double)aa * (double)aa;
                    }
                }
            }
        }
    }
    sq = warp_sum(sq);
    if (lane == 0) wsum[threadIdx.x / kWarp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kBlock / kWarp; ++i) t += wsum[i];
        part[blockIdx.x] = t;
    }
}

// Accept or reject the FP32 product of outer iteration k: bound = gamma_d (1 + gamma_d)
// sqrt(sum part) (the factor 1 + gamma_d covers the rounding of the absolute expression itself),
// allowed = ell tol ||b|| / (m |g_k|) with ||b|| = bnorm[0] and g_k = gk[0] (the current Givens
// residual).  flag[0] = 1 keeps the FP32 product (the FP64 launch that follows skips), flag[1]
// counts the kept products.  One block; the partial sums are added in a fixed order.
static __global__ void __launch_bounds__(kBlock) k_relax_decide(const double* part, int nblk, double gamma_d,
                                                         double ell, double tol, int m, const double* bnorm,
                                                         const double* gk, int* flag) {
    pdl_prologue();
    __shared__ double red[kBlock];
    double t = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kBlock) t += part[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = kBlock / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double bound = gamma_d * (1.0 + gamma_d) * sqrt(red[0]);
        const double g = fabs(gk[0]);
        const double allowed = g > 0.0 ? ell * tol * bnorm[0] / ((double)m * g) : 0.0;
        const int keep = isfinite(bound) && bound <= allowed ? 1 : 0;
        flag[0] = keep;
        flag[1] += keep;
    }
}

// rhs = [u0 ; 0 ; f_{n,i}]  (FD, M = I)
static __global__ void k_rhs(long long nx, int nt, int s, const double* f, int f_time_dep, const double* u0, double* out) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nv = (long long)(nt + 1) * nx;
    long long tot = nv + (long long)nt * s * nx;
    if (i >= tot) return;
    if (i < nx) out[i] = u0[i];
    else if (i < nv) out[i] = 0.0;
    else out[i] = f_time_dep ? f[i - nv] : f[(i - nv) % nx];
}

// grad_f = sum_{n,i} lambda_{V,n,i}  (FD, M = I)
static __global__ void k_grad_f(long long nx, int nt, int s, const double* lam, double* gf) {
    pdl_prologue();
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nx) return;
    const double* lV = lam + (long long)(nt + 1) * nx;
    double acc = 0.0;
    for (long long q = 0; q < (long long)nt * s; ++q) acc += lV[q * nx + p];
    gf[p] = acc;
}

}  // namespace aao
