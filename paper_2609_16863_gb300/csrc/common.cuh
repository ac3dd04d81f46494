// Shared device helpers: precision traits, per-row scaled storage, warp
// reductions, grid geometry and the finite-difference stiffness stencil.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <string>

#include "aao_rk.h"

namespace aao {

constexpr int kWarp = 32;
constexpr int kBlock = 256;              // threads per block of every row kernel
constexpr int kWarpsPerBlock = kBlock / kWarp;
constexpr int kMaxS = 8;                 // RK stages
constexpr int kMaxV = 16;                // values per lane of one row: n0 <= 512
constexpr int kMaxRowLen = kWarp * kMaxV;
constexpr int kMaxInner = 16;            // inner GMRES iterations
constexpr int kMaxRestart = 64;          // outer FGMRES restart
constexpr int kMaxNt = 65534;            // time steps: nt + 1 items fit the 65535 grid.y limit
constexpr int kMaxBatchThreads = 64;     // host workers of a batched solve
constexpr int kMaxLevels = 16;
constexpr int kMaxCoarsest = 512;        // unknowns of the dense coarsest solve
constexpr int kCoarsestTarget = 256;     // coarsening stops at the first level with at most this many unknowns
constexpr int kPtMaxThreads = 512;       // threads per CTA of the point-mapped row kernels

// ---------------------------------------------------------------------------
// Storage precision traits.  Arithmetic is double for FP64 storage and float
// for every lower precision; 16-bit storage carries one power-of-two scale per
// grid row (value = stored * scale), chosen so the row maximum is <= 2^14.
// ---------------------------------------------------------------------------
template <class S> struct PT;
template <> struct PT<double> {
    using A = double;
    static constexpr bool scaled = false;
    __device__ static double ld(double v) { return v; }
    __device__ static double st(double v) { return v; }
};
template <> struct PT<float> {
    using A = float;
    static constexpr bool scaled = false;
    __device__ static float ld(float v) { return v; }
    __device__ static float st(float v) { return v; }
};
template <> struct PT<__nv_bfloat16> {
    using A = float;
    static constexpr bool scaled = true;
    __device__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};
template <> struct PT<__half> {
    using A = float;
    static constexpr bool scaled = true;
    __device__ static float ld(__half v) { return __half2float(v); }
    __device__ static __half st(float v) { return __float2half_rn(v); }
};

// A batched vector in storage type S: item b starts at d + b*bs (elements);
// rows of n0 contiguous values; sc (scaled types only) holds one float per row.
template <class S> struct Vec {
    S* d = nullptr;
    float* sc = nullptr;
    long long bs = 0;
};

// Read-only view of one batch item (or one stage of it) with per-row scales.
template <class S> struct View {
    const S* d;
    const float* sc;
    int n0;
    __device__ __forceinline__ typename PT<S>::A at(long long row, int col) const {
        typename PT<S>::A v = PT<S>::ld(d[row * n0 + col]);
        if constexpr (PT<S>::scaled) v *= sc[row];
        return v;
    }
};

template <class S>
__device__ __forceinline__ View<S> view_of(const Vec<S>& v, long long b, long long elem_off, int n0) {
    View<S> w;
    long long base = b * v.bs + elem_off;
    w.d = v.d + base;
    w.sc = PT<S>::scaled ? v.sc + base / n0 : nullptr;
    w.n0 = n0;
    return w;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Store one row of n0 values f(col) at out (+ its scale at *out_sc) from one warp.
template <class S, class F>
__device__ __forceinline__ void row_store(S* out, float* out_sc, int n0, int lane, F&& f) {
    if constexpr (PT<S>::scaled) {
        float v[kMaxV];
        float m = 0.f;
#pragma unroll
        for (int t = 0; t < kMaxV; ++t) {
            int c = lane + kWarp * t;
            v[t] = 0.f;
            if (c < n0) {
                v[t] = (float)f(c);
                m = fmaxf(m, fabsf(v[t]));
            }
        }
        m = warp_max(m);
        int e = 0;
        float sc = 1.f, inv = 1.f;
        if (m > 0.f && m <= 3.0e38f) {
            frexpf(m, &e);                 // m <= 2^e
            sc = ldexpf(1.f, e - 14);
            inv = ldexpf(1.f, 14 - e);
        }
#pragma unroll
        for (int t = 0; t < kMaxV; ++t) {
            int c = lane + kWarp * t;
            if (c < n0) out[c] = PT<S>::st(v[t] * inv);
        }
        if (lane == 0) *out_sc = sc;
    } else {
        for (int c = lane; c < n0; c += kWarp) out[c] = PT<S>::st((typename PT<S>::A)f(c));
    }
}

// ---------------------------------------------------------------------------
// Point mapping of the row kernels.  A CTA of rpc * n0p threads covers rpc
// whole grid rows (n0p = n0 rounded up to a warp multiple, at most 512);
// thread (lrow, c0) computes columns c0, c0 + n0p, ... of its row.  Because a
// CTA holds whole rows, the per-row scale of a 16-bit row is a CTA-local
// reduction.
// ---------------------------------------------------------------------------
struct PtMap {
    int n0, n0p, rpc;
};

inline PtMap ptmap(int n0) {
    PtMap m;
    m.n0 = n0;
    int p = (n0 + kWarp - 1) / kWarp * kWarp;
    if (p > kPtMaxThreads) p = kPtMaxThreads;
    m.n0p = p;
    m.rpc = p >= 256 ? 1 : 256 / p;
    return m;
}
// Launch geometry: block (n0p, rpc) threads, grid (ceil(R / rpc), B): thread x is
// the column, thread y the row within the CTA, block y the batch item, so the
// kernels need no integer division to find their point.
inline dim3 pt_grid(const PtMap& m, long long R, int B) {
    long long bx = (R + m.rpc - 1) / m.rpc;
    return dim3((unsigned int)(bx < 1 ? 1 : bx), (unsigned int)(B < 1 ? 1 : B), 1);
}
inline dim3 pt_block(const PtMap& m) { return dim3((unsigned int)m.n0p, (unsigned int)m.rpc, 1); }

// Row coordinates of the calling thread for B items of R rows each.
struct PtPos {
    int lrow, c0, b;
    long long row;
    bool valid;
};
__device__ __forceinline__ PtPos pt_pos(const PtMap& m, int B, long long R, const int* active) {
    PtPos q;
    q.lrow = threadIdx.y;
    q.c0 = threadIdx.x;
    q.b = blockIdx.y;
    q.row = (long long)blockIdx.x * m.rpc + threadIdx.y;
    q.valid = q.row < R && q.b < B;
    if (q.valid && active && !active[q.b]) q.valid = false;
    return q;
}

// Store f(c) for this thread's columns of one row (scaled types: n0 <= n0p, one
// column per thread).  Every thread of the CTA must call it for scaled types.
template <class S, class F>
__device__ __forceinline__ void pt_store(S* out_row, float* out_sc, const PtMap& m, int c0, bool valid, F&& f) {
    if constexpr (PT<S>::scaled) {
        __shared__ float wmax[32];
        float v = 0.f;
        if (valid && c0 < m.n0) v = (float)f(c0);
        float a = warp_max(fabsf(v));
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        if ((tid & 31) == 0) wmax[tid >> 5] = a;
        __syncthreads();
        const int wpr = m.n0p >> 5, first = threadIdx.y * wpr;
        float mx = 0.f;
        for (int i = 0; i < wpr; ++i) mx = fmaxf(mx, wmax[first + i]);
        int e = 0;
        float sc = 1.f, inv = 1.f;
        if (mx > 0.f && mx <= 3.0e38f) {
            frexpf(mx, &e);
            sc = ldexpf(1.f, e - 14);
            inv = ldexpf(1.f, 14 - e);
        }
        if (valid && c0 < m.n0) out_row[c0] = PT<S>::st(v * inv);
        if (valid && c0 == 0) *out_sc = sc;
    } else {
        if (valid)
            for (int c = c0; c < m.n0; c += m.n0p) out_row[c] = PT<S>::st((typename PT<S>::A)f(c));
    }
}

template <class S>
__device__ __forceinline__ void row_store_ptrs(const Vec<S>& v, long long b, long long elem_off,
                                               long long row, int n0, S*& out, float*& out_sc) {
    long long base = b * v.bs + elem_off;
    out = v.d + base + row * n0;
    out_sc = PT<S>::scaled ? v.sc + base / n0 + row : nullptr;
}

// ---------------------------------------------------------------------------
// Geometry of one grid level and the FD stiffness K = -div(kappa grad).
// Rows are (j, k) lines along x: row = j + n1*k, R = n1*n2 rows.
// Face coefficients (kappa_f / h^2) are optional (nullptr = kappa == 1):
//   fx[row*(n0+1) + c]       face between x-nodes c-1 and c   (c = 0..n0)
//   fy[(k*(n1+1) + j)*n0 + c] face between y-nodes j-1 and j   (j = 0..n1)
//   fz[(k*n1 + j)*n0 + c]     face between z-nodes k-1 and k   (k = 0..n2)
// ---------------------------------------------------------------------------
struct Geo {
    int d;
    int n0, n1, n2;
    long long nx;   // n0*n1*n2
    int R;          // rows n1*n2
    double hx2, hy2, hz2;   // 1/h^2 per axis
};

// (j, k) of a grid row without 64-bit division (2D: k = 0).
__device__ __forceinline__ void row_jk(const Geo& g, long long row, int& j, int& k) {
    if (g.d == 2) {
        j = (int)row;
        k = 0;
    } else {
        const int r = (int)row;
        k = r / g.n1;
        j = r - k * g.n1;
    }
}

template <class T> struct Faces {
    const T* fx = nullptr;
    const T* fy = nullptr;
    const T* fz = nullptr;
};

// (K u)_P at column c of row (j,k) of view u.
template <class S, class T>
__device__ __forceinline__ typename PT<S>::A fd_K(const View<S>& u, const Geo& g, const Faces<T>& f,
                                                   long long row, int j, int k, int c) {
    using A = typename PT<S>::A;
    A uP = u.at(row, c);
    A uW = c > 0 ? u.at(row, c - 1) : A(0);
    A uE = c + 1 < g.n0 ? u.at(row, c + 1) : A(0);
    A uS = j > 0 ? u.at(row - 1, c) : A(0);
    A uN = j + 1 < g.n1 ? u.at(row + 1, c) : A(0);
    A out;
    if (f.fx == nullptr) {
        out = A(g.hx2) * (A(2) * uP - uW - uE) + A(g.hy2) * (A(2) * uP - uS - uN);
        if (g.d == 3) {
            A uD = k > 0 ? u.at(row - g.n1, c) : A(0);
            A uU = k + 1 < g.n2 ? u.at(row + g.n1, c) : A(0);
            out += A(g.hz2) * (A(2) * uP - uD - uU);
        }
    } else {
        const long long fxi = row * (g.n0 + 1) + c;
        const long long fyi = ((long long)k * (g.n1 + 1) + j) * g.n0 + c;
        out = A(f.fx[fxi]) * (uP - uW) + A(f.fx[fxi + 1]) * (uP - uE) +
              A(f.fy[fyi]) * (uP - uS) + A(f.fy[fyi + g.n0]) * (uP - uN);
        if (g.d == 3) {
            A uD = k > 0 ? u.at(row - g.n1, c) : A(0);
            A uU = k + 1 < g.n2 ? u.at(row + g.n1, c) : A(0);
            const long long fzi = ((long long)k * g.n1 + j) * g.n0 + c;
            out += A(f.fz[fzi]) * (uP - uD) + A(f.fz[fzi + (long long)g.n1 * g.n0]) * (uP - uU);
        }
    }
    return out;
}

// ---------------------------------------------------------------------------
// Q1 finite elements on the tensor vertex mesh (Sec. 5): M = (x)_a M1_a and
// K = sum_a (x)_{b != a} M1_b (x) K1_a with the 1D linear-element matrices
// M1 = h/6 tridiag(1, 4, 1), K1 = 1/h tridiag(-1, 2, -1) on the interior nodes.
// m[a][e], k[a][e] hold the 1D coefficients of offset e - 1 along axis a.
// ---------------------------------------------------------------------------
template <class T> struct Q1 {
    T m[3][3];
    T k[3][3];
};

// alpha_m (M u)_P + alpha_k (K u)_P for the Q1 stencils.
template <class S, class T>
__device__ __forceinline__ typename PT<S>::A q1_apply(const View<S>& u, const Geo& g, const Q1<T>& q, long long row,
                                                      int j, int k, int c, typename PT<S>::A am,
                                                      typename PT<S>::A ak) {
    using A = typename PT<S>::A;
    A acc = A(0);
    const int zlo = g.d == 3 ? -1 : 0, zhi = g.d == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        int kk = k + dz;
        if (kk < 0 || kk >= g.n2) continue;
        const A mz = g.d == 3 ? A(q.m[2][dz + 1]) : A(1), kz = g.d == 3 ? A(q.k[2][dz + 1]) : A(0);
        for (int dy = -1; dy <= 1; ++dy) {
            int jj = j + dy;
            if (jj < 0 || jj >= g.n1) continue;
            const A my = A(q.m[1][dy + 1]), ky = A(q.k[1][dy + 1]);
            long long rr = row + dy + (long long)dz * g.n1;
            for (int dx = -1; dx <= 1; ++dx) {
                int cc = c + dx;
                if (cc < 0 || cc >= g.n0) continue;
                const A mx = A(q.m[0][dx + 1]), kx = A(q.k[0][dx + 1]);
                A kcoef = kx * my * mz + mx * ky * mz;
                if (g.d == 3) kcoef += mx * my * kz;
                acc += (am * mx * my * mz + ak * kcoef) * A(u.at(rr, cc));
            }
        }
    }
    return acc;
}

template <class T> inline Q1<T> make_q1(const Geo& g, double hx, double hy, double hz) {
    Q1<T> q;
    const double h[3] = {hx, hy, hz};
    for (int a = 0; a < 3; ++a) {
        q.m[a][0] = T(h[a] / 6.0);
        q.m[a][1] = T(4.0 * h[a] / 6.0);
        q.m[a][2] = T(h[a] / 6.0);
        q.k[a][0] = T(-1.0 / h[a]);
        q.k[a][1] = T(2.0 / h[a]);
        q.k[a][2] = T(-1.0 / h[a]);
    }
    (void)g;
    return q;
}

// Spatial operator of the fine grid as the stage kernels see it: FD (faces,
// M = I) or Q1 (tensor stencils for M and K).
template <class T> struct SpaceOp {
    int q1 = 0;
    Q1<T> q;
    Faces<T> faces;
};

template <class S, class T>
__device__ __forceinline__ typename PT<S>::A op_K(const View<S>& u, const Geo& g, const SpaceOp<T>& op,
                                                  long long row, int j, int k, int c) {
    using A = typename PT<S>::A;
    if (op.q1) return q1_apply(u, g, op.q, row, j, k, c, A(0), A(1));
    return fd_K(u, g, op.faces, row, j, k, c);
}

template <class S, class T>
__device__ __forceinline__ typename PT<S>::A op_M(const View<S>& u, const Geo& g, const SpaceOp<T>& op,
                                                  long long row, int j, int k, int c) {
    using A = typename PT<S>::A;
    if (op.q1) return q1_apply(u, g, op.q, row, j, k, c, A(1), A(0));
    return A(u.at(row, c));
}

// Diagonal of K at a point.
template <class A, class T>
__device__ __forceinline__ A fd_K_diag(const Geo& g, const Faces<T>& f, long long row, int j, int k, int c) {
    if (f.fx == nullptr) {
        A dg = A(2) * A(g.hx2) + A(2) * A(g.hy2);
        if (g.d == 3) dg += A(2) * A(g.hz2);
        return dg;
    }
    const long long fxi = row * (g.n0 + 1) + c;
    const long long fyi = ((long long)k * (g.n1 + 1) + j) * g.n0 + c;
    A dg = A(f.fx[fxi]) + A(f.fx[fxi + 1]) + A(f.fy[fyi]) + A(f.fy[fyi + g.n0]);
    if (g.d == 3) {
        const long long fzi = ((long long)k * g.n1 + j) * g.n0 + c;
        dg += A(f.fz[fzi]) + A(f.fz[fzi + (long long)g.n1 * g.n0]);
    }
    return dg;
}

// First statement of every kernel of the library (see launch()).
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Global warp id and lane for row kernels.
__device__ __forceinline__ long long gwarp() {
    return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Every kernel of the library is launched through launch(): it counts launches
// (reported by aao_rk_launch_count) and forwards to <<<grid, block, shmem, stream>>>.
// When a profile is open (aao_rk_profile_begin), launches of kernels whose name
// contains the requested text are bracketed by CUDA events on their stream and
// credited with the algorithmic bytes the launch site declared by bytes_hint().
extern std::atomic<long long> g_launches;
extern thread_local long long g_thread_launches;   // launches issued by this host thread
extern bool g_prof_on;
extern thread_local double g_bytes_hint;
int prof_begin_launch(const void* k, cudaStream_t st, double bytes);
void prof_end_launch(int slot, cudaStream_t st);
inline void bytes_hint(double b) { g_bytes_hint = b; }
//
// Kernels are launched with programmatic stream serialisation (programmatic
// dependent launch): a kernel may be scheduled while its predecessor on the
// stream is still running, so every kernel starts with pdl_prologue(), which
// waits for the predecessor grid to complete (and its writes to be visible)
// before anything else, then allows its own successor to start launching.
// Stream order is therefore unchanged; only launch latency is overlapped.
template <class... KArgs, class... Args>
inline void launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t shmem, cudaStream_t st, Args... args) {
    ++g_launches;
    ++g_thread_launches;
    double bytes = g_bytes_hint;
    g_bytes_hint = 0.0;
    int slot = g_prof_on ? prof_begin_launch((const void*)k, st, bytes) : -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = shmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
    if (slot >= 0) prof_end_launch(slot, st);
}

// The same for a grid of thread-block clusters of `cluster` CTAs along x.
template <class... KArgs, class... Args>
inline void launch_cluster(void (*k)(KArgs...), dim3 grid, dim3 block, size_t shmem, cudaStream_t st, int cluster,
                           Args... args) {
    ++g_launches;
    ++g_thread_launches;
    double bytes = g_bytes_hint;
    g_bytes_hint = 0.0;
    int slot = g_prof_on ? prof_begin_launch((const void*)k, st, bytes) : -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = shmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = (unsigned)cluster;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, k, args...);
    if (slot >= 0) prof_end_launch(slot, st);
}

inline unsigned int blocks_for_rows(long long rows) {
    long long b = (rows + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return (unsigned int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// Error state (thread-local last error text)
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
const char* get_error();

#define AAO_CUDA_TRY(expr)                                                            \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess) {                                                      \
            ::aao::set_error(std::string(#expr " failed: ") + cudaGetErrorString(_e)); \
            return _e == cudaErrorMemoryAllocation ? AAO_ERR_OOM : AAO_ERR_CUDA;      \
        }                                                                             \
    } while (0)

#define AAO_TRY(expr)                          \
    do {                                       \
        aao_status _s = (expr);                \
        if (_s != AAO_OK) return _s;           \
    } while (0)

#define AAO_LAUNCH_CHECK()                                                          \
    do {                                                                            \
        cudaError_t _e = cudaGetLastError();                                        \
        if (_e != cudaSuccess) {                                                    \
            ::aao::set_error(std::string("kernel launch failed: ") + cudaGetErrorString(_e)); \
            return AAO_ERR_CUDA;                                                    \
        }                                                                           \
    } while (0)

}  // namespace aao
