// The solver handle and the interface of the precision-specialised
// preconditioner implementations.
#pragma once

#include <cstdlib>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "krylov.cuh"

namespace aao {

struct Handle;

// A named NVTX range over a host scope (the solve, an outer iteration, the P_tilde phases, the
// matvec): profilers that record NVTX can select kernels by phase (ncu --nvtx --nvtx-include).
// Without such a profiler attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Debug switch: with AAO_POISON_WORKSPACE set (and not "0") every device allocation of a handle
// starts filled with 0xFF bytes (NaN in every floating-point type), so that a read of workspace
// before its first write shows up as NaN in the results.
inline bool poison_workspace() {
    const char* v = std::getenv("AAO_POISON_WORKSPACE");
    return v && v[0] && !(v[0] == '0' && v[1] == 0);
}

// Device memory owned by a handle; freed in reverse order at destroy.
struct Arena {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    template <class T> aao_status alloc(T** p, size_t n) {
        *p = nullptr;
        if (n == 0) return AAO_OK;
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("cudaMalloc of ") + std::to_string(n * sizeof(T)) + " bytes failed: " +
                      cudaGetErrorString(e));
            return AAO_ERR_OOM;
        }
        if (poison_workspace()) {
            // the fill runs on the legacy stream: wait for it before any stream of the handle runs
            e = cudaMemset(q, 0xFF, n * sizeof(T));
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) {
                cudaFree(q);
                set_error(std::string("workspace poisoning failed: ") + cudaGetErrorString(e));
                return AAO_ERR_CUDA;
            }
        }
        ptrs.push_back(q);
        bytes += n * sizeof(T);
        *p = static_cast<T*>(q);
        return AAO_OK;
    }
    void release() {
        for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) cudaFree(*it);
        ptrs.clear();
        bytes = 0;
    }
};

class PrecondBase {
  public:
    virtual ~PrecondBase() {}
    virtual aao_status setup() = 0;
    // z = P_tilde^{-1} r (transpose: P_tilde^{-T} r); FP64 device vectors, n_st.
    virtual aao_status apply(const double* r, double* z, int transpose) = 0;
    virtual aao_status shifted_solve(int stage, const double* b, double* x) = 0;
    virtual aao_status pint_apply(const double* r, double* y, int transpose) = 0;
    virtual aao_status inner_solve(int nblocks, const double* r, double* z, int* its_host) = 0;
    virtual long long inner_its() = 0;   // running total (synchronises)
    virtual void reset_inner_its() = 0;
    virtual void release() = 0;
    virtual void accumulate_times() = 0;   // after a synchronising point
    virtual int nonfinite_flag() = 0;      // synchronises
    float t_theta_ms = 0.f, t_schur_ms = 0.f;
};

PrecondBase* make_precond(Handle* h, int prec_P, int prec_Pint);
PrecondBase* make_precond_f64(Handle* h);
PrecondBase* make_precond_f32(Handle* h, int prec_Pint);
PrecondBase* make_precond_lowP(Handle* h, int prec_P);   // P and P_int both BF16 / FP16

struct Handle {
    Geo g;
    int nt = 0, s = 0;
    double tau = 0.0;
    Tab tab;                       // A_RK row-major and b
    double c[kMaxS];
    double L[kMaxS * kMaxS], D[kMaxS];
    aao_options opt;
    cudaStream_t stream = nullptr;
    long long nx = 0, nv = 0, nst = 0;
    Arena arena;

    // device copies of the tableau pieces
    double* d_A = nullptr;         // s*s
    double* d_AT = nullptr;        // s*s transposed
    double* d_b = nullptr;         // s
    double* d_LDf = nullptr;       // s*s: row i holds (L D)_{ij}, j < i
    double* d_LDb = nullptr;       // s*s: row i holds (L D)_{ji}, j > i
    Faces<double> faces64;         // nullptr members for kappa == 1
    int has_kappa = 0;
    int q1 = 0;                    // Q1 finite elements (else finite differences, M = I)
    Q1<double> q1d;

    // outer FGMRES workspace
    int m = 0;                     // restart
    double* V = nullptr;           // (m+1) * nst
    double* Z = nullptr;           // m * nst (right preconditioning)
    double* bt = nullptr;          // nst: P^{-1} b (left preconditioning)
    double* w = nullptr;           // nst
    double* relax_part = nullptr;  // per-block sums of squares of |A||z| (relaxed FP32 product)
    int* relax_flag = nullptr;     // [0] keep the FP32 product of this iteration, [1] products kept
    double* r = nullptr;           // nst
    double* rhs = nullptr;         // nst (staging for solve / host inputs)
    double* xs = nullptr;          // nst (staging for host x)
    double* H = nullptr;           // (m+1)*m
    double* cs = nullptr;
    double* sn = nullptr;
    double* gv = nullptr;          // m+1
    double* y = nullptr;           // m
    double* beta = nullptr;        // [0] beta, [1] bnorm
    int* flags = nullptr;          // [0] active, [1] its, [2] nonfinite, [3] breakdown
    double* resid = nullptr;       // 1
    Red red;                       // reduction scratch
    int red_cap_items = 0, red_cap_chunks = 0;

    // pinned host mirror of the small per-iteration results
    struct Small {
        double resid;
        int active, its, nonfinite, breakdown;
        double beta;
    }* hsmall = nullptr;

    PrecondBase* P = nullptr;
    cudaEvent_t ev[4];
    int ev_ok = 0;

    // reduction blocks per item: about 8 blocks per SM over the whole batch, at
    // most one 32-column segment per warp
    int nchunk_for(int B, long long segments) const {
        // a single small item (the Schur sweep's inner solves): one block per SM, so fewer
        // partials and atomics on the item's counter; otherwise about eight blocks per SM in total
        // (enough loads in flight for the long outer vectors)
        const bool small_single = B == 1 && segments < 152LL * kWarpsPerBlock * 32;
        long long target = small_single ? 152LL : (152LL * 8 + B - 1) / B;
        long long maxc = (segments + kWarpsPerBlock - 1) / kWarpsPerBlock;
        long long c = target < maxc ? target : maxc;
        if (c > red_cap_chunks) c = red_cap_chunks;
        return (int)(c < 1 ? 1 : c);
    }
};

}  // namespace aao
