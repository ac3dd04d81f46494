// Handle set-up, the FP64 outer FGMRES (Algorithm 1 with P_L = I, P_R =
// P_tilde, restarted) and the extern "C" entry points of include/aao_rk.h.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "handle.cuh"

namespace aao {

std::atomic<long long> g_launches{0};
thread_local long long g_thread_launches = 0;
bool g_prof_on = false;
thread_local double g_bytes_hint = 0.0;
static thread_local std::string g_last_error;

// ---- launch profiling: events around launches of kernels matching a name
struct ProfState {
    std::string match;
    std::unordered_map<const void*, bool> hit;
    std::unordered_map<const void*, std::string> names;
    std::vector<cudaEvent_t> ev;      // pool, pairs
    std::vector<double> bytes;
    std::vector<const void*> kern;    // kernel of each slot
    size_t used = 0;
    std::string first_name;
    std::string report;               // per-kernel table of the last profile
};
static ProfState g_prof;

int prof_begin_launch(const void* k, cudaStream_t st, double bytes) {
    auto it = g_prof.hit.find(k);
    bool h;
    if (it == g_prof.hit.end()) {
        const char* name = nullptr;
        h = cudaFuncGetName(&name, k) == cudaSuccess && name && std::strstr(name, g_prof.match.c_str());
        if (h && g_prof.first_name.empty()) g_prof.first_name = name;
        if (h) g_prof.names[k] = name;
        cudaGetLastError();
        g_prof.hit[k] = h;
    } else {
        h = it->second;
    }
    if (!h) return -1;
    if (g_prof.used * 2 + 2 > g_prof.ev.size()) {
        if (g_prof.ev.size() >= 4000000) return -1;
        size_t add = g_prof.ev.size() ? g_prof.ev.size() : 4096;
        for (size_t i = 0; i < add; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            g_prof.ev.push_back(e);
        }
    }
    int slot = (int)g_prof.used++;
    g_prof.bytes.push_back(bytes);
    g_prof.kern.push_back(k);
    cudaEventRecord(g_prof.ev[2 * slot], st);
    return slot;
}

void prof_end_launch(int slot, cudaStream_t st) { cudaEventRecord(g_prof.ev[2 * slot + 1], st); }
void set_error(const std::string& msg) { g_last_error = msg; }
const char* get_error() { return g_last_error.c_str(); }

// kappa_f / h^2 on every face from nodal kappa (all (n+2)^d nodes).
__global__ void k_faces(Geo g, const double* kap, double* fx, double* fy, double* fz) {
    pdl_prologue();
    const long long N0 = g.n0 + 2, N1 = g.n1 + 2;
    auto node = [&](long long I, long long J, long long K) -> double {
        return kap[I + N0 * (J + N1 * K)];
    };
    const int kofs = g.d == 3 ? 1 : 0;
    long long nfx = (long long)(g.n0 + 1) * g.R;
    long long nfy = (long long)g.n0 * (g.n1 + 1) * g.n2;
    long long nfz = g.d == 3 ? (long long)g.n0 * g.n1 * (g.n2 + 1) : 0;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nfx) {
        long long row = i / (g.n0 + 1);
        int c = (int)(i % (g.n0 + 1));
        int j, k;
    row_jk(g, row, j, k);
        fx[i] = 0.5 * (node(c, j + 1, k + kofs) + node(c + 1, j + 1, k + kofs)) * g.hx2;
        return;
    }
    i -= nfx;
    if (i < nfy) {
        int c = (int)(i % g.n0);
        long long t = i / g.n0;
        int jp = (int)(t % (g.n1 + 1)), k = (int)(t / (g.n1 + 1));
        fy[i] = 0.5 * (node(c + 1, jp, k + kofs) + node(c + 1, jp + 1, k + kofs)) * g.hy2;
        return;
    }
    i -= nfy;
    if (i < nfz) {
        int c = (int)(i % g.n0);
        long long t = i / g.n0;
        int j, kp;
    row_jk(g, t, j, kp);
        fz[i] = 0.5 * (node(c + 1, j + 1, kp) + node(c + 1, j + 1, kp + 1)) * g.hz2;
    }
}

// grad_kappa_m = -sum_{n,i} sum_{faces f containing node m} 1/2 h^-2 (l_P - l_Q)(W_P - W_Q),
// W_{n,i} = v_n + tau sum_j a_ij V_{n,j}; one thread per node of the full grid.
__global__ void k_grad_kappa(Geo g, int nt, Tab tab, double tau, const double* lam, const double* x,
                             double* grad, int accumulate) {
    pdl_prologue();
    const long long N0 = g.n0 + 2, N1 = g.n1 + 2, N2 = g.d == 3 ? g.n2 + 2 : 1;
    long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N0 * N1 * N2) return;
    int I = (int)(m % N0), J = (int)((m / N0) % N1), K = (int)(m / (N0 * N1));
    auto interior = [&](int a, int b, int c) {
        return a >= 1 && a <= g.n0 && b >= 1 && b <= g.n1 && (g.d == 2 || (c >= 1 && c <= g.n2));
    };
    auto pidx = [&](int a, int b, int c) -> long long {
        return (a - 1) + (long long)g.n0 * ((b - 1) + (long long)g.n1 * (g.d == 3 ? c - 1 : 0));
    };
    const int s = tab.s;
    const long long nx = g.nx, voff = (long long)(nt + 1) * nx;
    double acc = 0.0;
    const int dI[6] = {1, -1, 0, 0, 0, 0}, dJ[6] = {0, 0, 1, -1, 0, 0}, dK[6] = {0, 0, 0, 0, 1, -1};
    const double h2[3] = {g.hx2, g.hy2, g.hz2};
    for (int e = 0; e < 2 * g.d; ++e) {
        int I2 = I + dI[e], J2 = J + dJ[e], K2 = K + dK[e];
        if (I2 < 0 || I2 >= N0 || J2 < 0 || J2 >= N1 || K2 < 0 || K2 >= N2) continue;
        bool inP = interior(I, J, K), inQ = interior(I2, J2, K2);
        if (!inP && !inQ) continue;
        long long P = inP ? pidx(I, J, K) : -1, Q = inQ ? pidx(I2, J2, K2) : -1;
        double wgt = 0.5 * h2[e / 2];
        for (int n = 0; n < nt; ++n) {
            double vP = inP ? x[(long long)n * nx + P] : 0.0, vQ = inQ ? x[(long long)n * nx + Q] : 0.0;
            double VP[kMaxS], VQ[kMaxS];
            for (int j = 0; j < s; ++j) {
                long long base = voff + ((long long)n * s + j) * nx;
                VP[j] = inP ? x[base + P] : 0.0;
                VQ[j] = inQ ? x[base + Q] : 0.0;
            }
            for (int i = 0; i < s; ++i) {
                double WP = vP, WQ = vQ;
                for (int j = 0; j < s; ++j) {
                    WP += tau * tab.A[i * s + j] * VP[j];
                    WQ += tau * tab.A[i * s + j] * VQ[j];
                }
                long long base = voff + ((long long)n * s + i) * nx;
                double lP = inP ? lam[base + P] : 0.0, lQ = inQ ? lam[base + Q] : 0.0;
                acc += wgt * (lP - lQ) * (WP - WQ);
            }
        }
    }
    grad[m] = accumulate ? grad[m] - acc : -acc;
}

__global__ void k_outer_init(double* g, int m, const double* beta, int* flags) {
    pdl_prologue();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int i = 0; i <= m; ++i) g[i] = i == 0 ? beta[0] : 0.0;
        flags[0] = 1;
        flags[1] = 0;
    }
}

// w = bt - w (the left-preconditioned residual P^{-1} b - P^{-1} A x).
__global__ void k_sub_from(double* w, const double* bt, long long n) {
    pdl_prologue();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = bt[i] - w[i];
}

struct SmallDev {
    double resid;
    int active, its, nonfinite, breakdown;
    double beta;
};

__global__ void k_pack_small(const double* resid, const int* flags, const double* beta, SmallDev* out) {
    pdl_prologue();
    out->resid = resid[0];
    out->active = flags[0];
    out->its = flags[1];
    out->nonfinite = flags[2];
    out->breakdown = flags[3];
    out->beta = beta[0];
}

// Device memory of the current device (or managed memory).  Device memory of
// another GPU is not taken as device memory: without peer access the kernels
// could not read it.
static bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device == dev;
}

// ---------------------------------------------------------------------------
// relax_matvec: finite and >= 0; > 0 needs the FD product (the FP32 kernel) and right
// preconditioning (the allowance is stated for the right-preconditioned residual).
static aao_status check_relax(double ell, bool q1, int precond_side) {
    if (!(ell >= 0.0) || !std::isfinite(ell)) {
        set_error("relax_matvec must be finite and >= 0");
        return AAO_ERR_ARG;
    }
    if (ell > 0.0 && (q1 || precond_side != 0)) {
        set_error("relax_matvec > 0 needs finite differences and right preconditioning");
        return AAO_ERR_UNSUPPORTED;
    }
    return AAO_OK;
}

static aao_status validate(const aao_grid* grid, double tau, int nt, const aao_tableau* tab,
                           const aao_options* o) {
    if (!grid || !tab || !o) {
        set_error("null argument");
        return AAO_ERR_ARG;
    }
    if (grid->dim != 2 && grid->dim != 3) {
        set_error("dim must be 2 or 3");
        return AAO_ERR_ARG;
    }
    for (int a = 0; a < grid->dim; ++a)
        if (grid->n[a] < 1 || !(grid->len[a] > 0.0) || !std::isfinite(grid->len[a])) {
            set_error("grid sizes and lengths must be positive (lengths finite)");
            return AAO_ERR_ARG;
        }
    if (grid->disc != AAO_DISC_FD && grid->disc != AAO_DISC_Q1) {
        set_error("unknown discretisation");
        return AAO_ERR_ARG;
    }
    if (grid->disc == AAO_DISC_Q1 && grid->kappa) {
        set_error("variable kappa is defined for the finite-difference discretisation only");
        return AAO_ERR_ARG;
    }
    if (!(tau > 0.0) || nt < 1) {
        set_error("tau must be > 0 and nt >= 1");
        return AAO_ERR_ARG;
    }
    if (nt > kMaxNt) {
        // batched launches put the time blocks (up to nt + 1) in the grid's y dimension
        set_error("nt must be at most 65534 (time blocks are a launch grid dimension)");
        return AAO_ERR_ARG;
    }
    if (tab->s < 1 || tab->s > kMaxS) {
        set_error("tableau stages must be in 1..8");
        return AAO_ERR_ARG;
    }
    if (o->restart < 1 || o->restart > kMaxRestart || o->maxit < 0 || !(o->tol >= 0.0)) {
        set_error("restart must be 1..64, maxit >= 0, tol >= 0");
        return AAO_ERR_ARG;
    }
    if (o->inner_maxit < 0 || o->inner_maxit > kMaxInner || o->mg_cycles < 1 || o->mg_pre < 0 || o->mg_post < 0 ||
        !(o->mg_omega > 0.0)) {
        set_error("inner_maxit 0..16, mg_cycles >= 1, mg_pre/mg_post >= 0, mg_omega > 0");
        return AAO_ERR_ARG;
    }
    int P = o->prec_P, I = o->prec_Pint;
    if (P < AAO_FP64 || P > AAO_FP16 || I < AAO_FP64 || I > AAO_FP16) {
        set_error("unknown precision");
        return AAO_ERR_ARG;
    }
    if ((P == AAO_FP64) != (I == AAO_FP64)) {
        set_error("an FP64 P_tilde needs an FP64 P_int and conversely");
        return AAO_ERR_ARG;
    }
    if ((P == AAO_BF16 || P == AAO_FP16) && I != P) {
        set_error("a 16-bit P_tilde needs the same 16-bit P_int");
        return AAO_ERR_ARG;
    }
    if (o->precond_side != 0 && o->precond_side != 1) {
        set_error("precond_side must be 0 (right) or 1 (left)");
        return AAO_ERR_ARG;
    }
    if (o->mgrit_m < 0 || o->mgrit_m == 1 || o->mgrit_m > nt) {
        set_error("mgrit_m must be 0 (substitution) or an m with 2 <= m <= nt");
        return AAO_ERR_ARG;
    }
    if (o->ckpt_every != 0) {
        set_error("ckpt_every must be 0: checkpointed gradients are summed by the caller over windows "
                  "(aao_rk_grad_kappa with accumulate)");
        return AAO_ERR_UNSUPPORTED;
    }
    return check_relax(o->relax_matvec, grid->disc == AAO_DISC_Q1, o->precond_side);
}

static void resolve_defaults(aao_options* o) {
    if (o->inner_maxit == 0) o->inner_maxit = o->prec_P == AAO_FP64 ? 5 : 3;
    if (o->inner_tol < 0.0) o->inner_tol = o->prec_P == AAO_FP64 ? 1e-6 : 1e-3;
}

static aao_status ldu(Handle* h) {
    const int s = h->s;
    double W[kMaxS * kMaxS];
    for (int i = 0; i < s * s; ++i) W[i] = h->tab.A[i];
    for (int i = 0; i < s * s; ++i) h->L[i] = 0.0;
    for (int k = 0; k < s; ++k) {
        h->L[k * s + k] = 1.0;
        double d = W[k * s + k];
        if (!(d > 0.0)) {
            set_error("A_RK has a non-positive LDU pivot");
            return AAO_ERR_BREAKDOWN;
        }
        h->D[k] = d;
        for (int i = k + 1; i < s; ++i) h->L[i * s + k] = W[i * s + k] / d;
        for (int i = k + 1; i < s; ++i)
            for (int j = k + 1; j < s; ++j) W[i * s + j] -= h->L[i * s + k] * W[k * s + j];
    }
    return AAO_OK;
}

static aao_status setup_handle(Handle* h, const aao_grid* grid, double tau, int nt, const aao_tableau* tab,
                               const aao_options* opts) {
    Geo& g = h->g;
    g.d = grid->dim;
    g.n0 = grid->n[0];
    g.n1 = grid->n[1];
    g.n2 = g.d == 3 ? grid->n[2] : 1;
    g.nx = (long long)g.n0 * g.n1 * g.n2;
    g.R = g.n1 * g.n2;
    double hx = grid->len[0] / (g.n0 + 1), hy = grid->len[1] / (g.n1 + 1);
    double hz = g.d == 3 ? grid->len[2] / (g.n2 + 1) : 1.0;
    g.hx2 = 1.0 / (hx * hx);
    g.hy2 = 1.0 / (hy * hy);
    g.hz2 = g.d == 3 ? 1.0 / (hz * hz) : 0.0;
    h->q1 = grid->disc == AAO_DISC_Q1;
    h->q1d = make_q1<double>(g, hx, hy, hz);
    h->nt = nt;
    h->s = tab->s;
    h->tau = tau;
    h->opt = *opts;
    resolve_defaults(&h->opt);
    h->stream = (cudaStream_t)opts->stream;
    h->tab.s = tab->s;
    for (int i = 0; i < tab->s; ++i)
        for (int j = 0; j < tab->s; ++j) h->tab.A[i * tab->s + j] = tab->A[i * tab->s + j];
    for (int i = 0; i < tab->s; ++i) {
        h->tab.b[i] = tab->b[i];
        h->c[i] = tab->c[i];
    }
    AAO_TRY(ldu(h));
    h->nx = g.nx;
    h->nv = (long long)(nt + 1) * g.nx;
    h->nst = h->nv + (long long)nt * h->s * g.nx;
    if (h->nst / g.n0 * ((g.n0 + kWarp - 1) / kWarp) >= (1LL << 32)) {
        set_error("problem too large for the reduction indexing");
        return AAO_ERR_ARG;
    }
    const int s = h->s;
    cudaStream_t st = h->stream;
    Arena& ar = h->arena;
    // tableau pieces
    double hA[kMaxS * kMaxS], hAT[kMaxS * kMaxS], hLDf[kMaxS * kMaxS], hLDb[kMaxS * kMaxS];
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) {
            hA[i * s + j] = h->tab.A[i * s + j];
            hAT[i * s + j] = h->tab.A[j * s + i];
            hLDf[i * s + j] = j < i ? h->L[i * s + j] * h->D[j] : 0.0;
            hLDb[i * s + j] = j > i ? h->L[j * s + i] * h->D[i] : 0.0;
        }
    AAO_TRY(ar.alloc(&h->d_A, s * s));
    AAO_TRY(ar.alloc(&h->d_AT, s * s));
    AAO_TRY(ar.alloc(&h->d_b, s));
    AAO_TRY(ar.alloc(&h->d_LDf, s * s));
    AAO_TRY(ar.alloc(&h->d_LDb, s * s));
    AAO_CUDA_TRY(cudaMemcpy(h->d_A, hA, sizeof(double) * s * s, cudaMemcpyHostToDevice));
    AAO_CUDA_TRY(cudaMemcpy(h->d_AT, hAT, sizeof(double) * s * s, cudaMemcpyHostToDevice));
    AAO_CUDA_TRY(cudaMemcpy(h->d_b, h->tab.b, sizeof(double) * s, cudaMemcpyHostToDevice));
    AAO_CUDA_TRY(cudaMemcpy(h->d_LDf, hLDf, sizeof(double) * s * s, cudaMemcpyHostToDevice));
    AAO_CUDA_TRY(cudaMemcpy(h->d_LDb, hLDb, sizeof(double) * s * s, cudaMemcpyHostToDevice));
    // kappa faces
    if (grid->kappa) {
        h->has_kappa = 1;
        long long nnode = (long long)(g.n0 + 2) * (g.n1 + 2) * (g.d == 3 ? g.n2 + 2 : 1);
        double* kap;
        AAO_TRY(ar.alloc(&kap, nnode));
        AAO_CUDA_TRY(cudaMemcpy(kap, grid->kappa, sizeof(double) * nnode, cudaMemcpyDefault));
        long long nfx = (long long)(g.n0 + 1) * g.R;
        long long nfy = (long long)g.n0 * (g.n1 + 1) * g.n2;
        long long nfz = g.d == 3 ? (long long)g.n0 * g.n1 * (g.n2 + 1) : 0;
        double *fx, *fy, *fz = nullptr;
        AAO_TRY(ar.alloc(&fx, nfx));
        AAO_TRY(ar.alloc(&fy, nfy));
        if (nfz) AAO_TRY(ar.alloc(&fz, nfz));
        long long tot = nfx + nfy + nfz;
        launch(k_faces, (unsigned)((tot + 255) / 256), 256, 0, st, g, kap, fx, fy, fz);
        AAO_LAUNCH_CHECK();
        h->faces64.fx = fx;
        h->faces64.fy = fy;
        h->faces64.fz = fz;
    }
    // outer workspace
    h->m = h->opt.restart;
    const int m = h->m;
    AAO_TRY(ar.alloc(&h->V, (size_t)(m + 1) * h->nst));
    if (h->opt.precond_side == 1) AAO_TRY(ar.alloc(&h->bt, (size_t)h->nst));   // left: P^{-1} b, no Z basis
    else AAO_TRY(ar.alloc(&h->Z, (size_t)m * h->nst));
    AAO_TRY(ar.alloc(&h->w, (size_t)h->nst));
    AAO_TRY(ar.alloc(&h->relax_part, (size_t)blocks_for_rows((long long)(nt + 1) * h->g.R)));
    AAO_TRY(ar.alloc(&h->relax_flag, 2));
    AAO_TRY(ar.alloc(&h->r, (size_t)h->nst));
    AAO_TRY(ar.alloc(&h->rhs, (size_t)h->nst));
    AAO_TRY(ar.alloc(&h->xs, (size_t)h->nst));
    AAO_TRY(ar.alloc(&h->H, (size_t)(m + 1) * m));
    AAO_TRY(ar.alloc(&h->cs, (size_t)m));
    AAO_TRY(ar.alloc(&h->sn, (size_t)m));
    AAO_TRY(ar.alloc(&h->gv, (size_t)m + 1));
    AAO_TRY(ar.alloc(&h->y, (size_t)m));
    AAO_TRY(ar.alloc(&h->beta, 2));
    AAO_TRY(ar.alloc(&h->flags, 4));
    AAO_TRY(ar.alloc(&h->resid, 1));
    AAO_CUDA_TRY(cudaMemset(h->flags, 0, 4 * sizeof(int)));
    h->red_cap_chunks = 152 * 8;
    h->red_cap_items = nt > 1 ? nt : 1;
    AAO_TRY(ar.alloc(&h->red.partials, (size_t)(h->red_cap_chunks + h->red_cap_items + 16)));
    AAO_TRY(ar.alloc(&h->red.count, (size_t)h->red_cap_items));
    AAO_CUDA_TRY(cudaMemset(h->red.count, 0, sizeof(unsigned int) * h->red_cap_items));
    AAO_CUDA_TRY(cudaMallocHost((void**)&h->hsmall, sizeof(SmallDev)));
    h->P = make_precond(h, h->opt.prec_P, h->opt.prec_Pint);
    if (!h->P) {
        set_error("unsupported precision pair");
        return AAO_ERR_ARG;
    }
    AAO_TRY(h->P->setup());
    AAO_CUDA_TRY(cudaDeviceSynchronize());
    return AAO_OK;
}

// ---------------------------------------------------------------------------
static aao_status matvec_dev(Handle* h, const double* x, double* y, const double* rhs, int transpose) {
    NvtxRange range_("aao.matvec");
    const Geo& g = h->g;
    if (h->q1) {
        bytes_hint(8.0 * h->nst * (rhs ? 3 : 2));
        launch(k_matvec_q1, blocks_for_rows((long long)(h->nt + 1) * g.R), kBlock, 0, h->stream, g, h->nt, h->tab,
               h->tau, h->q1d, x, y, rhs, transpose);
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }
    bytes_hint(8.0 * h->nst * (rhs ? 3 : 2));
    launch(k_matvec, blocks_for_rows((long long)(h->nt + 1) * g.R), kBlock, 0, h->stream, 
        g, h->nt, h->tab, h->tau, h->faces64, x, y, rhs, transpose, (const int*)nullptr);
    AAO_LAUNCH_CHECK();
    return AAO_OK;
}

// y = A z_k (transpose: A^T z_k) of outer iteration k with the relaxed precision of
// aao_options.relax_matvec: the FP32 product and its error bound, the decision on the device
// (gv[k] is the current least-squares residual |g_k|, beta[1] = ||b||), and the FP64 product in
// its place when the bound is above the allowance.  No host synchronisation.
static aao_status matvec_relaxed(Handle* h, const double* z, double* y, int k, int transpose) {
    NvtxRange range_("aao.matvec_relaxed");
    const Geo& g = h->g;
    const unsigned nblk = blocks_for_rows((long long)(h->nt + 1) * g.R);
    bytes_hint(8.0 * h->nst * 2);
    launch(k_matvec32, nblk, kBlock, 0, h->stream, g, h->nt, h->tab, h->tau, h->faces64, z, y, transpose,
           h->relax_part, (double*)nullptr);
    const double gam = (double)kRelaxDepth * 0x1p-24 / (1.0 - (double)kRelaxDepth * 0x1p-24);
    launch(k_relax_decide, 1, kBlock, 0, h->stream, (const double*)h->relax_part, (int)nblk, gam,
           h->opt.relax_matvec, h->opt.tol, h->m, (const double*)(h->beta + 1), (const double*)(h->gv + k),
           h->relax_flag);
    bytes_hint(8.0 * h->nst * 2);
    launch(k_matvec, nblk, kBlock, 0, h->stream, g, h->nt, h->tab, h->tau, h->faces64, z, y, (const double*)nullptr,
           transpose, (const int*)h->relax_flag);
    AAO_LAUNCH_CHECK();
    return AAO_OK;
}

static aao_status rhs_dev(Handle* h, const double* f, int f_time_dep, const double* u0, double* out) {
    if (h->q1) {
        const PtMap pm = ptmap(h->g.n0);
        launch(k_rhs_q1, pt_grid(pm, h->g.R, h->nt * h->s + 2), pt_block(pm), 0, h->stream, h->g, pm,
               h->nt, h->s, f, f_time_dep, u0, h->q1d, out);
    } else {
        launch(k_rhs, (unsigned)((h->nst + 255) / 256), 256, 0, h->stream, h->nx, h->nt, h->s, f, f_time_dep, u0, out);
    }
    AAO_LAUNCH_CHECK();
    return AAO_OK;
}

static aao_status norm_dev(Handle* h, const double* v, double* out) {
    const long long rows = h->nst / h->g.n0;
    dim3 grid(h->nchunk_for(1, rows * ((h->g.n0 + kWarp - 1) / kWarp)), 1);
    Red red = h->red;
    red.nchunk = grid.x;
    launch(k_norm<double>, grid, kBlock, 0, h->stream, h->g.n0, rows, 1, nullptr, v, h->nst, red, out, 1);
    AAO_LAUNCH_CHECK();
    return AAO_OK;
}

static aao_status read_small(Handle* h, SmallDev* sd) {
    launch(k_pack_small, 1, 1, 0, h->stream, h->resid, h->flags, h->beta, sd);
    AAO_CUDA_TRY(cudaMemcpyAsync(h->hsmall, sd, sizeof(SmallDev), cudaMemcpyDeviceToHost, h->stream));
    AAO_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return AAO_OK;
}

// Restarted FGMRES (Algorithm 1, P_L = I, P_R = P_tilde or P_tilde^T), FP64.
static aao_status fgmres(Handle* h, const double* b, double* x, int x0_given, int transpose, aao_info* info,
                         SmallDev* sd) {
    NvtxRange range_(transpose ? "aao.fgmres_adjoint" : "aao.fgmres");
    auto t0 = std::chrono::steady_clock::now();
    const long long nst = h->nst;
    const int n0 = h->g.n0, m = h->m;
    const long long rows = nst / n0;
    cudaStream_t st = h->stream;
    aao_info loc;
    memset(&loc, 0, sizeof(loc));
    h->P->t_theta_ms = h->P->t_schur_ms = 0.f;
    h->P->reset_inner_its();
    AAO_CUDA_TRY(cudaMemsetAsync(h->relax_flag, 0, 2 * sizeof(int), st));
    AAO_TRY(norm_dev(h, b, h->beta + 1));
    double bnorm = 0.0;
    AAO_CUDA_TRY(cudaMemcpyAsync(&bnorm, h->beta + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    AAO_CUDA_TRY(cudaStreamSynchronize(st));
    aao_status status = AAO_OK;
    if (!std::isfinite(bnorm)) {
        set_error("right-hand side is not finite");
        return AAO_ERR_NONFINITE;
    }
    if (bnorm == 0.0) {
        AAO_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * nst, st));
        loc.converged = 1;
    } else {
        if (x0_given) {
            AAO_TRY(matvec_dev(h, x, h->r, b, transpose));
        } else {
            AAO_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * nst, st));
            AAO_CUDA_TRY(cudaMemcpyAsync(h->r, b, sizeof(double) * nst, cudaMemcpyDeviceToDevice, st));
        }
        AAO_TRY(norm_dev(h, h->r, h->beta));
        AAO_TRY(read_small(h, sd));
        double beta = h->hsmall->beta;
        int total = 0;
        const double tol = h->opt.tol;
        Red red = h->red;
        red.nchunk = h->nchunk_for(1, rows * ((n0 + kWarp - 1) / kWarp));
        dim3 rgrid(red.nchunk, 1);
        const PtMap pmo = ptmap(n0);
        const dim3 nbp = pt_grid(pmo, rows, 1), ntp = pt_block(pmo);
        while (true) {
            if (!std::isfinite(beta)) {
                set_error("residual became non-finite");
                status = AAO_ERR_NONFINITE;
                break;
            }
            if (beta <= tol * bnorm) {
                loc.converged = 1;
                break;
            }
            if (total >= h->opt.maxit) break;
            Vec<double> V0{h->V, nullptr, nst};
            launch(k_scale_store<double, double>, nbp, ntp, 0, st, pmo, (int)rows, 1, (const int*)nullptr, (const double*)h->r, nst,
                   (const double*)h->beta, 0LL, V0);
            launch(k_outer_init, 1, 32, 0, st, h->gv, m, h->beta, h->flags);
            AAO_LAUNCH_CHECK();
            bool stop = false;
            for (int k = 0; k < m; ++k) {
                NvtxRange iter_("aao.outer_iteration");
                ++total;
                double* Vk = h->V + (long long)k * nst;
                double* Zk = h->Z + (long long)k * nst;
                AAO_TRY(h->P->apply(Vk, Zk, transpose));
                if (h->opt.relax_matvec > 0.0) AAO_TRY(matvec_relaxed(h, Zk, h->w, k, transpose));
                else AAO_TRY(matvec_dev(h, Zk, h->w, nullptr, transpose));
                {
                    NvtxRange ortho_("aao.orthogonalize");
                    Vec<double> none{};
                    Vec<double> Vfirst{h->V, nullptr, nst};
                    launch(k_mgs<double, double>, rgrid, kBlock, 0, st, n0, rows, 1, nullptr, h->w, nst, none,
                           nullptr, Vfirst, 0, red, h->H + k);
                    for (int i = 1; i <= k + 1; ++i) {
                        Vec<double> Vp{h->V + (long long)(i - 1) * nst, nullptr, nst};
                        Vec<double> Vn = i <= k ? Vec<double>{h->V + (long long)i * nst, nullptr, nst} : none;
                        launch(k_mgs<double, double>, rgrid, kBlock, 0, st, n0, rows, 1, nullptr, h->w, nst, Vp,
                               h->H + (i - 1) * m + k, Vn, 0, red, h->H + i * m + k);
                    }
                }
                launch(k_givens, 1, 32, 0, st, 1, k, m, h->H, 0, h->cs, h->sn, h->gv, h->beta + 1, tol, h->flags,
                                           h->flags + 1, h->flags + 2, h->resid);
                AAO_LAUNCH_CHECK();
                AAO_TRY(read_small(h, sd));
                h->P->accumulate_times();
                if (loc.n_history < 128) loc.history[loc.n_history++] = h->hsmall->resid / bnorm;
                if (h->hsmall->nonfinite || h->P->nonfinite_flag()) {
                    set_error("non-finite Krylov coefficient");
                    status = AAO_ERR_NONFINITE;
                    stop = true;
                    break;
                }
                if (!h->hsmall->active || total >= h->opt.maxit) break;
                Vec<double> Vn{h->V + (long long)(k + 1) * nst, nullptr, nst};
                launch(k_scale_store<double, double>, nbp, ntp, 0, st, pmo, (int)rows, 1, (const int*)nullptr, (const double*)h->w, nst,
                                                                     h->H + (k + 1) * m + k, 0, Vn);
                AAO_LAUNCH_CHECK();
            }
            if (stop) break;
            launch(k_hess_solve, 1, 32, 0, st, 1, m, h->H, 0, h->gv, h->flags + 1, h->y, h->flags + 3);
            Vec<double> Zc{h->Z, nullptr, nst};
            launch(k_combine<double, double>, nbp, ntp, 0, st, pmo, (int)rows, 1, Zc, nst, (const double*)h->y, m,
                   (const int*)(h->flags + 1), x, nst, 1);
            AAO_LAUNCH_CHECK();
            AAO_TRY(matvec_dev(h, x, h->r, b, transpose));
            AAO_TRY(norm_dev(h, h->r, h->beta));
            AAO_TRY(read_small(h, sd));
            beta = h->hsmall->beta;
        }
        loc.outer_its = total;
        loc.rel_res = beta / bnorm;
        if (status == AAO_OK && !loc.converged) {
            set_error("FGMRES reached maxit");
            status = AAO_ERR_NOT_CONVERGED;
        }
    }
    AAO_CUDA_TRY(cudaStreamSynchronize(st));
    {
        int rf[2] = {0, 0};
        AAO_CUDA_TRY(cudaMemcpy(rf, h->relax_flag, sizeof(rf), cudaMemcpyDeviceToHost));
        loc.relaxed_matvecs = rf[1];
    }
    loc.inner_its_total = h->P->inner_its();
    loc.t_theta_ms = h->P->t_theta_ms;
    loc.t_schur_ms = h->P->t_schur_ms;
    loc.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = loc;
    return status;
}

// Algorithm 1 with P_L = P_tilde (or P_tilde^T) and P_R = I, in FP64 (the left preconditioning of
// the paper's parallel runs, Sec. 5.2): r_0 = P^{-1} b - P^{-1} A x_0, beta_0 = ||r_0|| of the first
// cycle; iteration k: w = P^{-1} (A v_k), modified Gram--Schmidt, Givens; a cycle ends when
// |g_{k+1}| <= tol beta_0, h_{k+1,k} = 0, after `restart` iterations or at maxit; x += V_k y_k;
// the solve has converged when the recomputed ||P^{-1} b - P^{-1} A x|| <= tol beta_0.  rel_res
// reports the true ||b - A x|| / ||b||.
static aao_status fgmres_left(Handle* h, const double* b, double* x, int x0_given, int transpose, aao_info* info,
                              SmallDev* sd) {
    NvtxRange range_(transpose ? "aao.fgmres_left_adjoint" : "aao.fgmres_left");
    auto t0 = std::chrono::steady_clock::now();
    const long long nst = h->nst;
    const int n0 = h->g.n0, m = h->m;
    const long long rows = nst / n0;
    cudaStream_t st = h->stream;
    aao_info loc;
    memset(&loc, 0, sizeof(loc));
    h->P->t_theta_ms = h->P->t_schur_ms = 0.f;
    h->P->reset_inner_its();
    AAO_TRY(norm_dev(h, b, h->beta + 1));
    double bnorm = 0.0;
    AAO_CUDA_TRY(cudaMemcpyAsync(&bnorm, h->beta + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    AAO_CUDA_TRY(cudaStreamSynchronize(st));
    if (!std::isfinite(bnorm)) {
        set_error("right-hand side is not finite");
        return AAO_ERR_NONFINITE;
    }
    aao_status status = AAO_OK;
    const unsigned nbl = (unsigned)((nst + 255) / 256);
    if (bnorm == 0.0) {
        AAO_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * nst, st));
        loc.converged = 1;
    } else {
        if (!x0_given) AAO_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * nst, st));
        AAO_TRY(h->P->apply(b, h->bt, transpose));                 // P^{-1} b
        double beta0 = -1.0, beta = 0.0;
        int total = 0;
        const double tol = h->opt.tol;
        Red red = h->red;
        red.nchunk = h->nchunk_for(1, rows * ((n0 + kWarp - 1) / kWarp));
        dim3 rgrid(red.nchunk, 1);
        const PtMap pmo = ptmap(n0);
        const dim3 nbp = pt_grid(pmo, rows, 1), ntp = pt_block(pmo);
        while (true) {
            // r = P^{-1} b - P^{-1} (A x)
            AAO_TRY(matvec_dev(h, x, h->r, nullptr, transpose));
            AAO_TRY(h->P->apply(h->r, h->w, transpose));
            launch(k_sub_from, nbl, 256, 0, st, h->w, (const double*)h->bt, nst);
            AAO_TRY(norm_dev(h, h->w, h->beta));
            AAO_TRY(read_small(h, sd));
            beta = h->hsmall->beta;
            if (!std::isfinite(beta)) {
                set_error("residual became non-finite");
                status = AAO_ERR_NONFINITE;
                break;
            }
            if (beta0 < 0.0) {
                beta0 = beta;
                // k_givens tests |g_{k+1}| <= tol * beta[1]: the reference is beta_0 here
                AAO_CUDA_TRY(cudaMemcpyAsync(h->beta + 1, h->beta, sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
            if (beta <= tol * beta0) {
                loc.converged = 1;
                break;
            }
            if (total >= h->opt.maxit) break;
            Vec<double> V0{h->V, nullptr, nst};
            launch(k_scale_store<double, double>, nbp, ntp, 0, st, pmo, (int)rows, 1, (const int*)nullptr,
                   (const double*)h->w, nst, (const double*)h->beta, 0LL, V0);
            launch(k_outer_init, 1, 32, 0, st, h->gv, m, h->beta, h->flags);
            AAO_LAUNCH_CHECK();
            bool stop = false;
            for (int k = 0; k < m; ++k) {
                NvtxRange iter_("aao.outer_iteration");
                ++total;
                double* Vk = h->V + (long long)k * nst;
                AAO_TRY(matvec_dev(h, Vk, h->r, nullptr, transpose));
                AAO_TRY(h->P->apply(h->r, h->w, transpose));
                {
                    NvtxRange ortho_("aao.orthogonalize");
                    Vec<double> none{};
                    Vec<double> Vfirst{h->V, nullptr, nst};
                    launch(k_mgs<double, double>, rgrid, kBlock, 0, st, n0, rows, 1, nullptr, h->w, nst, none,
                           nullptr, Vfirst, 0, red, h->H + k);
                    for (int i = 1; i <= k + 1; ++i) {
                        Vec<double> Vp{h->V + (long long)(i - 1) * nst, nullptr, nst};
                        Vec<double> Vn = i <= k ? Vec<double>{h->V + (long long)i * nst, nullptr, nst} : none;
                        launch(k_mgs<double, double>, rgrid, kBlock, 0, st, n0, rows, 1, nullptr, h->w, nst, Vp,
                               h->H + (i - 1) * m + k, Vn, 0, red, h->H + i * m + k);
                    }
                }
                launch(k_givens, 1, 32, 0, st, 1, k, m, h->H, 0, h->cs, h->sn, h->gv, h->beta + 1, tol, h->flags,
                       h->flags + 1, h->flags + 2, h->resid);
                AAO_LAUNCH_CHECK();
                AAO_TRY(read_small(h, sd));
                h->P->accumulate_times();
                if (loc.n_history < 128) loc.history[loc.n_history++] = h->hsmall->resid / beta0;
                if (h->hsmall->nonfinite || h->P->nonfinite_flag()) {
                    set_error("non-finite Krylov coefficient");
                    status = AAO_ERR_NONFINITE;
                    stop = true;
                    break;
                }
                if (!h->hsmall->active || total >= h->opt.maxit) break;
                Vec<double> Vn{h->V + (long long)(k + 1) * nst, nullptr, nst};
                launch(k_scale_store<double, double>, nbp, ntp, 0, st, pmo, (int)rows, 1, (const int*)nullptr,
                       (const double*)h->w, nst, h->H + (k + 1) * m + k, 0, Vn);
                AAO_LAUNCH_CHECK();
            }
            if (stop) break;
            launch(k_hess_solve, 1, 32, 0, st, 1, m, h->H, 0, h->gv, h->flags + 1, h->y, h->flags + 3);
            Vec<double> Vc{h->V, nullptr, nst};
            launch(k_combine<double, double>, nbp, ntp, 0, st, pmo, (int)rows, 1, Vc, nst, (const double*)h->y, m,
                   (const int*)(h->flags + 1), x, nst, 1);
            AAO_LAUNCH_CHECK();
        }
        loc.outer_its = total;
        // true residual of the final iterate
        AAO_TRY(matvec_dev(h, x, h->r, b, transpose));
        AAO_TRY(norm_dev(h, h->r, h->beta));
        AAO_TRY(read_small(h, sd));
        loc.rel_res = h->hsmall->beta / bnorm;
        if (status == AAO_OK && !loc.converged) {
            set_error("FGMRES reached maxit");
            status = AAO_ERR_NOT_CONVERGED;
        }
    }
    AAO_CUDA_TRY(cudaStreamSynchronize(st));
    loc.inner_its_total = h->P->inner_its();
    loc.t_theta_ms = h->P->t_theta_ms;
    loc.t_schur_ms = h->P->t_schur_ms;
    loc.t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = loc;
    return status;
}

// The outer solver the options select.
static aao_status outer_solve(Handle* h, const double* b, double* x, int x0_given, int transpose, aao_info* info,
                              SmallDev* sd) {
    if (h->opt.precond_side == 1) return fgmres_left(h, b, x, x0_given, transpose, info, sd);
    return fgmres(h, b, x, x0_given, transpose, info, sd);
}

PrecondBase* make_precond(Handle* h, int prec_P, int prec_Pint) {
    if (prec_P == AAO_FP64) return make_precond_f64(h);
    if (prec_P == AAO_FP32) return make_precond_f32(h, prec_Pint);
    return make_precond_lowP(h, prec_P);
}

}  // namespace aao

using namespace aao;

struct aao_rk_handle_s {
    Handle h;
    SmallDev* sd = nullptr;
    double* stage_in = nullptr;   // nst
    double* stage_out = nullptr;  // nst
    double* stage_aux = nullptr;  // nst
};

#define H_CHECK(hh)                          \
    if (!(hh)) {                             \
        set_error("null handle");            \
        return AAO_ERR_ARG;                  \
    }

// Copy a (possibly host) input of n doubles to device memory; returns the device pointer.
static aao_status stage_in(aao_rk_handle hh, const double* p, size_t n, double* buf, const double** dev) {
    if (p == nullptr) {
        *dev = nullptr;
        return AAO_OK;
    }
    if (is_device_ptr(p)) {
        *dev = p;
        return AAO_OK;
    }
    AAO_CUDA_TRY(cudaMemcpyAsync(buf, p, sizeof(double) * n, cudaMemcpyHostToDevice, hh->h.stream));
    *dev = buf;
    return AAO_OK;
}

static aao_status stage_out_begin(const double* p, double* buf, double** dev) {
    if (is_device_ptr(p)) {
        *dev = const_cast<double*>(p);
        return AAO_OK;
    }
    *dev = buf;
    return AAO_OK;
}

static aao_status stage_out_end(aao_rk_handle hh, double* p, double* dev, size_t n) {
    if (dev == p) return AAO_OK;
    AAO_CUDA_TRY(cudaMemcpyAsync(p, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, hh->h.stream));
    AAO_CUDA_TRY(cudaStreamSynchronize(hh->h.stream));
    return AAO_OK;
}

extern "C" {

void aao_rk_default_options(aao_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->restart = 20;
    o->maxit = 100;
    o->inner_maxit = 0;
    o->inner_tol = -1.0;
    o->mg_cycles = 3;
    o->mg_pre = 2;
    o->mg_post = 2;
    o->mg_omega = 0.8;
    o->cheb_steps = 20;
    o->prec_P = AAO_FP64;
    o->prec_Pint = AAO_FP64;
    o->ckpt_every = 0;
    o->stream = nullptr;
    o->mgrit_m = 0;
    o->precond_side = 0;
    o->relax_matvec = 0.0;
}

const char* aao_rk_last_error(void) { return get_error(); }

long long aao_rk_launch_count(void) { return g_launches; }

aao_status aao_rk_profile_begin(const char* kernel_name) {
    if (!kernel_name || !*kernel_name) {
        set_error("empty kernel name");
        return AAO_ERR_ARG;
    }
    g_prof.match = kernel_name;
    g_prof.hit.clear();
    g_prof.bytes.clear();
    g_prof.kern.clear();
    g_prof.used = 0;
    g_prof.first_name.clear();
    g_prof_on = true;
    return AAO_OK;
}

aao_status aao_rk_profile_end(long long* launches, double* total_ms, double* total_bytes) {
    g_prof_on = false;
    AAO_CUDA_TRY(cudaDeviceSynchronize());
    double ms = 0.0, by = 0.0;
    struct Agg {
        long long n = 0;
        double ms = 0.0, bytes = 0.0;
    };
    std::unordered_map<const void*, Agg> agg;
    for (size_t i = 0; i < g_prof.used; ++i) {
        float t = 0.f;
        AAO_CUDA_TRY(cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]));
        ms += t;
        by += g_prof.bytes[i];
        Agg& a = agg[g_prof.kern[i]];
        a.n += 1;
        a.ms += t;
        a.bytes += g_prof.bytes[i];
    }
    g_prof.report.clear();
    for (auto& kv : agg) {
        char line[512];
        std::snprintf(line, sizeof(line), "%s\t%lld\t%.6f\t%.1f\n", g_prof.names[kv.first].c_str(), kv.second.n,
                      kv.second.ms, kv.second.bytes);
        g_prof.report += line;
    }
    if (launches) *launches = (long long)g_prof.used;
    if (total_ms) *total_ms = ms;
    if (total_bytes) *total_bytes = by;
    g_prof.used = 0;
    g_prof.bytes.clear();
    g_prof.kern.clear();
    return AAO_OK;
}

const char* aao_rk_profile_report(void) {
    return g_prof.report.c_str();
}

aao_status aao_rk_setup(const aao_grid* grid, double tau, int nt, const aao_tableau* tab, const aao_options* opts,
                        aao_rk_handle* out) {
    if (!out) {
        set_error("null output handle");
        return AAO_ERR_ARG;
    }
    *out = nullptr;
    AAO_TRY(validate(grid, tau, nt, tab, opts));
    aao_rk_handle hh = new (std::nothrow) aao_rk_handle_s();
    if (!hh) {
        set_error("host allocation failed");
        return AAO_ERR_OOM;
    }
    aao_status s = setup_handle(&hh->h, grid, tau, nt, tab, opts);
    if (s == AAO_OK) s = hh->h.arena.alloc(&hh->sd, 1);
    if (s == AAO_OK) s = hh->h.arena.alloc(&hh->stage_in, (size_t)hh->h.nst);
    if (s == AAO_OK) s = hh->h.arena.alloc(&hh->stage_out, (size_t)hh->h.nst);
    if (s == AAO_OK) s = hh->h.arena.alloc(&hh->stage_aux, (size_t)hh->h.nst);
    if (s != AAO_OK) {
        aao_rk_destroy(hh);
        return s;
    }
    *out = hh;
    return AAO_OK;
}

void aao_rk_destroy(aao_rk_handle hh) {
    if (!hh) return;
    if (hh->h.stream) cudaStreamSynchronize(hh->h.stream);
    else cudaDeviceSynchronize();
    if (hh->h.P) {
        delete hh->h.P;
        hh->h.P = nullptr;
    }
    if (hh->h.hsmall) cudaFreeHost(hh->h.hsmall);
    hh->h.arena.release();
    cudaGetLastError();
    delete hh;
}

aao_status aao_rk_sizes(aao_rk_handle hh, long long* n_x, long long* n_st) {
    H_CHECK(hh);
    if (n_x) *n_x = hh->h.nx;
    if (n_st) *n_st = hh->h.nst;
    return AAO_OK;
}

aao_status aao_rk_set_options(aao_rk_handle hh, const aao_options* o) {
    H_CHECK(hh);
    if (!o) {
        set_error("null options");
        return AAO_ERR_ARG;
    }
    const aao_options& c = hh->h.opt;
    if (o->prec_P != c.prec_P || o->prec_Pint != c.prec_Pint || o->mg_cycles != c.mg_cycles ||
        o->mg_pre != c.mg_pre || o->mg_post != c.mg_post || o->restart > c.restart || o->restart < 1 ||
        (o->inner_maxit != 0 && o->inner_maxit != c.inner_maxit) || o->mgrit_m != c.mgrit_m ||
        o->precond_side != c.precond_side) {
        set_error("precisions, multigrid shape, inner_maxit, mgrit_m, precond_side and a larger restart are "
                  "fixed at set-up");
        return AAO_ERR_ARG;
    }
    AAO_TRY(check_relax(o->relax_matvec, hh->h.q1 != 0, c.precond_side));
    aao_options n = *o;
    n.inner_maxit = c.inner_maxit;
    if (n.inner_tol < 0.0) n.inner_tol = c.inner_tol;
    if ((cudaStream_t)n.stream != hh->h.stream) {
        set_error("the stream is fixed at set-up");
        return AAO_ERR_ARG;
    }
    hh->h.opt = n;
    hh->h.m = n.restart;
    return AAO_OK;
}

aao_status aao_rk_rhs(aao_rk_handle hh, const double* f, int f_time_dep, const double* u0, double* rhs) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!f || !u0 || !rhs) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    const double *fd, *ud;
    AAO_TRY(stage_in(hh, f, f_time_dep ? (size_t)h->nt * h->s * h->nx : (size_t)h->nx, hh->stage_in, &fd));
    AAO_TRY(stage_in(hh, u0, (size_t)h->nx, hh->stage_aux, &ud));
    double* od;
    AAO_TRY(stage_out_begin(rhs, hh->stage_out, &od));
    AAO_TRY(rhs_dev(h, fd, f_time_dep, ud, od));
    AAO_LAUNCH_CHECK();
    return stage_out_end(hh, rhs, od, (size_t)h->nst);
}

static aao_status matvec_api(aao_rk_handle hh, const double* x, double* y, int transpose) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!x || !y) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    const double* xd;
    AAO_TRY(stage_in(hh, x, (size_t)h->nst, hh->stage_in, &xd));
    double* yd;
    AAO_TRY(stage_out_begin(y, hh->stage_out, &yd));
    AAO_TRY(matvec_dev(h, xd, yd, nullptr, transpose));
    return stage_out_end(hh, y, yd, (size_t)h->nst);
}

aao_status aao_rk_matvec(aao_rk_handle hh, const double* x, double* y) { return matvec_api(hh, x, y, 0); }

aao_status aao_rk_matvec_relaxed(aao_rk_handle hh, const double* x, double* y, double* absy, int transpose) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(absy)) {
        set_error("x, y and absy must be device arrays");
        return AAO_ERR_ARG;
    }
    if (h->q1) {
        set_error("the FP32 relaxed product is built for finite differences");
        return AAO_ERR_UNSUPPORTED;
    }
    const unsigned nblk = blocks_for_rows((long long)(h->nt + 1) * h->g.R);
    bytes_hint(8.0 * h->nst * 3);
    launch(k_matvec32, nblk, kBlock, 0, h->stream, h->g, h->nt, h->tab, h->tau, h->faces64, x, y, transpose ? 1 : 0,
           h->relax_part, absy);
    AAO_LAUNCH_CHECK();
    AAO_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return AAO_OK;
}
aao_status aao_rk_matvec_transpose(aao_rk_handle hh, const double* x, double* y) { return matvec_api(hh, x, y, 1); }

static aao_status precond_api(aao_rk_handle hh, const double* r, double* z, int transpose) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!r || !z || r == z) {
        set_error("null or aliased vectors");
        return AAO_ERR_ARG;
    }
    const double* rd;
    AAO_TRY(stage_in(hh, r, (size_t)h->nst, hh->stage_in, &rd));
    double* zd;
    AAO_TRY(stage_out_begin(z, hh->stage_out, &zd));
    AAO_TRY(h->P->apply(rd, zd, transpose));
    if (h->P->nonfinite_flag()) {
        set_error("non-finite value inside the preconditioner");
        return AAO_ERR_NONFINITE;
    }
    return stage_out_end(hh, z, zd, (size_t)h->nst);
}

aao_status aao_rk_precond_apply(aao_rk_handle hh, const double* r, double* z) { return precond_api(hh, r, z, 0); }
aao_status aao_rk_precond_apply_transpose(aao_rk_handle hh, const double* r, double* z) {
    return precond_api(hh, r, z, 1);
}

aao_status aao_rk_solve_rhs(aao_rk_handle hh, const double* rhs, double* x, int x0_given, aao_info* info) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!rhs || !x) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    const double* bd;
    AAO_TRY(stage_in(hh, rhs, (size_t)h->nst, hh->stage_in, &bd));
    double* xd;
    AAO_TRY(stage_out_begin(x, hh->stage_out, &xd));
    if (x0_given && xd != x) {
        AAO_CUDA_TRY(cudaMemcpyAsync(xd, x, sizeof(double) * h->nst, cudaMemcpyHostToDevice, h->stream));
    }
    aao_status s = outer_solve(h, bd, xd, x0_given, 0, info, hh->sd);
    aao_status s2 = stage_out_end(hh, x, xd, (size_t)h->nst);
    return s != AAO_OK ? s : s2;
}

aao_status aao_rk_solve(aao_rk_handle hh, const double* f, int f_time_dep, const double* u0, double* x,
                        int x0_given, aao_info* info) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!f || !u0 || !x) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    const double *fd, *ud;
    AAO_TRY(stage_in(hh, f, f_time_dep ? (size_t)h->nt * h->s * h->nx : (size_t)h->nx, hh->stage_in, &fd));
    AAO_TRY(stage_in(hh, u0, (size_t)h->nx, hh->stage_aux, &ud));
    AAO_TRY(rhs_dev(h, fd, f_time_dep, ud, h->rhs));
    AAO_LAUNCH_CHECK();
    double* xd;
    AAO_TRY(stage_out_begin(x, hh->stage_out, &xd));
    if (x0_given && xd != x) {
        AAO_CUDA_TRY(cudaMemcpyAsync(xd, x, sizeof(double) * h->nst, cudaMemcpyHostToDevice, h->stream));
    }
    aao_status s = outer_solve(h, h->rhs, xd, x0_given, 0, info, hh->sd);
    aao_status s2 = stage_out_end(hh, x, xd, (size_t)h->nst);
    return s != AAO_OK ? s : s2;
}

aao_status aao_rk_adjoint_solve(aao_rk_handle hh, const double* dJdx, double* lambda, const double* x_fwd,
                                double* grad_f, double* grad_kappa, aao_info* info) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!dJdx || !lambda) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    if (grad_kappa && !x_fwd) {
        set_error("grad_kappa needs the forward solution");
        return AAO_ERR_ARG;
    }
    const double* bd;
    AAO_TRY(stage_in(hh, dJdx, (size_t)h->nst, hh->stage_in, &bd));
    double* ld;
    AAO_TRY(stage_out_begin(lambda, hh->stage_out, &ld));
    aao_status s = outer_solve(h, bd, ld, 0, 1, info, hh->sd);
    if (s != AAO_OK && s != AAO_ERR_NOT_CONVERGED) return s;
    if (grad_kappa && h->q1) {
        set_error("grad_kappa is defined for the finite-difference discretisation only");
        return AAO_ERR_UNSUPPORTED;
    }
    if (grad_f) {
        double* gd = is_device_ptr(grad_f) ? grad_f : h->w;
        if (h->q1) {
            // grad_f = M^T sum lambda_V = M sum lambda_V
            launch(k_grad_f, (unsigned)((h->nx + 255) / 256), 256, 0, h->stream, h->nx, h->nt, h->s, (const double*)ld,
                   h->xs);
            const PtMap pm = ptmap(h->g.n0);
            launch(k_apply_M_q1, pt_grid(pm, h->g.R, 1), pt_block(pm), 0, h->stream, h->g, pm, h->q1d,
                   (const double*)h->xs, gd);
        } else {
            launch(k_grad_f, (unsigned)((h->nx + 255) / 256), 256, 0, h->stream, h->nx, h->nt, h->s, ld, gd);
        }
        AAO_LAUNCH_CHECK();
        if (gd != grad_f) {
            AAO_CUDA_TRY(cudaMemcpyAsync(grad_f, gd, sizeof(double) * h->nx, cudaMemcpyDeviceToHost, h->stream));
        }
    }
    if (grad_kappa) {
        const double* xd;
        AAO_TRY(stage_in(hh, x_fwd, (size_t)h->nst, hh->stage_aux, &xd));
        const Geo& g = h->g;
        long long nnode = (long long)(g.n0 + 2) * (g.n1 + 2) * (g.d == 3 ? g.n2 + 2 : 1);
        double* gd = is_device_ptr(grad_kappa) ? grad_kappa : h->r;
        launch(k_grad_kappa, (unsigned)((nnode + 127) / 128), 128, 0, h->stream, g, h->nt, h->tab, h->tau,
               (const double*)ld, xd, gd, 0);
        AAO_LAUNCH_CHECK();
        if (gd != grad_kappa) {
            AAO_CUDA_TRY(cudaMemcpyAsync(grad_kappa, gd, sizeof(double) * nnode, cudaMemcpyDeviceToHost, h->stream));
        }
    }
    aao_status s2 = stage_out_end(hh, lambda, ld, (size_t)h->nst);
    AAO_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return s != AAO_OK ? s : s2;
}

aao_status aao_rk_grad_kappa(aao_rk_handle hh, const double* lambda, const double* x_fwd, double* grad_kappa,
                             int accumulate) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!lambda || !x_fwd || !grad_kappa) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    if (h->q1) {
        set_error("grad_kappa is defined for the finite-difference discretisation only");
        return AAO_ERR_UNSUPPORTED;
    }
    if (!is_device_ptr(lambda) || !is_device_ptr(x_fwd) || !is_device_ptr(grad_kappa)) {
        set_error("aao_rk_grad_kappa takes device vectors");
        return AAO_ERR_ARG;
    }
    const Geo& g = h->g;
    long long nnode = (long long)(g.n0 + 2) * (g.n1 + 2) * (g.d == 3 ? g.n2 + 2 : 1);
    launch(k_grad_kappa, (unsigned)((nnode + 127) / 128), 128, 0, h->stream, g, h->nt, h->tab, h->tau, lambda, x_fwd,
           grad_kappa, accumulate ? 1 : 0);
    AAO_LAUNCH_CHECK();
    return AAO_OK;
}

aao_status aao_rk_solve_batched(int nprob, const aao_rk_handle* hs, const double* const* f, const double* const* u0,
                                double* const* x, aao_info* infos) {
    if (nprob < 0 || (nprob > 0 && (!hs || !f || !u0 || !x))) {
        set_error("bad batched arguments");
        return AAO_ERR_ARG;
    }
    for (int p = 0; p < nprob; ++p)
        if (!hs[p]) {
            set_error("null handle in batch");
            return AAO_ERR_ARG;
        }
    {
        // a handle is not thread-safe: each may appear once
        std::vector<const void*> seen(hs, hs + nprob);
        std::sort(seen.begin(), seen.end());
        if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
            set_error("a handle appears more than once in the batch");
            return AAO_ERR_ARG;
        }
    }
    if (nprob == 0) return AAO_OK;
    if (g_prof_on) {
        // the launch profile's bookkeeping is not shared between threads
        set_error("batched solves run on several threads: close the launch profile first");
        return AAO_ERR_ARG;
    }
    int dev = 0;
    AAO_CUDA_TRY(cudaGetDevice(&dev));
    // Host worker threads, one per problem up to kMaxBatchThreads: every
    // problem's FGMRES loop (and its per-iteration convergence test) runs
    // independently, so the GPU overlaps the latency-bound Schur sweeps of
    // different problems.  Workers take problems largest first (space-time
    // unknowns), so a long problem does not start last.  Problems whose handles
    // share a stream serialise on that stream.
    std::vector<int> order(nprob);
    for (int p = 0; p < nprob; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->h.nst > hs[b]->h.nst; });
    std::vector<aao_status> st(nprob, AAO_OK);
    std::vector<std::string> err(nprob);
    std::atomic<int> next{0};
    auto work = [&]() {
        cudaSetDevice(dev);
        for (int q = next++; q < nprob; q = next++) {
            const int p = order[q];
            st[p] = aao_rk_solve(hs[p], f[p], 0, u0[p], x[p], 0, infos ? &infos[p] : nullptr);
            if (st[p] != AAO_OK) err[p] = get_error();
        }
    };
    std::vector<std::thread> th;
    const int nworkers = std::min(nprob, kMaxBatchThreads);
    th.reserve(nworkers);
    for (int w = 0; w < nworkers; ++w) {
        try {
            th.emplace_back(work);
        } catch (const std::exception&) {
            break;   // fewer workers: the ones running take the remaining problems
        }
    }
    if (th.empty()) work();   // no thread could be created: solve on the caller's thread
    for (auto& t : th) t.join();
    for (int p = 0; p < nprob; ++p)
        if (st[p] != AAO_OK) {
            set_error("problem " + std::to_string(p) + ": " + err[p]);
            return st[p];
        }
    return AAO_OK;
}

aao_status aao_rk_shifted_solve(aao_rk_handle hh, int stage, const double* b, double* x) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (stage < 0 || stage >= h->s || !b || !x) {
        set_error("bad stage or null vector");
        return AAO_ERR_ARG;
    }
    const double* bd;
    AAO_TRY(stage_in(hh, b, (size_t)h->nx, hh->stage_in, &bd));
    double* xd;
    AAO_TRY(stage_out_begin(x, hh->stage_out, &xd));
    AAO_TRY(h->P->shifted_solve(stage, bd, xd));
    return stage_out_end(hh, x, xd, (size_t)h->nx);
}

aao_status aao_rk_pint_apply(aao_rk_handle hh, const double* r, double* y, int transpose) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!r || !y) {
        set_error("null vector");
        return AAO_ERR_ARG;
    }
    size_t n = (size_t)h->s * h->nx;
    const double* rd;
    AAO_TRY(stage_in(hh, r, n, hh->stage_in, &rd));
    double* yd;
    AAO_TRY(stage_out_begin(y, hh->stage_out, &yd));
    AAO_TRY(h->P->pint_apply(rd, yd, transpose));
    return stage_out_end(hh, y, yd, n);
}

aao_status aao_rk_inner_solve(aao_rk_handle hh, int nblocks, const double* r, double* z, int* its) {
    H_CHECK(hh);
    Handle* h = &hh->h;
    if (!r || !z || nblocks < 1 || nblocks > h->nt) {
        set_error("null vector or nblocks outside 1..nt");
        return AAO_ERR_ARG;
    }
    size_t n = (size_t)nblocks * h->s * h->nx;
    const double* rd;
    AAO_TRY(stage_in(hh, r, n, hh->stage_in, &rd));
    double* zd;
    AAO_TRY(stage_out_begin(z, hh->stage_out, &zd));
    AAO_TRY(h->P->inner_solve(nblocks, rd, zd, its));
    return stage_out_end(hh, z, zd, n);
}

}  // extern "C"
