// aao_rk_shifted_solve_noalloc: the multigrid shifted solve x ~= (I + c K)^{-1} b
// without any device allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at all: code running inside a
// memory pool that forbids cudaMalloc, kernels-as-a-service hosts that only
// hand out pre-registered buffers, or applications that must not allocate
// after start-up.  For them this entry point keeps every piece of scratch
// (level vectors, Galerkin stencils, the coarsest dense inverse) in one
// file-scope __device__ array of fixed size, g_noalloc_scratch below.  Every
// GPU that loads the library holds that array until the process exits.
#include <cmath>
#include <mutex>

#include "handle.cuh"
#include "mg.cuh"

namespace aao {

// 5 MiB of FP64 scratch: enough for 2D grids of up to 256 x 256 points and 3D
// grids of up to 40^3 points (kNoAllocMaxPoints), with the hierarchy below.
constexpr long long kNoAllocDoubles = 655360;
constexpr long long kNoAllocMaxPoints = 65536;
constexpr int kNoAllocMaxCoarsest = kCoarsestTarget;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device (the
// first call on that device).  The address stays valid for the life of the
// device's primary context: after cudaDeviceReset it may be stale, so the
// allocation-free entry point must not be used across a device reset.
static double* g_noalloc_ptr[64] = {};
static std::mutex g_noalloc_mutex;

static aao_status noalloc_scratch(double** out) {
    int dev = 0;
    AAO_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal out of range");
        return AAO_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch) failed: ") + cudaGetErrorString(e));
            return AAO_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AAO_OK;
}

// Device (or managed) memory of the current device.  Memory of another GPU is
// refused: without peer access the kernels could not read it.
static bool device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
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

}  // namespace aao

using namespace aao;

extern "C" aao_status aao_rk_shifted_solve_noalloc(const aao_grid* grid, double c, int cycles, int pre, int post,
                                                   double omega, const double* b, double* x, void* stream) {
    if (!grid || !b || !x) {
        set_error("null argument");
        return AAO_ERR_ARG;
    }
    if (grid->dim != 2 && grid->dim != 3) {
        set_error("dim must be 2 or 3");
        return AAO_ERR_ARG;
    }
    if (grid->disc != AAO_DISC_FD || grid->kappa != nullptr) {
        set_error("the allocation-free solve supports the constant-coefficient FD grid only");
        return AAO_ERR_ARG;
    }
    if (!(c >= 0.0) || !std::isfinite(c) || cycles < 1 || pre < 0 || post < 0 || !(omega > 0.0) ||
        !std::isfinite(omega)) {
        set_error("need a finite c >= 0, cycles >= 1, pre/post >= 0 and a finite omega > 0");
        return AAO_ERR_ARG;
    }
    for (int a = 0; a < grid->dim; ++a)
        if (!(grid->len[a] > 0.0) || !std::isfinite(grid->len[a])) {
            set_error("grid lengths must be finite and positive");
            return AAO_ERR_ARG;
        }
    Geo g;
    g.d = grid->dim;
    g.n0 = grid->n[0];
    g.n1 = grid->n[1];
    g.n2 = g.d == 3 ? grid->n[2] : 1;
    if (g.n0 < 1 || g.n1 < 1 || g.n2 < 1) {
        set_error("grid sizes must be positive");
        return AAO_ERR_ARG;
    }
    g.nx = (long long)g.n0 * g.n1 * g.n2;
    g.R = g.n1 * g.n2;
    if (g.nx > kNoAllocMaxPoints) {
        set_error("grid too large for the allocation-free solve (at most 65536 points)");
        return AAO_ERR_ARG;
    }
    double hx = grid->len[0] / (g.n0 + 1), hy = grid->len[1] / (g.n1 + 1);
    double hz = g.d == 3 ? grid->len[2] / (g.n2 + 1) : 1.0;
    g.hx2 = 1.0 / (hx * hx);
    g.hy2 = 1.0 / (hy * hy);
    g.hz2 = g.d == 3 ? 1.0 / (hz * hz) : 0.0;
    if (!device_pointer(b) || !device_pointer(x)) {
        set_error("b and x must be device memory");
        return AAO_ERR_ARG;
    }
    // levels: coarsen every axis while the level has more than kCoarsestTarget points and each
    // axis keeps N/2 >= 2 (same hierarchy as the handle path)
    Geo lev[kMaxLevels];
    int L = 0;
    Geo cur = g;
    while (true) {
        lev[L++] = cur;
        bool more = cur.nx > kCoarsestTarget && cur.n0 / 2 >= 2 && cur.n1 / 2 >= 2 && (cur.d == 2 || cur.n2 / 2 >= 2);
        if (!more || L == kMaxLevels) break;
        Geo nx = cur;
        nx.n0 = cur.n0 / 2;
        nx.n1 = cur.n1 / 2;
        nx.n2 = cur.d == 3 ? cur.n2 / 2 : 1;
        nx.nx = (long long)nx.n0 * nx.n1 * nx.n2;
        nx.R = nx.n1 * nx.n2;
        cur = nx;
    }
    const int nc = (int)lev[L - 1].nx;
    if (nc > kNoAllocMaxCoarsest) {
        set_error("coarsest level too large for the allocation-free solve (anisotropic grid)");
        return AAO_ERR_ARG;
    }
    const int ncoef = g.d == 3 ? 27 : 9;
    // carve the scratch: per level T0, T1, Rr (and Bb, X below the finest), stencils, dense coarsest
    double* base = nullptr;
    AAO_TRY(noalloc_scratch(&base));
    long long off = 0;
    auto take = [&](long long n) {
        double* p = base + off;
        off += (n + 31) / 32 * 32;   // keep 256-byte alignment
        return p;
    };
    Vec<double> T0[kMaxLevels], T1[kMaxLevels], Rr[kMaxLevels], Bb[kMaxLevels], X[kMaxLevels];
    double* sten[kMaxLevels] = {};
    for (int l = 0; l < L; ++l) {
        long long n = lev[l].nx;
        T0[l] = Vec<double>{take(n), nullptr, n};
        T1[l] = Vec<double>{take(n), nullptr, n};
        Rr[l] = Vec<double>{take(n), nullptr, n};
        if (l > 0) {
            Bb[l] = Vec<double>{take(n), nullptr, n};
            X[l] = Vec<double>{take(n), nullptr, n};
            sten[l] = take(ncoef * n);
        }
    }
    double* dense = take((long long)nc * nc);
    double* dinv = take((long long)nc * nc);
    int* fail = reinterpret_cast<int*>(take(1));
    if (off > kNoAllocDoubles) {
        set_error("scratch requirement exceeds the allocation-free array");
        return AAO_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // Galerkin hierarchy of I + c K and the dense coarsest inverse (recomputed every call)
    FineDesc fd;
    fd.g = g;
    fd.fine = 1;
    fd.sigma = 1.0;
    fd.c = c;
    fd.faces = Faces<double>{};
    fd.sten = nullptr;
    for (int l = 1; l < L; ++l) {
        launch(k_galerkin, (unsigned)((lev[l].nx + 127) / 128), 128, 0, st, fd, lev[l], sten[l]);
        fd.g = lev[l];
        fd.fine = 0;
        fd.sigma = 0.0;
        fd.c = 0.0;
        fd.sten = sten[l];
    }
    launch(k_dense_level, (unsigned)((nc + 127) / 128), 128, 0, st, fd, dense);
    // the scratch keeps the previous call's contents: the breakdown flag must start at zero
    AAO_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), st));
    launch(k_gauss_jordan, 1, 1024, 0, st, dense, dinv, nc, fail);
    AAO_LAUNCH_CHECK();
    LevelOp<double> ops[kMaxLevels];
    for (int l = 0; l < L; ++l) {
        LevelOp<double>& op = ops[l];
        op.g = lev[l];
        op.ncoef = ncoef;
        if (l == 0) {
            op.fine = 1;
            op.sigma = 1.0;
            op.c = c;
        } else {
            op.fine = 0;
            op.sten = sten[l];
        }
    }
    Vec<double> bv{const_cast<double*>(b), nullptr, g.nx};
    Vec<double> xv{x, nullptr, g.nx};
    // V-cycle, level by level (same sweep order as the handle path)
    struct Rec {
        static aao_status run(int l, int L, Geo* lev, Vec<double> xin, Vec<double> bvec, Vec<double> xout,
                              Vec<double>* T0, Vec<double>* T1, Vec<double>* Rr, Vec<double>* Bb, Vec<double>* X,
                              const double* dinv, int pre, int post, double omega, cudaStream_t st,
                              const LevelOp<double>* ops) {
            const Geo& gl = lev[l];
            const PtMap pm = ptmap(gl.n0);
            if (l == L - 1) {
                launch(k_coarse_solve<double>, pt_grid(pm, gl.R, 1), pt_block(pm), 0, st, gl, pm, 1, (const int*)nullptr, dinv,
                       bvec, xout);
                AAO_LAUNCH_CHECK();
                return AAO_OK;
            }
            const LevelOp<double>& op = ops[l];
            const PtMap pmc = ptmap(lev[l + 1].n0);
            const int nops = pre + 1 + post;
            int opi = 0;
            Vec<double> cur = xin;
            auto dest = [&]() -> Vec<double> {
                ++opi;
                if (opi == nops) return xout;
                return cur.d == T0[l].d ? T1[l] : T0[l];
            };
            for (int q = 0; q < pre; ++q) {
                Vec<double> d = dest();
                launch(k_smooth<double>, pt_grid(pm, gl.R, 1), pt_block(pm), 0, st, op, pm, 1, (const int*)nullptr, cur,
                       bvec, d, omega);
                cur = d;
            }
            const Geo& gc = lev[l + 1];
            if (cur.d == nullptr) {
                launch(k_restrict<double>, pt_grid(pmc, gc.R, 1), pt_block(pmc), 0, st, gl, gc, pmc, 1, (const int*)nullptr, bvec,
                       Bb[l + 1]);
            } else {
                launch(k_residual<double>, pt_grid(pm, gl.R, 1), pt_block(pm), 0, st, op, pm, 1, (const int*)nullptr, cur, bvec,
                       Rr[l]);
                launch(k_restrict<double>, pt_grid(pmc, gc.R, 1), pt_block(pmc), 0, st, gl, gc, pmc, 1, (const int*)nullptr,
                       Rr[l], Bb[l + 1]);
            }
            AAO_LAUNCH_CHECK();
            AAO_TRY(run(l + 1, L, lev, Vec<double>{}, Bb[l + 1], X[l + 1], T0, T1, Rr, Bb, X, dinv, pre, post, omega,
                        st, ops));
            {
                Vec<double> d = dest();
                launch(k_prolong_add<double>, pt_grid(pm, gl.R, 1), pt_block(pm), 0, st, gl, gc, pm, 1, (const int*)nullptr,
                       X[l + 1], cur, d);
                cur = d;
            }
            for (int q = 0; q < post; ++q) {
                Vec<double> d = dest();
                launch(k_smooth<double>, pt_grid(pm, gl.R, 1), pt_block(pm), 0, st, op, pm, 1, (const int*)nullptr, cur,
                       bvec, d, omega);
                cur = d;
            }
            AAO_LAUNCH_CHECK();
            return AAO_OK;
        }
    };
    for (int cyc = 0; cyc < cycles; ++cyc) {
        AAO_TRY(Rec::run(0, L, lev, cyc == 0 ? Vec<double>{} : xv, bv, xv, T0, T1, Rr, Bb, X, dinv, pre, post,
                         omega, st, ops));
    }
    // the coarsest operator's inversion reports a zero or negative pivot in the flag: read it
    // back (the call therefore returns after its work on `stream` has finished)
    int hfail = 0;
    AAO_CUDA_TRY(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    AAO_CUDA_TRY(cudaStreamSynchronize(st));
    if (hfail) {
        set_error("coarsest multigrid operator is not positive definite");
        return AAO_ERR_BREAKDOWN;
    }
    return AAO_OK;
}
