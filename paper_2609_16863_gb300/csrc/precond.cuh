// P_tilde of Eq. (AppPrec) in storage precisions SP (Theta_tilde's GMRES basis
// and the S_tilde recurrence) and SI (Rana's sweep, V-cycles, coarse stencils).
// Arithmetic is double when SP is double, else float.
//
// apply(r):   z_V = Theta_tilde^{-1} r_V, all nt time blocks batched (inner
//             GMRES, right-preconditioned by P_int);
//             g_{n+1} = r_{v,n+1} + tau sum_i b_i z_{V,n,i}; w = M^{-1} g (FD: w = g);
//             z_{v,0} = w_0, z_{v,n+1} = w_{n+1} + z_{v,n} - tau (b^T (x) I)
//             Theta_tilde^{-1} (e (x) K z_{v,n})    (forward substitution, Eq. AppSchur).
// apply_T(r): u_nt = r_{v,nt}, u_n = r_{v,n} + u_{n+1} - tau (e^T (x) K)
//             Theta_tilde^{-T} (b (x) u_{n+1}); z_v = M^{-1} u;
//             z_V = Theta_tilde^{-T} (r_V + tau (b (x) M) z_{v,n+1}).
#pragma once

#include <algorithm>
#include <cstring>
#include <memory>
#include <type_traits>

#include "cluster_mg.cuh"
#include "handle.cuh"
#include "mg.cuh"

namespace aao {

template <class SP, class SI>
class Precond : public PrecondBase {
    using A = typename PT<SP>::A;
    static_assert(std::is_same<typename PT<SP>::A, typename PT<SI>::A>::value,
                  "P and P_int arithmetic must agree");

    struct Level {
        Geo g;
        // per-stage stored stencils (levels >= 1)
        SI* sten[kMaxS] = {};
        float* sten_sc[kMaxS] = {};
        // scratch, Bmax items of nx each
        Vec<SI> T0, T1, Rr, Bb, X;
    };

    Handle* h;
    Arena ar;
    int Bmax = 0;
    int L = 0;
    Level lev[kMaxLevels];
    A* Dinv[kMaxS] = {};           // dense coarsest inverse per stage
    Faces<A> facesA;
    SpaceOp<A> sopA;                 // fine-grid K (and M for Q1) for the stage kernels
    A* cheb[3] = {};                 // Q1: Chebyshev x, r, d ((nt+1)*nx each)
    int kin = 0;                   // inner maxit
    double itol = 0.0;
    // inner GMRES state
    Vec<SP> V0;                    // (kin+1) bases, stride vstride elements
    long long vstride = 0;
    Vec<SI> Z0;                    // kin bases, stride zstride
    long long zstride = 0;
    A* wv = nullptr;               // Bmax * s*nx
    Vec<SI> mgb;                   // Rana rhs, Bmax * nx
    double *Hh = nullptr, *csh = nullptr, *snh = nullptr, *gh = nullptr, *yh = nullptr, *betah = nullptr;
    int *activeh = nullptr, *itsh = nullptr, *nonfin = nullptr, *brk = nullptr;
    long long* itcount = nullptr;  // running total of inner iterations (device)
    // Schur state
    A* wbuf = nullptr;             // (nt+1)*nx
    A* tbuf = nullptr;             // s*nx
    A* qbuf = nullptr;             // s*nx
    A* tV = nullptr;               // nt*s*nx (transposed apply)
    double* tmp64 = nullptr;       // Bmax*s*nx staging for component entry points
    cudaEvent_t e0, e1, e2;
    int nact = 0;                  // active items of the current batch (exact only while profiling)
    // Fused on-chip tail: two variants, for single-item V-cycles (the Schur
    // sweep, where a smaller tail plus fused level kernels is faster) and for
    // batched V-cycles (every item's tail on its own SM).
    struct Tail {
        int lc = 0;                // first level handled by the tail kernel
        size_t smem = 0;
        TailCtx<SI> ctx[kMaxS];
    };
    Tail tails[2];                 // [0]: B == 1, [1]: B > 1
    int tail_threads = 1024;
    // Cluster-resident shifted solves for single 2D items (the Schur sweep).
    int cl_C = 0;                  // CTAs per cluster of the single-item plan; 0: no cluster plan
    struct ClPlan {
        int C = 0;                 // CTAs per cluster; 0: none
        size_t smem = 0;
        ClCtx<SI>* ctx = nullptr;  // device, one context per stage
    };
    ClPlan clp[2];                 // [0] single items, [1] batches of at least kClBatch8 items
    int* hact = nullptr;           // pinned mirror of activeh (profiling)

    cudaStream_t cur_stream = nullptr;     // stream of the next launch (capture stream while capturing)
    cudaStream_t cap_stream = nullptr;
    // one captured graph per step kind [transpose][kind]: 0 one time step, 1 a batched MGRIT
    // relaxation step, 2 the batched C-point residual step, 3 a batched relaxation step that also
    // relaxes the shorter final interval (mg_r > 0)
    cudaGraphExec_t gexec[2][4] = {};
    long long graph_nodes[2][4] = {};
    StepPtrs* stepp = nullptr;
    // two-level MGRIT for S_tilde's recurrence (mg_m = 0: forward substitution): the coarse
    // propagator is the substitution step of a second preconditioner built for step size
    // mg_m tau and mg_nc = nt / mg_m (rounded down) steps; C-points are the multiples of mg_m, and
    // the mg_r = nt - mg_nc mg_m steps after the last one form a shorter final interval
    int mg_m = 0, mg_nc = 0, mg_r = 0;
    std::unique_ptr<Handle> hc;
    Precond* coarse = nullptr;
    double* ebuf = nullptr;        // (nc+1)*nx: coarse error recurrence
    double* rbufT = nullptr;       // (nc+1)*nx: transposed C-point residuals (the coarse source)
    // The intervals' recurrences run as single-item steps on worker preconditioners (same
    // operators, one stream each, their own Krylov and reduction workspace; they read this
    // preconditioner's w), ordered by events: the dataflow of one two-level MGRIT iteration.
    static constexpr int kMaxWorkers = 16;
    int nwork = 0;
    std::unique_ptr<Handle> hw[kMaxWorkers];
    Precond* work[kMaxWorkers] = {};
    cudaStream_t wst[kMaxWorkers] = {};
    cudaEvent_t ev_start = nullptr, ev_join[kMaxWorkers] = {};
    std::vector<cudaEvent_t> ev_f1, ev_c;    // per interval: first relaxation done, C-point corrected
    const A* wsrc = nullptr;       // a worker's source w (the owner's wbuf); nullptr: its own

    cudaStream_t st() const { return cur_stream; }

    // While a launch profile is open, read back how many batch items are still
    // active so the byte hints count only the work that is done.
    void refresh_nact(int B) {
        nact = B;
        if (!g_prof_on || !hact) return;
        cudaMemcpyAsync(hact, activeh, sizeof(int) * B, cudaMemcpyDeviceToHost, st());
        cudaStreamSynchronize(st());
        int c = 0;
        for (int b = 0; b < B; ++b) c += hact[b] != 0;
        nact = c;
    }

    template <class S> aao_status alloc_vec(Vec<S>& v, long long items, long long item_len, int n0) {
        AAO_TRY(ar.alloc(&v.d, (size_t)(items * item_len)));
        v.bs = item_len;
        v.sc = nullptr;
        if (PT<S>::scaled) AAO_TRY(ar.alloc(&v.sc, (size_t)(items * item_len / n0)));
        return AAO_OK;
    }

  public:
    explicit Precond(Handle* hh) : h(hh), cur_stream(hh->stream) {}
    ~Precond() override { release(); }

    void release() override {
        if (coarse) delete coarse;
        coarse = nullptr;
        hc.reset();
        for (int w = 0; w < kMaxWorkers; ++w) {
            if (work[w]) delete work[w];
            work[w] = nullptr;
            hw[w].reset();
            if (wst[w]) cudaStreamDestroy(wst[w]);
            wst[w] = nullptr;
            if (ev_join[w]) cudaEventDestroy(ev_join[w]);
            ev_join[w] = nullptr;
        }
        nwork = 0;
        for (cudaEvent_t e : ev_f1) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_c) cudaEventDestroy(e);
        ev_f1.clear();
        ev_c.clear();
        if (ev_start) cudaEventDestroy(ev_start);
        ev_start = nullptr;
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 4; ++k) {
                if (gexec[i][k]) cudaGraphExecDestroy(gexec[i][k]);
                gexec[i][k] = nullptr;
            }
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cap_stream = nullptr;
        ar.release();
        if (hact) cudaFreeHost(hact);
        hact = nullptr;
    }

    aao_status setup() override {
        const Geo& g0 = h->g;
        const int s = h->s;
        if (PT<SI>::scaled || PT<SP>::scaled) {
            if (g0.n0 > kMaxRowLen) {
                set_error("16-bit storage needs n[0] <= 512");
                return AAO_ERR_ARG;
            }
        }
        Bmax = h->nt;
        kin = h->opt.inner_maxit;
        itol = h->opt.inner_tol;
        // ---- levels
        L = 0;
        Geo g = g0;
        while (true) {
            lev[L].g = g;
            ++L;
            bool more = g.nx > kCoarsestTarget && g.n0 / 2 >= 2 && g.n1 / 2 >= 2 && (g.d == 2 || g.n2 / 2 >= 2);
            if (!more || L == kMaxLevels) break;
            Geo c = g;
            c.n0 = g.n0 / 2;
            c.n1 = g.n1 / 2;
            c.n2 = g.d == 3 ? g.n2 / 2 : 1;
            c.nx = (long long)c.n0 * c.n1 * c.n2;
            c.R = c.n1 * c.n2;
            g = c;
        }
        if (lev[L - 1].g.nx > kMaxCoarsest) {
            set_error("coarsest multigrid level too large (anisotropic grid?)");
            return AAO_ERR_ARG;
        }
        // ---- faces in arithmetic precision
        if (h->has_kappa) {
            long long nfx = (long long)(g0.n0 + 1) * g0.R;
            long long nfy = (long long)g0.n0 * (g0.n1 + 1) * g0.n2;
            long long nfz = g0.d == 3 ? (long long)g0.nx / g0.n2 * (g0.n2 + 1) : 0;
            A *fx, *fy, *fz = nullptr;
            AAO_TRY(ar.alloc(&fx, nfx));
            AAO_TRY(ar.alloc(&fy, nfy));
            if (nfz) AAO_TRY(ar.alloc(&fz, nfz));
            launch(k_convert<double, A>, (unsigned)((nfx + 255) / 256), 256, 0, st(), h->faces64.fx, fx, nfx);
            launch(k_convert<double, A>, (unsigned)((nfy + 255) / 256), 256, 0, st(), h->faces64.fy, fy, nfy);
            if (nfz) launch(k_convert<double, A>, (unsigned)((nfz + 255) / 256), 256, 0, st(), h->faces64.fz, fz, nfz);
            AAO_LAUNCH_CHECK();
            facesA.fx = fx;
            facesA.fy = fy;
            facesA.fz = fz;
        }
        sopA.faces = facesA;
        sopA.q1 = h->q1;
        if (h->q1) {
            for (int a = 0; a < 3; ++a)
                for (int e = 0; e < 3; ++e) {
                    sopA.q.m[a][e] = (A)h->q1d.m[a][e];
                    sopA.q.k[a][e] = (A)h->q1d.k[a][e];
                }
        }
        // ---- Galerkin hierarchy per stage shift c_i = tau d_i
        const int ncoef = g0.d == 3 ? 27 : 9;
        double* sten0 = nullptr;             // Q1: stored fine-level stencil of M + c K (FP64)
        if (h->q1) AAO_TRY(ar.alloc(&sten0, (size_t)(ncoef * g0.nx)));
        double* sten64[kMaxLevels] = {};
        for (int l = 1; l < L; ++l) AAO_TRY(ar.alloc(&sten64[l], (size_t)(ncoef * lev[l].g.nx)));
        const Geo& gcst = lev[L - 1].g;
        const int ncst = (int)gcst.nx;
        double *dense, *dinv64;
        int* fail;
        AAO_TRY(ar.alloc(&dense, (size_t)ncst * ncst));
        AAO_TRY(ar.alloc(&dinv64, (size_t)ncst * ncst));
        AAO_TRY(ar.alloc(&fail, 1));
        AAO_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int), st()));
        for (int i = 0; i < s; ++i) {
            FineDesc fd;
            fd.g = g0;
            fd.fine = 1;
            fd.sigma = 1.0;
            fd.c = h->tau * h->D[i];
            fd.faces = h->faces64;
            fd.sten = nullptr;
            if (h->q1) {
                launch(k_q1_stencil, (unsigned)((g0.nx + 127) / 128), 128, 0, st(), g0, h->q1d, h->tau * h->D[i],
                       sten0);
                AAO_LAUNCH_CHECK();
                AAO_TRY(store_stencil(0, i, sten0, ncoef));
                fd.fine = 0;
                fd.sigma = 0.0;
                fd.c = 0.0;
                fd.sten = sten0;
            }
            for (int l = 1; l < L; ++l) {
                launch(k_galerkin, (unsigned)((lev[l].g.nx + 127) / 128), 128, 0, st(), fd, lev[l].g, sten64[l]);
                AAO_LAUNCH_CHECK();
                AAO_TRY(store_stencil(l, i, sten64[l], ncoef));
                FineDesc nd;
                nd.g = lev[l].g;
                nd.fine = 0;
                nd.sigma = 0;
                nd.c = 0;
                nd.sten = sten64[l];
                fd = nd;   // level l+1 is the Galerkin product of this level
            }
            // coarsest dense inverse from the FP64 description of level L-1
            FineDesc cd;
            if (L == 1) {
                cd.g = g0;
                cd.fine = h->q1 ? 0 : 1;
                cd.sigma = h->q1 ? 0.0 : 1.0;
                cd.c = h->q1 ? 0.0 : h->tau * h->D[i];
                cd.faces = h->faces64;
                cd.sten = h->q1 ? sten0 : nullptr;
            } else {
                cd.g = gcst;
                cd.fine = 0;
                cd.sigma = 0;
                cd.c = 0;
                cd.sten = sten64[L - 1];
            }
            launch(k_dense_level, (unsigned)((ncst + 127) / 128), 128, 0, st(), cd, dense);
            launch(k_gauss_jordan, 1, 1024, 0, st(), dense, dinv64, ncst, fail);
            AAO_LAUNCH_CHECK();
            AAO_TRY(ar.alloc(&Dinv[i], (size_t)ncst * ncst));
            launch(k_convert_dense<A>, (unsigned)(((long long)ncst * ncst + 255) / 256), 256, 0, st(), 
                dinv64, Dinv[i], (long long)ncst * ncst);
            AAO_LAUNCH_CHECK();
        }
        int hfail = 0;
        AAO_CUDA_TRY(cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st()));
        AAO_CUDA_TRY(cudaStreamSynchronize(st()));
        if (hfail) {
            set_error("coarsest multigrid operator is not positive definite");
            return AAO_ERR_BREAKDOWN;
        }
        // ---- fused tails: the coarsest levels that fit on one SM
        int optin = 0;
        {
            int dev = 0;
            AAO_CUDA_TRY(cudaGetDevice(&dev));
            AAO_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        }
        for (int v = 0; v < 2; ++v) AAO_TRY(build_tail(tails[v], v == 0 ? kTailMaxPointsSingle : kTailMaxPoints, optin));
        // the attribute is per kernel for the whole process: always set the device's
        // opt-in maximum so that handles with larger tails keep working
        AAO_CUDA_TRY(cudaFuncSetAttribute(k_vcycle_tail<SI>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        AAO_CUDA_TRY(cudaFuncSetAttribute(k_vcycle_tail_2d<SI>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        AAO_TRY(build_cluster(optin));
        // ---- level scratch
        for (int l = 0; l < L; ++l) {
            const Geo& gl = lev[l].g;
            AAO_TRY(alloc_vec(lev[l].T0, Bmax, gl.nx, gl.n0));
            AAO_TRY(alloc_vec(lev[l].T1, Bmax, gl.nx, gl.n0));
            AAO_TRY(alloc_vec(lev[l].Rr, Bmax, gl.nx, gl.n0));
            if (l > 0) {
                AAO_TRY(alloc_vec(lev[l].Bb, Bmax, gl.nx, gl.n0));
                AAO_TRY(alloc_vec(lev[l].X, Bmax, gl.nx, gl.n0));
            }
        }
        // ---- inner GMRES state
        const long long item = (long long)s * g0.nx;
        vstride = (long long)Bmax * item;
        zstride = vstride;
        AAO_TRY(alloc_vec(V0, (long long)(kin + 1) * Bmax, item, g0.n0));
        V0.bs = item;
        AAO_TRY(alloc_vec(Z0, (long long)kin * Bmax, item, g0.n0));
        Z0.bs = item;
        AAO_TRY(ar.alloc(&wv, (size_t)(Bmax * item)));
        AAO_TRY(alloc_vec(mgb, Bmax, g0.nx, g0.n0));
        AAO_TRY(ar.alloc(&Hh, (size_t)Bmax * (kin + 1) * kin));
        AAO_TRY(ar.alloc(&csh, (size_t)Bmax * kin));
        AAO_TRY(ar.alloc(&snh, (size_t)Bmax * kin));
        AAO_TRY(ar.alloc(&gh, (size_t)Bmax * (kin + 1)));
        AAO_TRY(ar.alloc(&yh, (size_t)Bmax * kin));
        AAO_TRY(ar.alloc(&betah, (size_t)Bmax));
        AAO_TRY(ar.alloc(&activeh, (size_t)Bmax));
        AAO_TRY(ar.alloc(&itsh, (size_t)Bmax));
        AAO_TRY(ar.alloc(&nonfin, 2));
        brk = nonfin + 1;
        AAO_TRY(ar.alloc(&itcount, 1));
        AAO_CUDA_TRY(cudaMemsetAsync(nonfin, 0, 2 * sizeof(int), st()));
        AAO_CUDA_TRY(cudaMemsetAsync(itcount, 0, sizeof(long long), st()));
        // ---- Schur state
        if (h->opt.mgrit_m > 0) {
            mg_m = h->opt.mgrit_m;
            mg_nc = h->nt / mg_m;
            mg_r = h->nt - mg_nc * mg_m;
        }
        const long long steps_b = std::max(mg_nc + (mg_r > 0 ? 1 : 0), 1);     // items of a batched step
        AAO_TRY(ar.alloc(&wbuf, (size_t)((h->nt + 1) * g0.nx)));
        AAO_TRY(ar.alloc(&tbuf, (size_t)(steps_b * item)));
        AAO_TRY(ar.alloc(&qbuf, (size_t)(steps_b * item)));
        AAO_TRY(ar.alloc(&tV, (size_t)(h->nt * item)));
        AAO_TRY(ar.alloc(&tmp64, (size_t)(Bmax * item)));
        AAO_TRY(ar.alloc(&stepp, 1));
        if (h->q1)
            for (int i = 0; i < 3; ++i) AAO_TRY(ar.alloc(&cheb[i], (size_t)((h->nt + 1) * g0.nx)));
        AAO_CUDA_TRY(cudaEventCreate(&e0));
        AAO_CUDA_TRY(cudaEventCreate(&e1));
        AAO_CUDA_TRY(cudaEventCreate(&e2));
        AAO_CUDA_TRY(cudaMallocHost((void**)&hact, sizeof(int) * Bmax));
        if (mg_m > 0) {
            // the coarse level of MGRIT: the same operators with step mg_m tau over mg_nc steps
            hc.reset(new Handle(*h));
            hc->arena = Arena();
            hc->P = nullptr;
            hc->nt = mg_nc;
            hc->tau = mg_m * h->tau;
            hc->nv = (long long)(mg_nc + 1) * g0.nx;
            hc->nst = hc->nv + (long long)mg_nc * s * g0.nx;
            hc->opt.mgrit_m = 0;
            coarse = new Precond(hc.get());
            AAO_TRY(coarse->setup());
            AAO_TRY(ar.alloc(&ebuf, (size_t)((mg_nc + 1) * g0.nx)));
            AAO_TRY(ar.alloc(&rbufT, (size_t)((mg_nc + 1) * g0.nx)));
            // the dataflow schedule needs no clusters: with a cluster plan the lock-step schedule runs
            nwork = cl_C > 0 ? 0 : std::min(mg_nc, (int)kMaxWorkers);
            for (int w = 0; w < nwork; ++w) {
                AAO_CUDA_TRY(cudaStreamCreateWithFlags(&wst[w], cudaStreamNonBlocking));
                AAO_CUDA_TRY(cudaEventCreateWithFlags(&ev_join[w], cudaEventDisableTiming));
                hw[w].reset(new Handle(*h));
                Handle* q = hw[w].get();
                q->arena = Arena();
                q->P = nullptr;
                q->nt = 1;
                q->nv = 2 * g0.nx;
                q->nst = q->nv + (long long)s * g0.nx;
                q->opt.mgrit_m = 0;
                q->stream = wst[w];
                // a worker's reductions run concurrently with the others': its own scratch
                q->red_cap_items = 1;
                AAO_TRY(ar.alloc(&q->red.partials, (size_t)(q->red_cap_chunks + 1 + 16)));
                AAO_TRY(ar.alloc(&q->red.count, 1));
                AAO_CUDA_TRY(cudaMemsetAsync(q->red.count, 0, sizeof(unsigned int), st()));
                work[w] = new Precond(q);
                AAO_TRY(work[w]->setup());
                work[w]->wsrc = wbuf;
            }
            ev_f1.assign(mg_nc, nullptr);
            ev_c.assign(mg_nc + 1, nullptr);
            for (auto& e : ev_f1) AAO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            for (auto& e : ev_c) AAO_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            AAO_CUDA_TRY(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
        }
        AAO_CUDA_TRY(cudaStreamSynchronize(st()));
        return AAO_OK;
    }

    // Choose the tail's top level (at most max_points points, shared memory within the
    // device limit) and fill its per-stage contexts.
    aao_status build_tail(Tail& T, long long max_points, int optin) {
        const Geo& g0 = h->g;
        const int s = h->s;
        const size_t cap = 200 * 1024;
        const int ncf = g0.d == 3 ? 27 : 9;
        int lc = L - 1;
        size_t acc = 0;
        for (int l = L - 1; l >= 0; --l) {
            acc += 3 * (size_t)lev[l].g.nx * sizeof(A);
            if (lev[l].g.nx > max_points || lev[l].g.nx > (long long)kTailPmax * tail_threads || acc > cap) break;
            lc = l;
        }
        size_t vec_bytes = 0;
        for (int l = lc; l < L; ++l) vec_bytes += 3 * (size_t)lev[l].g.nx * sizeof(A);
        vec_bytes = (vec_bytes + 15) / 16 * 16;
        // stage as many of the coarsest stencils as fit next to the vectors
        int stage_from = L;
        size_t sb = 0;
        for (int l = L - 1; l >= (lc > 1 ? lc : 1); --l) {
            size_t add = ((size_t)ncf * lev[l].g.nx * sizeof(SI) + 15) / 16 * 16;
            if (vec_bytes + sb + add > cap) break;
            sb += add;
            stage_from = l;
        }
        T.lc = lc;
        T.smem = vec_bytes + sb;
        if ((long long)T.smem > optin) {
            set_error("fused multigrid tail does not fit in shared memory");
            return AAO_ERR_ARG;
        }
        for (int i = 0; i < s; ++i) {
            TailCtx<SI>& t = T.ctx[i];
            t.lc = lc;
            t.L = L;
            int o = 0;
            for (int l = lc; l < L; ++l) {
                t.op[l] = level_op(l, i);
                t.off[l] = o;
                o += 3 * (int)lev[l].g.nx;
            }
            t.vec_bytes = (int)vec_bytes;
            t.stage_from = stage_from;
            size_t so = vec_bytes;
            for (int l = 0; l < kMaxLevels; ++l) t.sten_off[l] = 0;
            for (int l = stage_from; l < L; ++l) {
                t.sten_off[l] = (int)so;
                so += ((size_t)ncf * lev[l].g.nx * sizeof(SI) + 15) / 16 * 16;
            }
            t.Dinv = Dinv[i];
            t.omega = (A)h->opt.mg_omega;
            t.nu1 = h->opt.mg_pre;
            t.nu2 = h->opt.mg_post;
        }
        return AAO_OK;
    }

    // Plan the cluster-resident shifted solve: 2D, at least one level above the coarsest, every
    // CTA owning rows of every distributed level, its share within shared memory, and the cluster
    // co-resident on the device.  Two plans: one for single items (16 CTAs where the full layout
    // fits, else 8) and one for batches (8 CTAs, so that about twice as many items run at once:
    // at 256^2 only 7 clusters of 16 are resident).  A plan that does not fit shared memory is made
    // lean step by step: level 0's Jacobi weight as a scalar (FD, kappa = 1), the rows of A_c^{-1}
    // read from global memory, then the coarse stencils read from global memory (L2) from level 1
    // on (only where the storage type is the arithmetic type).  Lean plans give the same values.
    bool plan_cluster(int C, int lean, long long dyn_max, ClCtx<SI>& t, long long& bytes) {
        const Geo& g0 = h->g;
        const int T = L - 1;
        if (g0.n1 < C) return false;
        const bool fine0 = !h->q1;
        const bool faces = fine0 && h->has_kappa;
        const bool same = std::is_same<SI, A>::value;
        const bool w0c = lean >= 1 && fine0 && !faces;
        // lean >= 2 reads coarse stencils from global memory: in place where the storage type is the
        // arithmetic type, else (16-bit storage) through the vector steps only, so those levels
        // must take vectors (checked below)
        std::memset(&t, 0, sizeof(t));
        t.C = C;
        t.L = L;
        t.T = T;
        t.cycles = h->opt.mg_cycles;
        t.nu1 = h->opt.mg_pre;
        t.nu2 = h->opt.mg_post;
        t.omega = (A)h->opt.mg_omega;
        t.sigma = A(1);
        t.fine0 = fine0 ? 1 : 0;
        t.has_faces = faces ? 1 : 0;
        t.fx = facesA.fx;
        t.fy = facesA.fy;
        t.w0_const = w0c ? 1 : 0;
        t.dinv_global = lean >= 1 ? 1 : 0;

        long long o = 0;
        auto take = [&](long long n) {
            long long at = o;
            o += (n + 3) / 4 * 4;
            return (int)at;
        };
        // Every CTA must own at least one row of every distributed level: a CTA whose coarse
        // range is empty would interpolate from coarse ghost rows that no neighbour stores to
        // (neighbours push only to non-empty CTAs).  Grids with few rows for their width
        // (e.g. 120 x 17 at C = 16) fail this and take a smaller cluster or the level kernels.
        bool nonempty = true;
        for (int l = 0; l < L; ++l) {
            const Geo& gl = lev[l].g;
            t.g[l] = gl;
            t.magic[l] = (unsigned)((4294967296ULL + (unsigned long long)gl.n0 - 1) / (unsigned long long)gl.n0);
            // 16-byte vectors of points: the FD level 0 with kappa = 1 and every stored-stencil level
            constexpr int VN = (int)(16 / sizeof(A));
            const bool stencil_level = l >= 1 || !fine0;
            t.vec[l] = (l < L - 1 && gl.n0 % VN == 0 && (stencil_level || !faces)) ? 1 : 0;
            const unsigned long long nv = (unsigned long long)(gl.n0 / VN > 0 ? gl.n0 / VN : 1);
            t.magicv[l] = (unsigned)((4294967296ULL + nv - 1) / nv);
            if (l < T) {
                for (int r = 0; r <= C; ++r)
                    t.rlo[l][r] = l == 0 ? (int)((long long)r * gl.n1 / C) : t.rlo[l - 1][r] / 2;
                int mr = 0;
                for (int r = 0; r < C; ++r) {
                    mr = std::max(mr, t.rlo[l][r + 1] - t.rlo[l][r]);
                    nonempty = nonempty && t.rlo[l][r + 1] > t.rlo[l][r];
                }
                t.maxr[l] = std::max(mr, 1);
            } else {
                t.maxr[l] = gl.n1;
            }
            t.off[l] = take(3LL * (t.maxr[l] + 2) * (gl.n0 + 2 * kClPad));
        }
        if (!nonempty) return false;
        for (int l = 1; l < L - 1; ++l) {
            t.sten_global[l] = (lean >= 3 || (lean == 2 && l == 1)) ? 1 : 0;
            if (t.sten_global[l] && !same && !t.vec[l]) return false;
        }
        for (int l = 0; l < L; ++l) {
            t.soff[l] = t.woff[l] = -1;
            if ((l >= 1 || !fine0) && l < L - 1 && !t.sten_global[l]) t.soff[l] = take(9LL * t.maxr[l] * lev[l].g.n0);
            if (l < L - 1 && !(l == 0 && w0c)) t.woff[l] = take((long long)t.maxr[l] * lev[l].g.n0);
        }
        t.fxoff = t.fyoff = -1;
        if (faces) {
            t.fxoff = take((long long)t.maxr[0] * (g0.n0 + 1));
            t.fyoff = take((long long)(t.maxr[0] + 1) * g0.n0);
        }
        const long long ncst = lev[L - 1].g.nx;
        int msl = 0;
        for (int r = 0; r <= C; ++r) t.cs[r] = (int)((long long)r * ncst / C);
        for (int r = 0; r < C; ++r) msl = std::max(msl, t.cs[r + 1] - t.cs[r]);
        t.dinv_off = t.dinv_global ? -1 : take((long long)msl * ncst);
        t.rowtab_off = take(((long long)lev[T - 1].g.n1 * (long long)sizeof(void*) + sizeof(A) - 1) / sizeof(A));
        bytes = o * (long long)sizeof(A);
        if (bytes > dyn_max) return false;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = (size_t)bytes;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_cluster_mg<SI>, &cfg) != cudaSuccess || nclusters < 1) {
            cudaGetLastError();
            return false;
        }
        return true;
    }

    aao_status store_cluster_plan(ClPlan& pl, const ClCtx<SI>& t, long long bytes) {
        ClCtx<SI> hc[kMaxS];
        for (int i = 0; i < h->s; ++i) {
            hc[i] = t;
            hc[i].c = (A)(h->tau * h->D[i]);
            for (int l = 0; l < L; ++l) {
                hc[i].sten[l] = lev[l].sten[i];
                hc[i].sten_sc[l] = lev[l].sten_sc[i];
            }
            hc[i].Dinv = Dinv[i];
        }
        AAO_TRY(ar.alloc(&pl.ctx, (size_t)h->s));
        AAO_CUDA_TRY(cudaMemcpy(pl.ctx, hc, sizeof(ClCtx<SI>) * h->s, cudaMemcpyHostToDevice));
        pl.C = t.C;
        pl.smem = (size_t)bytes;
        return AAO_OK;
    }

    aao_status build_cluster(int optin) {
        cl_C = 0;
        clp[0] = clp[1] = ClPlan{};
        const Geo& g0 = h->g;
        if (g0.d != 2 || L < 2) return AAO_OK;
        cudaFuncAttributes fa;
        AAO_CUDA_TRY(cudaFuncGetAttributes(&fa, k_cluster_mg<SI>));
        const long long dyn_max = (long long)optin - (long long)fa.sharedSizeBytes;
        if (dyn_max <= 0) return AAO_OK;
        AAO_CUDA_TRY(cudaFuncSetAttribute(k_cluster_mg<SI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max));
        AAO_CUDA_TRY(cudaFuncSetAttribute(k_cluster_mg<SI>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        ClCtx<SI> t;
        long long bytes = 0;
        // single items: the full layout first (staged once per launch), 16 CTAs before 8
        bool found = false;
        for (int C : {16, 8}) {
            for (int lean = 0; lean <= 3 && !found; ++lean) found = plan_cluster(C, lean, dyn_max, t, bytes);
            if (found) break;
        }
        if (!found) return AAO_OK;
        AAO_TRY(store_cluster_plan(clp[0], t, bytes));
        // batches: 8 CTAs per item, the leanest layout that fits
        if (clp[0].C == 8) {
            clp[1] = clp[0];
        } else {
            bool fb = false;
            for (int lean = 0; lean <= 3 && !fb; ++lean) fb = plan_cluster(8, lean, dyn_max, t, bytes);
            if (fb) AAO_TRY(store_cluster_plan(clp[1], t, bytes));
        }
        cl_C = clp[0].C;
        return AAO_OK;
    }

    // Keep the FP64 stencil of level l (shift `stage`) in the P_int storage type.
    aao_status store_stencil(int l, int i, const double* s64, int ncoef) {
        const long long n = (long long)ncoef * lev[l].g.nx;
        if constexpr (std::is_same<SI, double>::value) {
            SI* keep;
            AAO_TRY(ar.alloc(&keep, (size_t)n));
            AAO_CUDA_TRY(cudaMemcpyAsync(keep, s64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st()));
            lev[l].sten[i] = keep;
        } else {
            float* sc;
            AAO_TRY(ar.alloc(&sc, ncoef));
            if (PT<SI>::scaled) {
                launch(k_stencil_absmax, ncoef, kBlock, 0, st(), s64, lev[l].g.nx, sc);
            } else {
                AAO_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(float) * ncoef, st()));
            }
            SI* out;
            AAO_TRY(ar.alloc(&out, (size_t)n));
            launch(k_stencil_convert<SI>, (unsigned)((n + 255) / 256), 256, 0, st(), s64, lev[l].g.nx, ncoef,
                   (const float*)sc, out);
            AAO_LAUNCH_CHECK();
            lev[l].sten[i] = out;
            lev[l].sten_sc[i] = sc;
        }
        return AAO_OK;
    }

    // Q1: buf <- M^{-1} buf for B blocks of n_x by `cheb_steps` Chebyshev steps
    // with Jacobi splitting on the spectrum bounds [2^-d, (3/2)^d] of D^{-1}M.
    aao_status mass_inverse(A* buf, int B) {
        const Geo& g = h->g;
        const long long n = (long long)B * g.nx;
        const double lo = std::pow(0.5, g.d), hi = std::pow(1.5, g.d);
        const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
        double dinv = 1.0;
        for (int a = 0; a < g.d; ++a) dinv /= h->q1d.m[a][1];
        double rho = 1.0 / sigma;
        const unsigned nb = (unsigned)((n + 255) / 256);
        const PtMap pm = ptmap(g.n0);
        launch(k_cheb_init<A>, nb, 256, 0, st(), n, (const A*)buf, (A)(dinv / theta), cheb[0], cheb[1], cheb[2]);
        for (int it = 0; it < h->opt.cheb_steps; ++it) {
            launch(k_cheb_a<A>, pt_grid(pm, g.R, B), pt_block(pm), 0, st(), g, pm, B, sopA.q,
                   (const A*)cheb[2], cheb[0], cheb[1]);
            const double rn = 1.0 / (2.0 * sigma - rho);
            launch(k_cheb_b<A>, nb, 256, 0, st(), n, (A)(rn * rho), (A)(2.0 * rn / delta * dinv), (const A*)cheb[1],
                   cheb[2]);
            rho = rn;
        }
        AAO_CUDA_TRY(cudaMemcpyAsync(buf, cheb[0], sizeof(A) * n, cudaMemcpyDeviceToDevice, st()));
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    // ---------------------------------------------------------------- MG
    LevelOp<SI> level_op(int l, int stage) const {
        LevelOp<SI> op;
        op.g = lev[l].g;
        op.ncoef = op.g.d == 3 ? 27 : 9;
        if (l == 0 && !h->q1) {
            op.fine = 1;
            op.sigma = A(1);
            op.c = (A)(h->tau * h->D[stage]);
            op.faces = facesA;
        } else {
            op.fine = 0;
            op.sten = lev[l].sten[stage];
            op.sten_sc = lev[l].sten_sc[stage];
        }
        return op;
    }

    template <class S> static Vec<S> shift_vec(Vec<S> v, long long elems, int n0) {
        v.d += elems;
        if (PT<S>::scaled) v.sc += elems / n0;
        return v;
    }

    // Smoother and residual launches specialised by level kind (2D matrix-free, 2D stored; 3D generic).
    // Large batches of the 2D matrix-free level (kappa = 1) take the streaming strip kernel.
    void launch_smooth(int kind, dim3 grid, dim3 block, const LevelOp<SI>& op, const PtMap& pm, int B, const int* act,
                       Vec<SI> x, Vec<SI> b, Vec<SI> out, A om) {
        if constexpr (PT<SI>::scaled) {
            if (vec16_ok(op)) {
                const int gs = vec16_group(op.g.n0);
                if (x.d) launch(k_vec16<SI, 0>, vec16_grid(op, B), kVecThreads, 0, st(), op, gs, B, act, x, b, out, om);
                else launch(k_vec16<SI, 1>, vec16_grid(op, B), kVecThreads, 0, st(), op, gs, B, act, x, b, out, om);
                return;
            }
        }
        if constexpr (!PT<SI>::scaled) {
            if (kind == 4 && grid.y >= 16 && strip_ok(op)) {
                if (x.d) launch(k_strip2d<SI, 0>, strip_grid(op, B), kStripThreads, 0, st(), op, B, act, x, b, out, om);
                else launch(k_strip2d<SI, 1>, strip_grid(op, B), kStripThreads, 0, st(), op, B, act, x, b, out, om);
                return;
            }
            if (kind == 2 && grid.y >= 16 && strip_st_ok(op)) {
                const int rs = strip_st_rows(op, B);
                if (x.d) launch(k_strip2d_st<SI, 0>, strip_st_grid(op, B, rs), kStripThreads, 0, st(), op, B, act, x, b, out, om, rs);
                else launch(k_strip2d_st<SI, 1>, strip_st_grid(op, B, rs), kStripThreads, 0, st(), op, B, act, x, b, out, om, rs);
                return;
            }
        }
        launch_smooth_rows(kind, grid, block, op, pm, B, act, x, b, out, om);
    }
    template <class... Args> void launch_smooth_rows(int kind, dim3 grid, dim3 block, Args... args) {
        if constexpr (!PT<SI>::scaled) {
            // large 2D batches: four rows per thread (grid.y = items)
            constexpr int kRows = 4;
            if ((kind == 4 || kind == 2) && grid.y >= 16) {
                dim3 gr((grid.x + kRows - 1) / kRows, grid.y);
                if (kind == 4) launch(k_smooth_rows<SI, 4, kRows>, gr, block, 0, st(), args...);
                else launch(k_smooth_rows<SI, 2, kRows>, gr, block, 0, st(), args...);
                return;
            }
        }
        if (kind == 4) launch(k_smooth<SI, 4>, grid, block, 0, st(), args...);
        else if (kind == 2) launch(k_smooth<SI, 2>, grid, block, 0, st(), args...);
        else launch(k_smooth<SI, 0>, grid, block, 0, st(), args...);
    }
    void launch_residual(int kind, dim3 grid, dim3 block, const LevelOp<SI>& op, const PtMap& pm, int B,
                         const int* act, Vec<SI> x, Vec<SI> b, Vec<SI> out) {
        if constexpr (PT<SI>::scaled) {
            if (vec16_ok(op) && x.d) {
                launch(k_vec16<SI, 2>, vec16_grid(op, B), kVecThreads, 0, st(), op, vec16_group(op.g.n0), B, act, x,
                       b, out, A(0));
                return;
            }
        }
        if constexpr (!PT<SI>::scaled) {
            if (kind == 4 && grid.y >= 16 && strip_ok(op) && x.d) {
                launch(k_strip2d<SI, 2>, strip_grid(op, B), kStripThreads, 0, st(), op, B, act, x, b, out, A(0));
                return;
            }
            if (kind == 2 && grid.y >= 16 && strip_st_ok(op) && x.d) {
                const int rs = strip_st_rows(op, B);
                launch(k_strip2d_st<SI, 2>, strip_st_grid(op, B, rs), kStripThreads, 0, st(), op, B, act, x, b, out, A(0), rs);
                return;
            }
        }
        launch_residual_rows(kind, grid, block, op, pm, B, act, x, b, out);
    }
    template <class... Args> void launch_residual_rows(int kind, dim3 grid, dim3 block, Args... args) {
        if constexpr (!PT<SI>::scaled) {
            constexpr int kRows = 4;
            if ((kind == 4 || kind == 2) && grid.y >= 16) {
                dim3 gr((grid.x + kRows - 1) / kRows, grid.y);
                if (kind == 4) launch(k_residual_rows<SI, 4, kRows>, gr, block, 0, st(), args...);
                else launch(k_residual_rows<SI, 2, kRows>, gr, block, 0, st(), args...);
                return;
            }
        }
        if (kind == 4) launch(k_residual<SI, 4>, grid, block, 0, st(), args...);
        else if (kind == 2) launch(k_residual<SI, 2>, grid, block, 0, st(), args...);
        else launch(k_residual<SI, 0>, grid, block, 0, st(), args...);
    }

    // x_out = V-cycle(l) applied to (x_in, b); x_in.d == nullptr: zero guess.
    aao_status vcycle(int l, int stage, int B, const int* act, Vec<SI> xin, Vec<SI> b, Vec<SI> xout) {
        const Geo& g = lev[l].g;
        const PtMap pm = ptmap(g.n0);
        const dim3 pbl = pt_grid(pm, g.R, B), pth = pt_block(pm);
        const Tail& T = tails[B > 1 ? 1 : 0];
        if (l == T.lc) {
            bytes_hint((xin.d ? 3.0 : 2.0) * nact * g.nx * sizeof(SI));
            if (g.d == 2)
                launch(k_vcycle_tail_2d<SI>, (unsigned)B, dim3(32, 32), T.smem, st(), T.ctx[stage], B, act, b, xin,
                       xout);
            else
                launch(k_vcycle_tail<SI>, (unsigned)B, tail_threads, T.smem, st(), T.ctx[stage], B, act, b, xin, xout);
            AAO_LAUNCH_CHECK();
            return AAO_OK;
        }
        if (l == L - 1) {
            bytes_hint(2.0 * nact * g.nx * sizeof(SI));
            launch(k_coarse_solve<SI>, pt_grid(pm, g.R, B), pt_block(pm), 0, st(), g, pm, B, act, Dinv[stage], b,
                   xout);
            AAO_LAUNCH_CHECK();
            return AAO_OK;
        }
        LevelOp<SI> op = level_op(l, stage);
        const Geo& gc = lev[l + 1].g;
        const PtMap pmc = ptmap(gc.n0);
        const dim3 cbl = pt_grid(pmc, gc.R, B), cth = pt_block(pmc);
        const A om = (A)h->opt.mg_omega;
        const int nu1 = h->opt.mg_pre, nu2 = h->opt.mg_post;
        // Fused kernels trade recomputation for launches: they pay off where the
        // V-cycle is latency bound (small batches: the Schur sweep), not in the
        // bandwidth- or FP64-bound batched phase.  Only on 2D levels and on the
        // matrix-free fine level (a 27-point stored stencil makes the neighbour
        // recomputation too costly).
        // (a finest level that streams through k_vec16 is not fused: its separate sweeps are cheaper
        // than the fused kernels' recomputation)
        const bool fuse = (long long)B * g.nx <= kFuseMaxPoints && (g.d == 2 || op.fine) && !vec16_ok(op);
        const bool f2 = fuse && nu1 >= 2, fps = fuse && nu2 >= 1;
        const int pre_l = f2 ? nu1 - 1 : nu1;
        const int post_l = fps ? nu2 : nu2 + 1;
        const int nops = pre_l + post_l;
        Vec<SI> cur = xin;
        int opi = 0;
        auto dest = [&](void) -> Vec<SI> {
            ++opi;
            if (opi == nops) return xout;
            return (cur.d == lev[l].T0.d) ? lev[l].T1 : lev[l].T0;
        };
        int q = 0;
        if (f2) {
            Vec<SI> d = dest();
            bytes_hint((cur.d ? 3.0 : 2.0) * nact * g.nx * sizeof(SI));
            launch(k_smooth2<SI>, pbl, pth, 0, st(), op, pm, B, act, cur, b, d, om);
            cur = d;
            q = 2;
        }
        for (; q < nu1; ++q) {
            Vec<SI> d = dest();
            bytes_hint((cur.d ? 3.0 : 2.0) * nact * g.nx * sizeof(SI));
            launch_smooth(level_kind(op.fine, g.d), pbl, pth, op, pm, B, act, cur, b, d, om);
            cur = d;
        }
        // residual and restriction
        if (fuse) {
            bytes_hint(((cur.d ? 2.0 : 1.0) * g.nx + gc.nx) * nact * sizeof(SI));
            launch(k_resid_restrict<SI>, cbl, cth, 0, st(), op, gc, pmc, B, act, cur, b, lev[l + 1].Bb);
        } else if (cur.d == nullptr) {
            bytes_hint(1.0 * nact * (g.nx + gc.nx) * sizeof(SI));
            launch(k_restrict<SI>, cbl, cth, 0, st(), g, gc, pmc, B, act, b, lev[l + 1].Bb);
        } else {
            bytes_hint(3.0 * nact * g.nx * sizeof(SI));
            launch_residual(level_kind(op.fine, g.d), pbl, pth, op, pm, B, act, cur, b, lev[l].Rr);
            bytes_hint(1.0 * nact * (g.nx + gc.nx) * sizeof(SI));
            launch(k_restrict<SI>, cbl, cth, 0, st(), g, gc, pmc, B, act, lev[l].Rr, lev[l + 1].Bb);
        }
        AAO_LAUNCH_CHECK();
        Vec<SI> zero{};
        AAO_TRY(vcycle(l + 1, stage, B, act, zero, lev[l + 1].Bb, lev[l + 1].X));
        q = 0;
        if (fps) {
            Vec<SI> d = dest();
            bytes_hint(1.0 * nact * (gc.nx + (cur.d ? 3.0 : 2.0) * g.nx) * sizeof(SI));
            launch(k_prolong_smooth<SI>, pbl, pth, 0, st(), op, gc, pm, B, act, lev[l + 1].X, cur, b, d, om);
            cur = d;
            q = 1;
        } else {
            Vec<SI> d = dest();
            bytes_hint(1.0 * nact * (gc.nx + (cur.d ? 2.0 : 1.0) * g.nx) * sizeof(SI));
            bool rows_done = false;
            if constexpr (!PT<SI>::scaled) {
                if (g.d == 2 && B >= 16) {
                    launch(k_prolong_add_rows<SI, 4>, dim3((pbl.x + 3) / 4, pbl.y), pth, 0, st(), g, gc, pm, B, act,
                           lev[l + 1].X, cur, d);
                    rows_done = true;
                }
            }
            if (!rows_done) launch(k_prolong_add<SI>, pbl, pth, 0, st(), g, gc, pm, B, act, lev[l + 1].X, cur, d);
            cur = d;
        }
        for (; q < nu2; ++q) {
            Vec<SI> d = dest();
            bytes_hint(3.0 * nact * g.nx * sizeof(SI));
            launch_smooth(level_kind(op.fine, g.d), pbl, pth, op, pm, B, act, cur, b, d, om);
            cur = d;
        }
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    aao_status mg_solve(int stage, int B, const int* act, Vec<SI> b, Vec<SI> out) {
        if (B <= kClMaxBatch && cl_C > 0) {
            // one cluster per item: small batches (single time steps, MGRIT's batched steps)
            const ClPlan& pl = B >= kClBatch8 && clp[1].C > 0 ? clp[1] : clp[0];
            bytes_hint(2.0 * nact * h->g.nx * sizeof(SI));
            launch_cluster(k_cluster_mg<SI>, dim3((unsigned)(pl.C * B)), dim3(kClThreads), pl.smem, st(), pl.C,
                           (const ClCtx<SI>*)(pl.ctx + stage), act, b, out);
            AAO_LAUNCH_CHECK();
            return AAO_OK;
        }
        Vec<SI> zero{};
        for (int cyc = 0; cyc < h->opt.mg_cycles; ++cyc) AAO_TRY(vcycle(0, stage, B, act, cyc == 0 ? zero : out, b, out));
        return AAO_OK;
    }

    // Z = P_int^{-1} V (items of s*nx), forward or backward stage sweep.
    aao_status rana(int B, const int* act, Vec<SP> V, Vec<SI> Z, int transpose) {
        const Geo& g = h->g;
        const int s = h->s;
        const PtMap pm0 = ptmap(g.n0);
        for (int t = 0; t < s; ++t) {
            int i = transpose ? s - 1 - t : t;
            const double* coef = (transpose ? h->d_LDb : h->d_LDf) + i * s;
            Vec<SI> Zi = shift_vec(Z, (long long)i * g.nx, g.n0);
            if constexpr (std::is_same<SP, SI>::value && !PT<SI>::scaled) {
                // the sweep's first stage has no coupling (L is unit lower triangular): its right-hand
                // side is V_i itself, which the shifted solve reads in place (the copy into mgb would
                // store the same values)
                if (t == 0) {
                    AAO_TRY(mg_solve(i, B, act, shift_vec(V, (long long)i * g.nx, g.n0), Zi));
                    continue;
                }
            }
            bytes_hint(1.0 * nact * g.nx * (sizeof(SP) + (transpose ? s - 1 - i : i) * sizeof(SI) + sizeof(SI)));
            launch(k_rana_rhs<SP, SI>, pt_grid(pm0, g.R, B), pt_block(pm0), 0, st(), g, pm0, B, act, V, i, Z, s,
                   coef, (A)h->tau, sopA, mgb);
            AAO_LAUNCH_CHECK();
            AAO_TRY(mg_solve(i, B, act, mgb, Zi));
        }
        return AAO_OK;
    }

    // ------------------------------------------------------- inner GMRES
    // Batched GMRES(kin) on Theta_hat (or Theta_hat^T) for B items of s*nx;
    // rhs item b at src + b*sbs (type SR, unscaled).  On exit Z0/yh/itsh hold the
    // Krylov solution of every item; out (if given) receives sum_k y_k Z_k.
    template <class SR>
    aao_status inner(int B, const SR* src, long long sbs, double* out, long long obs, int transpose) {
        const Geo& g = h->g;
        const int s = h->s;
        const long long item = (long long)s * g.nx;
        const long long rows = (long long)s * g.R;
        const PtMap pm0 = ptmap(g.n0);
        const dim3 nbp = pt_grid(pm0, rows, B), ntp = pt_block(pm0);
        Red red = h->red;
        red.nchunk = h->nchunk_for(B, rows * ((g.n0 + kWarp - 1) / kWarp));
        dim3 rgrid(red.nchunk, B);
        launch(k_norm<SR>, rgrid, kBlock, 0, st(), g.n0, rows, B, nullptr, src, sbs, red, betah, 1);
        launch(k_inner_init, (B + 127) / 128, 128, 0, st(), B, kin, betah, activeh, itsh, gh, nonfin);
        refresh_nact(B);
        launch(k_scale_store<SP, SR>, nbp, ntp, 0, st(), pm0, (int)rows, B, activeh, src, sbs, (const double*)betah, 1LL, V0);
        AAO_LAUNCH_CHECK();
        const long long HS = (long long)(kin + 1) * kin;
        for (int k = 0; k < kin; ++k) {
            Vec<SP> Vk = shift_vec(V0, k * vstride, g.n0);
            Vec<SI> Zk = shift_vec(Z0, k * zstride, g.n0);
            AAO_TRY(rana(B, activeh, Vk, Zk, transpose));
            bytes_hint(1.0 * nact * item * (sizeof(SI) + sizeof(A)));
            launch(k_theta<SI, A>, pt_grid(pm0, g.R, B), pt_block(pm0), 0, st(), g, pm0, B, (const int*)activeh, Zk,
                   wv, item, s, transpose ? h->d_AT : h->d_A,
                                                     (A)h->tau, sopA);
            AAO_LAUNCH_CHECK();
            // modified Gram--Schmidt: h_{0,k} = V_0.w; then w -= h_{i-1,k} V_{i-1}, h_{i,k} = V_i.w
            Vec<SP> none{};
            bytes_hint(1.0 * nact * item * (sizeof(A) + sizeof(SP)));
            launch(k_mgs<SP, A>, rgrid, kBlock, 0, st(), g.n0, rows, B, activeh, wv, item, none, nullptr, V0, HS,
                                                     red, Hh + k);
            for (int i = 1; i <= k + 1; ++i) {
                Vec<SP> Vp = shift_vec(V0, (i - 1) * vstride, g.n0);
                Vec<SP> Vn = i <= k ? shift_vec(V0, i * vstride, g.n0) : none;
                bytes_hint(1.0 * nact * item * (2 * sizeof(A) + (i <= k ? 2 : 1) * sizeof(SP)));
                launch(k_mgs<SP, A>, rgrid, kBlock, 0, st(), g.n0, rows, B, activeh, wv, item, Vp,
                                                         Hh + (i - 1) * kin + k, Vn, HS, red, Hh + i * kin + k);
            }
            launch(k_givens, (B + 127) / 128, 128, 0, st(), B, k, kin, Hh, HS, csh, snh, gh, betah, itol, activeh, itsh,
                                                        nonfin, nullptr);
            AAO_LAUNCH_CHECK();
            refresh_nact(B);
            if (k + 1 < kin) {
                Vec<SP> Vn = shift_vec(V0, (k + 1) * vstride, g.n0);
                launch(k_scale_store<SP, A>, nbp, ntp, 0, st(), pm0, (int)rows, B, (const int*)activeh, (const A*)wv, item,
                                                              Hh + (k + 1) * kin + k, HS, Vn);
                AAO_LAUNCH_CHECK();
            }
        }
        launch(k_hess_solve, (B + 127) / 128, 128, 0, st(), B, kin, Hh, HS, gh, itsh, yh, brk);
        launch(k_count_its, 1, 128, 0, st(), B, itsh, itcount);
        if (out) {
            Vec<SI> Zc = Z0;
            launch(k_combine<SI, double>, nbp, ntp, 0, st(), pm0, (int)rows, B, Zc, zstride, (const double*)yh, kin,
                   (const int*)itsh, out, obs, 0);
        }
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    // ------------------------------------------------------------- P_tilde
    // One step of the Schur substitution (forward: z_{v,n} -> z_{v,n+1};
    // transposed: u_{n+1} -> u_n), with n, z and r read from device memory.
    aao_status schur_step(int transpose) {
        const Geo& g = h->g;
        const int s = h->s;
        const long long item = (long long)s * g.nx;
        const unsigned nbr = blocks_for_rows(g.R);
        if (!transpose) {
            launch(k_schur_rhs<A>, nbr, kBlock, 0, st(), g, s, (const StepPtrs*)stepp, tbuf, sopA);
            AAO_TRY(inner<A>(1, tbuf, item, nullptr, 0, 0));
            launch(k_schur_update<SI, A>, nbr, kBlock, 0, st(), g, s, wsrc ? wsrc : (const A*)wbuf,
                   (const StepPtrs*)stepp, Z0,
                   zstride, (const double*)yh, kin, (const int*)itsh, (const double*)h->d_b, h->tau);
            launch(k_step_add, 1, 1, 0, st(), stepp, 1);
        } else {
            launch(k_schurT_rhs<A>, (unsigned)((item + 255) / 256), 256, 0, st(), g.nx, s, (const StepPtrs*)stepp,
                   (const double*)h->d_b, tbuf);
            AAO_TRY(inner<A>(1, tbuf, item, nullptr, 0, 1));
            Vec<SI> Zc = Z0;
            launch(k_combine<SI, A>, pt_grid(ptmap(g.n0), (long long)s * g.R, 1), pt_block(ptmap(g.n0)), 0, st(), ptmap(g.n0),
                   s * g.R, 1,
                   Zc, zstride, (const double*)yh, kin, (const int*)itsh, qbuf, item, 0);
            launch(k_schurT_update<A>, nbr, kBlock, 0, st(), g, s, (const StepPtrs*)stepp, (const A*)qbuf, h->tau,
                   sopA);
            launch(k_step_add, 1, 1, 0, st(), stepp, -1);
        }
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    // A batched step of the recurrence over B of MGRIT's intervals (items b = 0..B-1 at time
    // indices sp->n +- b mg_m), or with `residual` the C-point residuals into the coarse source.
    aao_status schur_step_b(int transpose, int residual, int B) {
        const Geo& g = h->g;
        const int s = h->s;
        const int stride = mg_m;
        const long long item = (long long)s * g.nx;
        const unsigned nbr = blocks_for_rows(g.R);
        if (!transpose) {
            launch(k_schur_rhs_b<A>, dim3(nbr, (unsigned)B), kBlock, 0, st(), g, s, (const StepPtrs*)stepp, stride, tbuf,
                   sopA);
            AAO_TRY(inner<A>(B, tbuf, item, nullptr, 0, 0));
            launch(k_schur_update_b<SI, A>, dim3(nbr, (unsigned)B), kBlock, 0, st(), g, s, (const A*)wbuf,
                   (const StepPtrs*)stepp, stride, Z0, zstride, (const double*)yh, kin, (const int*)itsh,
                   (const double*)h->d_b, h->tau, residual ? coarse->wbuf : (A*)nullptr);
            launch(k_step_add, 1, 1, 0, st(), stepp, 1);
        } else {
            launch(k_schurT_rhs_b<A>, dim3((unsigned)((item + 255) / 256), (unsigned)B), 256, 0, st(), g.nx, s,
                   (const StepPtrs*)stepp, stride, (const double*)h->d_b, tbuf);
            AAO_TRY(inner<A>(B, tbuf, item, nullptr, 0, 1));
            const PtMap pm = ptmap(g.n0);
            Vec<SI> Zc = Z0;
            launch(k_combine<SI, A>, pt_grid(pm, (long long)s * g.R, B), pt_block(pm), 0, st(), pm, s * g.R, B, Zc,
                   zstride, (const double*)yh, kin, (const int*)itsh, qbuf, item, 0);
            launch(k_schurT_update_b<A>, dim3(nbr, (unsigned)B), kBlock, 0, st(), g, s, (const StepPtrs*)stepp, stride,
                   (const A*)qbuf, h->tau, sopA, residual ? rbufT : (double*)nullptr, B);
            launch(k_step_add, 1, 1, 0, st(), stepp, -1);
        }
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    aao_status step_of_kind(int transpose, int kind) {
        if (kind == 0) return schur_step(transpose);
        return schur_step_b(transpose, kind == 2, kind == 3 ? mg_nc + 1 : mg_nc);
    }

    // Capture one step of a kind into a CUDA graph (on a private stream) the first time
    // it is needed; replays then issue the whole step with one launch.
    aao_status ensure_graph(int transpose, int kind) {
        if (gexec[transpose][kind]) return AAO_OK;
        if (!cap_stream) AAO_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
        cudaStream_t keep = cur_stream;
        cur_stream = cap_stream;
        const long long before = g_thread_launches;
        AAO_CUDA_TRY(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
        aao_status st_ = step_of_kind(transpose, kind);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
        cur_stream = keep;
        // captured launches run only when the graph is replayed: count them there
        g_launches -= g_thread_launches - before;
        g_thread_launches = before;
        if (st_ != AAO_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st_;
        }
        if (e != cudaSuccess) {
            set_error(std::string("graph capture failed: ") + cudaGetErrorString(e));
            return AAO_ERR_CUDA;
        }
        size_t nodes = 0;
        cudaGraphGetNodes(graph, nullptr, &nodes);
        graph_nodes[transpose][kind] = (long long)nodes;
        e = cudaGraphInstantiate(&gexec[transpose][kind], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            gexec[transpose][kind] = nullptr;
            set_error(std::string("graph instantiation failed: ") + cudaGetErrorString(e));
            return AAO_ERR_CUDA;
        }
        return AAO_OK;
    }

    // `count` steps of a kind, each a graph replay (eager launches while a launch profile is open,
    // which needs one event pair per kernel).
    aao_status run_steps(int transpose, int kind, int count) {
        const bool use_graph = !g_prof_on;
        if (use_graph) AAO_TRY(ensure_graph(transpose, kind));
        for (int q = 0; q < count; ++q) {
            if (use_graph) {
                AAO_CUDA_TRY(cudaGraphLaunch(gexec[transpose][kind], st()));
                g_launches += graph_nodes[transpose][kind];
            } else {
                AAO_TRY(step_of_kind(transpose, kind));
            }
        }
        return AAO_OK;
    }

    aao_status schur_sweep(int transpose) { return run_steps(transpose, 0, h->nt); }

    // S_tilde's recurrence z_0 = w_0, z_{n+1} = Phi(z_n) + w_{n+1} by one two-level MGRIT
    // iteration with C-points n = c m (F-relaxation; initial guess z_0 = w_0, zero C-points):
    //   1. interval c relaxes from its C-point to the next one; z_{cm+1} = Phi(0) + w_{cm+1} =
    //      w_{cm+1} for c > 0, and the interval's last step yields the next C-point's residual
    //      r_{c+1} = w_{(c+1)m} + Phi(z_{(c+1)m-1}) - 0 in place of that (zero) C-point;
    //   2. the coarse recurrence e_c = Phi_c(e_{c-1}) + r_c (the substitution step with step m tau),
    //      and the corrected C-point z_{cm} = 0 + e_c;
    //   3. a final F-relaxation of every interval from its corrected C-point.
    // The intervals run on the workers' streams; event c orders interval c's first relaxation before
    // coarse step c+1, and coarse step c before interval c's final relaxation, so the coarse chain
    // overlaps the intervals' work.  Used when the shifted solves run as level kernels (no cluster
    // plan): concurrent single-item steps then fill the GPU.  w is in wbuf; z_0 is set by the caller.
    aao_status mgrit_dataflow_forward(double* z) {
        const long long nx = h->g.nx;
        const int m = mg_m, nc = mg_nc, K = nwork;
        const unsigned nb = (unsigned)((nx + 255) / 256);
        AAO_CUDA_TRY(cudaEventRecord(ev_start, st()));
        for (int w = 0; w < K; ++w) AAO_CUDA_TRY(cudaStreamWaitEvent(wst[w], ev_start, 0));
        for (int c = 0; c < nc; ++c) {
            Precond* W = work[c % K];
            if (c == 0) {
                launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, (const double*)nullptr, 0);
                AAO_TRY(W->run_steps(0, 0, m));
            } else {
                launch(k_convert<A, double>, nb, 256, 0, W->st(), (const A*)(wbuf + (long long)(c * m + 1) * nx),
                       z + (long long)(c * m + 1) * nx, nx);
                launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, (const double*)nullptr, c * m + 1);
                AAO_TRY(W->run_steps(0, 0, m - 1));
            }
            AAO_CUDA_TRY(cudaEventRecord(ev_f1[c], W->st()));
        }
        AAO_CUDA_TRY(cudaMemsetAsync(coarse->wbuf, 0, sizeof(A) * nx, st()));
        AAO_CUDA_TRY(cudaMemsetAsync(ebuf, 0, sizeof(double) * nx, st()));
        launch(k_step_set, 1, 1, 0, st(), coarse->stepp, ebuf, (const double*)nullptr, 0);
        for (int c = 1; c <= nc; ++c) {
            AAO_CUDA_TRY(cudaStreamWaitEvent(st(), ev_f1[c - 1], 0));
            launch(k_convert<double, A>, nb, 256, 0, st(), (const double*)(z + (long long)c * m * nx),
                   coarse->wbuf + (long long)c * nx, nx);
            AAO_TRY(coarse->run_steps(0, 0, 1));
            AAO_CUDA_TRY(cudaMemcpyAsync(z + (long long)c * m * nx, ebuf + (long long)c * nx, sizeof(double) * nx,
                                         cudaMemcpyDeviceToDevice, st()));
            AAO_CUDA_TRY(cudaEventRecord(ev_c[c], st()));
        }
        for (int c = 0; c < nc; ++c) {
            Precond* W = work[c % K];
            if (c > 0) AAO_CUDA_TRY(cudaStreamWaitEvent(W->st(), ev_c[c], 0));
            launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, (const double*)nullptr, c * m);
            AAO_TRY(W->run_steps(0, 0, m - 1));
        }
        if (mg_r > 0) {           // the shorter final interval, from the last C-point
            Precond* W = work[nc % K];
            AAO_CUDA_TRY(cudaStreamWaitEvent(W->st(), ev_c[nc], 0));
            launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, (const double*)nullptr, nc * m);
            AAO_TRY(W->run_steps(0, 0, mg_r));
        }
        for (int w = 0; w < K; ++w) {
            AAO_CUDA_TRY(cudaEventRecord(ev_join[w], wst[w]));
            AAO_CUDA_TRY(cudaStreamWaitEvent(st(), ev_join[w], 0));
        }
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    // The same for S_tilde^T's backward recurrence u_nt = r_{v,nt}, u_n = Phi^T(u_{n+1}) + r_{v,n},
    // run forward in reversed time (C-points n = nt - c m).  u_nt is set by the caller.
    aao_status mgrit_dataflow_transpose(double* z, const double* r) {
        const long long nx = h->g.nx;
        const int m = mg_m, nc = mg_nc, K = nwork, nt = h->nt;
        AAO_CUDA_TRY(cudaEventRecord(ev_start, st()));
        for (int w = 0; w < K; ++w) AAO_CUDA_TRY(cudaStreamWaitEvent(wst[w], ev_start, 0));
        for (int c = 0; c < nc; ++c) {
            Precond* W = work[c % K];
            if (c == 0) {
                launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, r, nt - 1);
                AAO_TRY(W->run_steps(1, 0, m));
            } else {
                const long long n1 = nt - c * m - 1;
                AAO_CUDA_TRY(cudaMemcpyAsync(z + n1 * nx, r + n1 * nx, sizeof(double) * nx, cudaMemcpyDeviceToDevice,
                                             W->st()));
                launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, r, (int)n1 - 1);
                AAO_TRY(W->run_steps(1, 0, m - 1));
            }
            AAO_CUDA_TRY(cudaEventRecord(ev_f1[c], W->st()));
        }
        AAO_CUDA_TRY(cudaMemsetAsync(rbufT + (long long)nc * nx, 0, sizeof(double) * nx, st()));
        AAO_CUDA_TRY(cudaMemsetAsync(ebuf + (long long)nc * nx, 0, sizeof(double) * nx, st()));
        launch(k_step_set, 1, 1, 0, st(), coarse->stepp, ebuf, (const double*)rbufT, nc - 1);
        for (int c = 1; c <= nc; ++c) {
            AAO_CUDA_TRY(cudaStreamWaitEvent(st(), ev_f1[c - 1], 0));
            const long long zc = (long long)(nt - c * m) * nx, ec = (long long)(nc - c) * nx;
            AAO_CUDA_TRY(cudaMemcpyAsync(rbufT + ec, z + zc, sizeof(double) * nx, cudaMemcpyDeviceToDevice, st()));
            AAO_TRY(coarse->run_steps(1, 0, 1));
            AAO_CUDA_TRY(cudaMemcpyAsync(z + zc, ebuf + ec, sizeof(double) * nx, cudaMemcpyDeviceToDevice, st()));
            AAO_CUDA_TRY(cudaEventRecord(ev_c[c], st()));
        }
        for (int c = 0; c < nc; ++c) {
            Precond* W = work[c % K];
            if (c > 0) AAO_CUDA_TRY(cudaStreamWaitEvent(W->st(), ev_c[c], 0));
            launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, r, nt - c * m - 1);
            AAO_TRY(W->run_steps(1, 0, m - 1));
        }
        if (mg_r > 0) {           // the shorter final interval (the first steps in time)
            Precond* W = work[nc % K];
            AAO_CUDA_TRY(cudaStreamWaitEvent(W->st(), ev_c[nc], 0));
            launch(k_step_set, 1, 1, 0, W->st(), W->stepp, z, r, nt - nc * m - 1);
            AAO_TRY(W->run_steps(1, 0, mg_r));
        }
        for (int w = 0; w < K; ++w) {
            AAO_CUDA_TRY(cudaEventRecord(ev_join[w], wst[w]));
            AAO_CUDA_TRY(cudaStreamWaitEvent(st(), ev_join[w], 0));
        }
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    // Lock-step schedule of the same MGRIT iteration (used when a shifted solve runs on one
    // thread-block cluster: one launch then holds every interval's clusters): F-relaxation as
    // batched steps over the mg_nc intervals from z_0 = w_0 and zero C-points, the C-point
    // residuals, the coarse error recurrence e_c = Phi_c(e_{c-1}) + r_c by substitution with step
    // m tau, the C-point correction z_{cm} += e_c and a final F-relaxation (which also relaxes the
    // shorter last interval when m does not divide nt).  w is in wbuf; z_0 is set by the caller.
    aao_status mgrit_batched_forward(double* z) {
        const long long nx = h->g.nx;
        const int m = mg_m, nc = mg_nc;
        const unsigned nb = (unsigned)(((long long)nc * nx + 255) / 256);
        launch(k_mgrit_cpoints, nb, 256, 0, st(), z, (const double*)nullptr, nx, nc, m, 0, 1, 0, 1);
        launch(k_step_set, 1, 1, 0, st(), stepp, z, (const double*)nullptr, 0);
        AAO_LAUNCH_CHECK();
        AAO_TRY(run_steps(0, 1, m - 1));
        launch(k_step_set, 1, 1, 0, st(), stepp, z, (const double*)nullptr, m - 1);
        AAO_TRY(run_steps(0, 2, 1));
        AAO_CUDA_TRY(cudaMemsetAsync(coarse->wbuf, 0, sizeof(A) * nx, st()));
        AAO_CUDA_TRY(cudaMemsetAsync(ebuf, 0, sizeof(double) * nx, st()));
        launch(k_step_set, 1, 1, 0, st(), coarse->stepp, ebuf, (const double*)nullptr, 0);
        AAO_LAUNCH_CHECK();
        AAO_TRY(coarse->run_steps(0, 0, nc));
        launch(k_mgrit_cpoints, nb, 256, 0, st(), z, (const double*)ebuf, nx, nc, m, 0, 1, 0, 1);
        launch(k_step_set, 1, 1, 0, st(), stepp, z, (const double*)nullptr, 0);
        AAO_LAUNCH_CHECK();
        // the final F-relaxation; its first mg_r steps also relax the shorter final interval from
        // the last C-point
        if (mg_r > 0) AAO_TRY(run_steps(0, 3, mg_r));
        return run_steps(0, 1, m - 1 - mg_r);
    }

    // The same for S_tilde^T's backward recurrence u_nt = r_{v,nt}, u_n = Phi^T(u_{n+1}) + r_{v,n},
    // run forward in reversed time (C-points n = nt - c m).  u_nt is set by the caller.
    aao_status mgrit_batched_transpose(double* z, const double* r) {
        const long long nx = h->g.nx;
        const int m = mg_m, nc = mg_nc, nt = h->nt;
        const unsigned nb = (unsigned)(((long long)nc * nx + 255) / 256);
        launch(k_mgrit_cpoints, nb, 256, 0, st(), z, (const double*)nullptr, nx, nc, m, nt, -1, 0, 1);
        launch(k_step_set, 1, 1, 0, st(), stepp, z, r, nt - 1);
        AAO_LAUNCH_CHECK();
        AAO_TRY(run_steps(1, 1, m - 1));
        launch(k_step_set, 1, 1, 0, st(), stepp, z, r, nt - m);
        AAO_TRY(run_steps(1, 2, 1));
        AAO_CUDA_TRY(cudaMemsetAsync(rbufT + (long long)nc * nx, 0, sizeof(double) * nx, st()));
        AAO_CUDA_TRY(cudaMemsetAsync(ebuf + (long long)nc * nx, 0, sizeof(double) * nx, st()));
        launch(k_step_set, 1, 1, 0, st(), coarse->stepp, ebuf, (const double*)rbufT, nc - 1);
        AAO_LAUNCH_CHECK();
        AAO_TRY(coarse->run_steps(1, 0, nc));
        launch(k_mgrit_cpoints, nb, 256, 0, st(), z, (const double*)ebuf, nx, nc, m, nt, -1, nc, -1);
        launch(k_step_set, 1, 1, 0, st(), stepp, z, r, nt - 1);
        AAO_LAUNCH_CHECK();
        if (mg_r > 0) AAO_TRY(run_steps(1, 3, mg_r));
        return run_steps(1, 1, m - 1 - mg_r);
    }

    aao_status mgrit_forward(double* z) { return nwork ? mgrit_dataflow_forward(z) : mgrit_batched_forward(z); }
    aao_status mgrit_transpose(double* z, const double* r) {
        return nwork ? mgrit_dataflow_transpose(z, r) : mgrit_batched_transpose(z, r);
    }

    aao_status apply(const double* r, double* z, int transpose) override {
        const Geo& g = h->g;
        const int s = h->s, nt = h->nt;
        const long long nx = g.nx, nv = h->nv, item = (long long)s * nx;
        cudaEventRecord(e0, st());
        if (!transpose) {
            {
                NvtxRange range_("aao.precond.theta_phase");
                AAO_TRY(inner<double>(nt, r + nv, item, z + nv, item, 0));
            }
            cudaEventRecord(e1, st());
            long long tot = (nt + 1) * nx;
            if (h->q1) {
                // g = r_v - Psi_1 z_V with M, then w = M^{-1} g, z_{v,0} = w_0
                const PtMap pm = ptmap(g.n0);
                launch(k_schur_g_q1<A>, pt_grid(pm, g.R, nt + 1), pt_block(pm), 0, st(), g, pm, nt,
                       s, r, (const double*)(z + nv), (const double*)h->d_b, h->tau, sopA.q, wbuf);
                AAO_TRY(mass_inverse(wbuf, nt + 1));
                launch(k_convert<A, double>, (unsigned)((nx + 255) / 256), 256, 0, st(), (const A*)wbuf, z, nx);
            } else {
                launch(k_schur_g<A>, (unsigned)((tot + 255) / 256), 256, 0, st(), nx, nt, s, r,
                       (const double*)(z + nv), (const double*)h->d_b, h->tau, wbuf, z);
            }
            launch(k_step_set, 1, 1, 0, st(), stepp, z, r, 0);
            AAO_LAUNCH_CHECK();
            {
                NvtxRange range_("aao.precond.schur_sweep");
                AAO_TRY(mg_m > 0 ? mgrit_forward(z) : schur_sweep(0));
            }
            cudaEventRecord(e2, st());
        } else {
            // S_tilde^T: backward substitution, u stored in z's v-part (M = I: z_v = u)
            AAO_CUDA_TRY(cudaMemcpyAsync(z + nt * nx, r + nt * nx, sizeof(double) * nx, cudaMemcpyDeviceToDevice,
                                         st()));
            launch(k_step_set, 1, 1, 0, st(), stepp, z, r, nt - 1);
            AAO_LAUNCH_CHECK();
            {
                NvtxRange range_("aao.precond.schur_sweep_transposed");
                AAO_TRY(mg_m > 0 ? mgrit_transpose(z, r) : schur_sweep(1));
            }
            cudaEventRecord(e1, st());
            long long tot = (long long)nt * item;
            if (h->q1) {
                // z_v = M^{-1} u (Chebyshev in the recurrence precision), then the stage rhs with M
                const long long nvx = (long long)(nt + 1) * nx;
                launch(k_convert<double, A>, (unsigned)((nvx + 255) / 256), 256, 0, st(), (const double*)z, wbuf, nvx);
                AAO_TRY(mass_inverse(wbuf, nt + 1));
                launch(k_convert<A, double>, (unsigned)((nvx + 255) / 256), 256, 0, st(), (const A*)wbuf, z, nvx);
                const PtMap pm = ptmap(g.n0);
                launch(k_schurT_vrhs_q1<A>, pt_grid(pm, g.R, nt), pt_block(pm), 0, st(), g, pm, nt, s,
                       r + nv, (const double*)z, (const double*)h->d_b, h->tau, sopA.q, tV);
            } else {
                launch(k_schurT_vrhs<A>, (unsigned)((tot + 255) / 256), 256, 0, st(), nx, nt, s, r + nv,
                       (const double*)z, (const double*)h->d_b, h->tau, tV);
            }
            AAO_LAUNCH_CHECK();
            {
                NvtxRange range_("aao.precond.theta_phase_transposed");
                AAO_TRY(inner<A>(nt, tV, item, z + nv, item, 1));
            }
            cudaEventRecord(e2, st());
        }
        return AAO_OK;
    }

    void accumulate_times() override {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, e0, e1) == cudaSuccess && cudaEventElapsedTime(&b, e1, e2) == cudaSuccess) {
            t_theta_ms += a;
            t_schur_ms += b;
        }
        cudaGetLastError();
    }

    // ------------------------------------------------- component entry points
    aao_status shifted_solve(int stage, const double* b, double* x) override {
        const Geo& g = h->g;
        nact = 1;
        launch(k_scale_store<SI, double>, pt_grid(ptmap(g.n0), g.R, 1), pt_block(ptmap(g.n0)), 0, st(), ptmap(g.n0), g.R, 1,
               (const int*)nullptr, b, g.nx,
                                                                             nullptr, 0, mgb);
        AAO_LAUNCH_CHECK();
        Vec<SI> out = Z0;   // item 0, stage 0 of the first Z basis
        AAO_TRY(mg_solve(stage, 1, nullptr, mgb, out));
        launch(k_load<SI, double>, pt_grid(ptmap(g.n0), g.R, 1), pt_block(ptmap(g.n0)), 0, st(), ptmap(g.n0), g.R, 1, out, x,
               g.nx);
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    aao_status pint_apply(const double* r, double* y, int transpose) override {
        const Geo& g = h->g;
        nact = 1;
        const long long rows = (long long)h->s * g.R;
        launch(k_scale_store<SP, double>, pt_grid(ptmap(g.n0), rows, 1), pt_block(ptmap(g.n0)), 0, st(), ptmap(g.n0),
               (int)rows, 1, (const int*)nullptr, r,
                                                                              (long long)h->s * g.nx, nullptr, 0, V0);
        AAO_LAUNCH_CHECK();
        AAO_TRY(rana(1, nullptr, V0, Z0, transpose));
        launch(k_load<SI, double>, pt_grid(ptmap(g.n0), rows, 1), pt_block(ptmap(g.n0)), 0, st(), ptmap(g.n0), (int)rows, 1,
               Z0, y, (long long)h->s * g.nx);
        AAO_LAUNCH_CHECK();
        return AAO_OK;
    }

    aao_status inner_solve(int nblocks, const double* r, double* z, int* its_host) override {
        if (nblocks < 1 || nblocks > Bmax) {
            set_error("inner_solve: nblocks must be in 1..nt");
            return AAO_ERR_ARG;
        }
        const long long item = (long long)h->s * h->g.nx;
        AAO_TRY(inner<double>(nblocks, r, item, z, item, 0));
        if (its_host) {
            AAO_CUDA_TRY(cudaMemcpyAsync(its_host, itsh, sizeof(int) * nblocks, cudaMemcpyDeviceToHost, st()));
            AAO_CUDA_TRY(cudaStreamSynchronize(st()));
        }
        return AAO_OK;
    }

    long long inner_its() override {
        long long v = 0;
        cudaMemcpyAsync(&v, itcount, sizeof(long long), cudaMemcpyDeviceToHost, st());
        cudaStreamSynchronize(st());
        for (int w = 0; w < nwork; ++w) v += work[w]->inner_its();
        return v + (coarse ? coarse->inner_its() : 0);
    }
    void reset_inner_its() override {
        cudaMemsetAsync(itcount, 0, sizeof(long long), st());
        if (coarse) coarse->reset_inner_its();
        for (int w = 0; w < nwork; ++w) work[w]->reset_inner_its();
    }

    int nonfinite_flag() override {
        int v[2] = {0, 0};
        cudaMemcpyAsync(v, nonfin, 2 * sizeof(int), cudaMemcpyDeviceToHost, st());
        cudaStreamSynchronize(st());
        int wf = 0;
        for (int w = 0; w < nwork; ++w) wf |= work[w]->nonfinite_flag();
        return v[0] | v[1] | wf | (coarse ? coarse->nonfinite_flag() : 0);
    }
};

}  // namespace aao
