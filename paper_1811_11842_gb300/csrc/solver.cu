// Krylov drivers: preconditioned CG in the W inner product (the velocity
// predictor and the singular pressure system are W-symmetric), GMRES(m)
// with right preconditioning for the non-symmetric phase-field system (the
// paper's KSP choice, §4.1 Listing 4) and FP64 iterative refinement around
// FP32 inner solves.  Convergence: ||b - A x||_W <= rtol ||b||_W; GMRES
// confirms it on the true residual at each restart.  Written once for the
// host-loop and the graph-capture modes (see solver.h).
#include <cmath>

#include "solver.h"

namespace cahn {

thread_local int64_t* g_frame = nullptr;
void set_launch_frame(int64_t* frame) { g_frame = frame; }

int GraphCount::add_loop() {
    // The table is reserved once and never reallocated: g_frame points into
    // it while nested loops are being added.
    if (body.capacity() < (size_t)capacity) body.reserve(capacity);
    if ((int)body.size() >= capacity) throw ArgError("too many loops in one captured graph");
    body.push_back(0);
    return (int)body.size() - 1;
}

template <typename T>
static T* dalloc(std::vector<void*>& list, size_t count) {
    void* p = nullptr;
    CAHN_CUDA_TRY(cudaMalloc(&p, count * sizeof(T)));
    list.push_back(p);
    return static_cast<T*>(p);
}

template <typename T>
void KrylovWs<T>::alloc(const Grid& grid, int restart, bool gmres, RedWs red, bool flexible) {
    g = grid;
    n = grid.n();
    m = restart;
    r = dalloc<T>(allocs, n);
    z = dalloc<T>(allocs, n);
    p = dalloc<T>(allocs, n);
    q = dalloc<T>(allocs, n);
    CAHN_CUDA_TRY(cudaMemset(p, 0, n * sizeof(T)));
    // GMRES and BiCGStab work vector; the CG's s = A p (Chronopoulos-Gear)
    w = dalloc<T>(allocs, n);
    if (gmres) {
        u = dalloc<T>(allocs, n);
        vk = dalloc<T>(allocs, n);
        V = dalloc<T>(allocs, n * (size_t)(m + 1));
        if (flexible) Z = dalloc<T>(allocs, n * (size_t)(m + 1));
        gm.ldh = m + 1;
        gm.H = dalloc<double>(allocs, (size_t)(m + 1) * m);
        gm.cs = dalloc<double>(allocs, m + 1);
        gm.sn = dalloc<double>(allocs, m + 1);
        gm.g = dalloc<double>(allocs, m + 2);
        gm.y = dalloc<double>(allocs, m + 1);
    }
    sd.scal = dalloc<double>(allocs, S_COUNT);
    sd.ctl = dalloc<Ctl>(allocs, 1);
    CAHN_CUDA_TRY(cudaMemset(sd.scal, 0, S_COUNT * sizeof(double)));
    CAHN_CUDA_TRY(cudaMemset(sd.ctl, 0, sizeof(Ctl)));
    sd.red = red;
    CAHN_CUDA_TRY(cudaMallocHost(&h_ctl, sizeof(Ctl)));
    CAHN_CUDA_TRY(cudaMallocHost(&h_scal, S_COUNT * sizeof(double)));
}

template <typename T>
void KrylovWs<T>::release() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_scal) cudaFreeHost(h_scal);
    h_ctl = nullptr;
    h_scal = nullptr;
}

template <typename T>
void KrylovWs<T>::read_back(cudaStream_t s) {
    CAHN_CUDA_TRY(cudaMemcpyAsync(h_ctl, sd.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(h_scal, sd.scal, S_COUNT * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
    CAHN_CUDA_TRY(cudaStreamSynchronize(s));
}

void loop_while(Driver& d, const int* stop, const std::function<void(Driver&)>& body,
                int predict, int cap, const std::function<bool()>& poll) {
    if (!d.graph) {
        int launched = 0;
        int chunk = predict > 0 ? predict : 1;
        for (;;) {
            for (int c = 0; c < chunk; ++c) body(d);
            launched += chunk;
            if (poll() || launched >= cap) break;
            chunk = launched / 4 > 1 ? launched / 4 : 1;
        }
        return;
    }
    if (!d.pool || d.depth + 1 >= (int)d.pool->size()) throw ArgError("loops nested too deep");
    cudaStreamCaptureStatus cst;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    CAHN_CUDA_TRY(cudaStreamGetCaptureInfo(d.s, &cst, nullptr, &g, &deps, &edges, &ndeps));
    cudaGraphConditionalHandle h;
    CAHN_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    launch_set_cond(h, stop, nullptr, d.s);   // enter only if not finished yet
    CAHN_CUDA_TRY(cudaStreamGetCaptureInfo(d.s, &cst, nullptr, &g, &deps, &edges, &ndeps));
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    CAHN_CUDA_TRY(cudaGraphAddNode(&node, g, deps, edges, ndeps, &prm));
    cudaGraph_t bodyg = prm.conditional.phGraph_out[0];
    Driver in = d;
    in.depth = d.depth + 1;
    in.s = (*d.pool)[in.depth];
    const int idx = d.gc->add_loop();
    int64_t* saved = g_frame;
    g_frame = &d.gc->body[idx];
    CAHN_CUDA_TRY(cudaStreamBeginCaptureToGraph(in.s, bodyg, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeRelaxed));
    try {
        body(in);
        launch_set_cond(h, stop, d.gc->d_counters + idx, in.s);
    } catch (...) {
        // end this body's capture (the graph belongs to the conditional
        // node) so the stream is usable again, then let the caller unwind
        g_frame = saved;
        cudaGraph_t unused = nullptr;
        cudaStreamEndCapture(in.s, &unused);
        cudaGetLastError();
        throw;
    }
    CAHN_CUDA_TRY(cudaStreamEndCapture(in.s, &bodyg));
    g_frame = saved;
    CAHN_CUDA_TRY(cudaStreamUpdateCaptureDependencies(d.s, &node, nullptr, 1,
                                                      cudaStreamSetCaptureDependencies));
}

template <typename T>
static void precondition(size_t n, const T* dinv, const PrecFn<T>* prec, const T* in, T* out,
                         const int* gate, cudaStream_t s) {
    if (dinv)
        launch_scale_by<T>(n, dinv, in, out, gate, s);
    else
        (*prec)(in, out, gate, s);
}

template <typename T>
SolveResult cg_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                     const PrecFn<T>* prec, double rtol, int maxit, bool project,
                     double inv_sumw, int& predict, Driver& d, const int* skip,
                     bool zero_guess) {
    const Grid& g = op.g;
    const size_t n = g.n();
    const cudaStream_t s = d.s;
    const int* done = &W.sd.ctl->done;
    const SolveDev sd = W.sd;
    launch_ctl_init(sd.ctl, maxit, s, skip);
    if (zero_guess)
        launch_start_zero<T>(g, b, x, W.r, sd, rtol, done, s);
    else
        launch_op<T>(op, EPI_RESID, x, b, W.r, sd, done, rtol, s);
    // Singular system: keep the residual W-orthogonal to the constants.  The
    // rounding of every update leaves a null-space component in r that no
    // iteration can remove; in FP32 it grows to ~eps32 cond(A) and stalls
    // the solve, so it is deflated after every update.
    auto deflate = [&](cudaStream_t st) {
        if (!project) return;
        launch_wdot<T>(g, W.r, (const T*)nullptr, sd, S_TMP3, inv_sumw, done, st);
        launch_sub_scalar<T>(W.r, n, sd.scal + S_TMP3, done, st);
    };
    deflate(s);
    if (W.w) {
        // Chronopoulos-Gear CG (the same iterates in exact arithmetic): one
        // operator apply with both inner products <r,z> and <z,Az> fused in
        // its epilogue, then one update of p, s = A p, x and r with the norm
        // and the stopping test -- two launches per iteration besides the
        // preconditioner, where the textbook form takes four
        loop_while(
            d, done,
            [&](Driver& di) {
                const cudaStream_t st = di.s;
                if (dinv)
                    launch_scale_by<T>(n, dinv, W.r, W.z, done, st);
                else
                    (*prec)(W.r, W.z, done, st);
                launch_op<T>(op, EPI_CGCG, W.z, W.r, W.q, sd, done, rtol, st);
                launch_cgcg_update<T>(g, x, W.r, W.p, W.w, W.z, W.q, sd, done, st);
                deflate(st);
            },
            predict, maxit + 2,
            [&]() {
                W.read_back(s);
                return W.h_ctl->done != 0;
            });
    } else {
        if (dinv) {
            launch_cg_rz<T>(g, W.r, dinv, W.z, sd, 1, done, s);
        } else {
            (*prec)(W.r, W.z, done, s);
            launch_cg_rz<T>(g, W.r, nullptr, W.z, sd, 1, done, s);
        }
        launch_copy<T>(W.z, W.p, n, s, done);
        loop_while(
            d, done,
            [&](Driver& di) {
                const cudaStream_t st = di.s;
                launch_op<T>(op, EPI_DOTXY, W.p, nullptr, W.q, sd, done, rtol, st);
                launch_cg_update<T>(g, x, W.r, W.p, W.q, sd, done, st);
                deflate(st);
                if (dinv) {
                    launch_cg_rz<T>(g, W.r, dinv, W.z, sd, 0, done, st);
                } else {
                    (*prec)(W.r, W.z, done, st);
                    launch_cg_rz<T>(g, W.r, nullptr, W.z, sd, 0, done, st);
                }
                launch_cg_p<T>(n, W.z, W.p, sd, done, st);
            },
            predict, maxit + 2,
            [&]() {
                W.read_back(s);
                return W.h_ctl->done != 0;
            });
    }
    if (project) {
        launch_wdot<T>(g, x, (const T*)nullptr, sd, S_TMP3, inv_sumw, nullptr, s);
        launch_sub_scalar<T>(x, n, sd.scal + S_TMP3, nullptr, s);
    }
    launch_zero_if_b0<T>(n, x, sd.scal, s);
    SolveResult res;
    if (!d.graph) {
        W.read_back(s);
        res.it = W.h_ctl->it;
        res.status = W.h_ctl->status;
        res.rel_res = W.h_scal[S_BN] > 0 ? W.h_scal[S_RES0] / W.h_scal[S_BN] : 0.0;
        predict = res.it > 0 ? res.it : 1;
    }
    return res;
}

// Right-preconditioned BiCGStab (the alternative Krylov method for the
// non-symmetric phase-field system): two preconditioner applications and
// two operator applies per iteration, scalars on the device, stopping on
// the updated residual ||r||_W <= rtol ||b||_W.  Vectors from the GMRES
// workspace: rhat = vk, v = q, phat = z, s = w, shat = u, t = V_0.
template <typename T>
SolveResult bicgstab_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                           const PrecFn<T>* prec, double rtol, int maxit, int& predict,
                           Driver& d, const int* skip, bool zero_guess) {
    const Grid& g = op.g;
    const size_t n = g.n();
    const cudaStream_t s = d.s;
    const SolveDev sd = W.sd;
    const int* done = &sd.ctl->done;
    T *rhat = W.vk, *v = W.q, *phat = W.z, *sv = W.w, *shat = W.u, *t = W.V;
    launch_ctl_init(sd.ctl, maxit, s, skip);
    if (zero_guess)
        launch_start_zero<T>(g, b, x, W.r, sd, rtol, done, s);
    else
        launch_op<T>(op, EPI_RESID, x, b, W.r, sd, done, rtol, s);
    launch_bicg_init<T>(n, W.r, rhat, W.p, v, sd.scal, done, s);
    loop_while(
        d, done,
        [&](Driver& di) {
            const cudaStream_t st = di.s;
            launch_bicg_rho<T>(g, rhat, W.r, sd, done, st);
            launch_bicg_p<T>(n, W.r, W.p, v, sd.scal, done, st);
            precondition(n, dinv, prec, W.p, phat, done, st);
            launch_op<T>(op, EPI_APPLY, phat, nullptr, v, sd, done, rtol, st);
            launch_bicg_alpha<T>(g, rhat, v, sd, done, st);
            launch_bicg_s<T>(n, W.r, v, sv, sd.scal, done, st);
            precondition(n, dinv, prec, sv, shat, done, st);
            launch_op<T>(op, EPI_APPLY, shat, nullptr, t, sd, done, rtol, st);
            launch_bicg_omega<T>(g, t, sv, sd, done, st);
            launch_bicg_x<T>(g, x, W.r, phat, shat, sv, t, sd, done, st);
        },
        predict, maxit + 2,
        [&]() {
            W.read_back(s);
            return W.h_ctl->done != 0;
        });
    launch_zero_if_b0<T>(n, x, sd.scal, s);
    SolveResult res;
    if (!d.graph) {
        W.read_back(s);
        res.it = W.h_ctl->it;
        res.status = W.h_ctl->status;
        res.rel_res = W.h_scal[S_BN] > 0 ? W.h_scal[S_RES0] / W.h_scal[S_BN] : 0.0;
        predict = res.it > 0 ? res.it : 1;
    }
    return res;
}

template <typename T>
SolveResult gmres_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                        const PrecFn<T>* prec, double rtol, int maxit, int& predict,
                        Driver& d, const int* skip, bool zero_guess) {
    const Grid& g = op.g;
    const size_t n = g.n();
    const cudaStream_t s = d.s;
    const SolveDev sd = W.sd;
    Ctl* c = sd.ctl;
    const int* done = &c->done;
    const int* cyc = &c->cycle_end;
    const int* idle = &c->idle;
    const int m = W.m;
    // flexible GMRES when the workspace keeps the preconditioned basis
    const bool flexible = !dinv && W.Z != nullptr;
    launch_ctl_init(c, maxit, s, skip);
    // the true residual before the first cycle, then after each cycle
    if (zero_guess)
        launch_start_zero<T>(g, b, x, W.r, sd, rtol, done, s);
    else
        launch_op<T>(op, EPI_RESID, x, b, W.r, sd, done, rtol, s);
    int first_chunk = predict < m ? predict : m;
    loop_while(
        d, done,
        [&](Driver& d1) {
            const cudaStream_t s1 = d1.s;
            launch_gm_start<T>(g, W.r, W.V, W.vk, sd, W.gm, s1);
            loop_while(
                d1, cyc,
                [&](Driver& d2) {
                    const cudaStream_t s2 = d2.s;
                    precondition<T>(n, dinv, prec, W.vk, W.z, cyc, s2);
                    launch_op<T>(op, EPI_APPLY, W.z, nullptr, W.w, sd, cyc, rtol, s2);
                    launch_gm_arnoldi<T>(g, W.w, W.V, n, W.vk, sd, W.gm, m, s2,
                                         flexible ? W.z : nullptr, flexible ? W.Z : nullptr);
                },
                first_chunk, m,
                [&]() {
                    W.read_back(s);
                    return W.h_ctl->cycle_end != 0;
                });
            first_chunk = m;
            if (dinv) {
                launch_gm_update<T>(g, W.V, n, x, dinv, sd, W.gm, s1);
            } else if (flexible) {
                // x += Z y: no preconditioner application at the cycle's end
                launch_gm_update<T>(g, W.Z, n, x, nullptr, sd, W.gm, s1, 1);
            } else {
                launch_gm_update<T>(g, W.V, n, W.u, nullptr, sd, W.gm, s1);
                (*prec)(W.u, W.z, idle, s1);
                launch_add<T>(n, x, W.z, nullptr, idle, s1);
            }
            launch_gm_finish(c, s1);
            launch_op<T>(op, EPI_RESID, x, b, W.r, sd, done, rtol, s1);
        },
        1, maxit + 2,
        [&]() {
            W.read_back(s);
            return W.h_ctl->done != 0;
        });
    launch_zero_if_b0<T>(n, x, sd.scal, s);
    SolveResult res;
    if (!d.graph) {
        W.read_back(s);
        res.it = W.h_ctl->it;
        res.status = W.h_ctl->status;
        res.rel_res = W.h_scal[S_BN] > 0 ? W.h_scal[S_RES0] / W.h_scal[S_BN] : 0.0;
        predict = res.it > 0 ? res.it : 1;
    }
    return res;
}

IrResult ir_solve(KrylovWs<double>& W, const Op& op64, double* x, const double* b, float* r32,
                  float* d32, const InnerSolve& inner, double rtol, int max_outer, bool project,
                  double inv_sumw, double anorm, Driver& d) {
    const Grid& g = op64.g;
    const size_t n = g.n();
    const cudaStream_t s = d.s;
    SolveDev sd = W.sd;
    sd.anorm = anorm;   // the residual launch's last block makes the sweep test
    const int* done = &sd.ctl->done;
    IrResult out;
    launch_ctl_init(sd.ctl, max_outer, s, nullptr);
    loop_while(
        d, done,
        [&](Driver& d1) {
            const cudaStream_t s1 = d1.s;
            // r = b - A x with ||b||, ||r|| and ||x|| (the rounding floor) in one
            // pass, the sweep's stopping test in its last block
            launch_op<double>(op64, EPI_RESIDX, x, b, W.r, sd, done, rtol, s1);
            launch_ir_down(n, W.r, r32, sd.scal, done, s1);
            SolveResult ri = inner(r32, d32, d1, done);   // from d32 = 0 (zero-guess start)
            out.inner_it += ri.it;
            launch_ir_up(n, x, d32, sd.scal, done, s1);
        },
        1, max_outer + 2,
        [&]() {
            W.read_back(s);
            return W.h_ctl->done != 0;
        });
    if (project) {
        launch_wdot<double>(g, x, (const double*)nullptr, sd, S_TMP3, inv_sumw, nullptr, s);
        launch_sub_scalar<double>(x, n, sd.scal + S_TMP3, nullptr, s);
    }
    launch_zero_if_b0<double>(n, x, sd.scal, s);
    if (!d.graph) {
        W.read_back(s);
        out.outer.it = W.h_ctl->it;
        out.outer.status = W.h_ctl->status;
        out.outer.rel_res = W.h_scal[S_BN] > 0 ? W.h_scal[S_RES0] / W.h_scal[S_BN] : 0.0;
    }
    return out;
}

template struct KrylovWs<double>;
template struct KrylovWs<float>;
template SolveResult cg_solve<double>(KrylovWs<double>&, const Op&, double*, const double*,
                                      const double*, const PrecFn<double>*, double, int, bool,
                                      double, int&, Driver&, const int*, bool);
template SolveResult cg_solve<float>(KrylovWs<float>&, const Op&, float*, const float*,
                                     const float*, const PrecFn<float>*, double, int, bool,
                                     double, int&, Driver&, const int*, bool);
template SolveResult gmres_solve<double>(KrylovWs<double>&, const Op&, double*, const double*,
                                         const double*, const PrecFn<double>*, double, int, int&,
                                         Driver&, const int*, bool);
template SolveResult gmres_solve<float>(KrylovWs<float>&, const Op&, float*, const float*,
                                        const float*, const PrecFn<float>*, double, int, int&,
                                        Driver&, const int*, bool);
template SolveResult bicgstab_solve<double>(KrylovWs<double>&, const Op&, double*, const double*,
                                            const double*, const PrecFn<double>*, double, int,
                                            int&, Driver&, const int*, bool);
template SolveResult bicgstab_solve<float>(KrylovWs<float>&, const Op&, float*, const float*,
                                           const float*, const PrecFn<float>*, double, int, int&,
                                           Driver&, const int*, bool);

}  // namespace cahn
