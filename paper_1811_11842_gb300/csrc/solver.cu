// Krylov drivers: preconditioned CG in the W inner product (the velocity
// predictor and the singular pressure system are W-symmetric) and GMRES(m)
// with right preconditioning for the non-symmetric phase-field system (the
// paper's KSP choice, §4.1 Listing 4).  Convergence: ||b - A x||_W <=
// rtol ||b||_W; GMRES confirms it on the true residual at each restart.
#include <cmath>

#include "solver.h"

namespace cahn {

template <typename T>
static T* dalloc(std::vector<void*>& list, size_t count) {
    void* p = nullptr;
    CAHN_CUDA_TRY(cudaMalloc(&p, count * sizeof(T)));
    list.push_back(p);
    return static_cast<T*>(p);
}

template <typename T>
void KrylovWs<T>::alloc(const Grid& grid, int restart, bool gmres, RedWs red) {
    g = grid;
    n = grid.n();
    m = restart;
    r = dalloc<T>(allocs, n);
    z = dalloc<T>(allocs, n);
    p = dalloc<T>(allocs, n);
    q = dalloc<T>(allocs, n);
    CAHN_CUDA_TRY(cudaMemset(p, 0, n * sizeof(T)));
    if (gmres) {
        w = dalloc<T>(allocs, n);
        u = dalloc<T>(allocs, n);
        vk = dalloc<T>(allocs, n);
        V = dalloc<T>(allocs, n * (size_t)(m + 1));
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

// Queue `body` in chunks until stop(ctl) holds.
template <typename T, typename Body, typename Stop>
static void host_loop(KrylovWs<T>& W, Body body, Stop stop, int predict, int cap, Driver& d) {
    int launched = 0;
    int chunk = predict > 0 ? predict : 1;
    for (;;) {
        for (int c = 0; c < chunk; ++c) body();
        launched += chunk;
        W.read_back(d.s);
        if (stop(*W.h_ctl) || launched >= cap) break;
        chunk = launched / 4 > 1 ? launched / 4 : 1;
    }
}

template <typename T>
static void precondition(KrylovWs<T>& W, const T* dinv, const PrecFn<T>* prec, const T* in,
                         T* out, const int* gate, Driver& d) {
    if (dinv)
        launch_scale_by<T>(W.n, dinv, in, out, gate, d.s);
    else
        (*prec)(in, out, gate, d.s);
}

template <typename T>
SolveResult cg_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                     const PrecFn<T>* prec, double rtol, int maxit, bool project,
                     double inv_sumw, int& predict, Driver& d) {
    const Grid& g = op.g;
    const size_t n = g.n();
    cudaStream_t s = d.s;
    const int* done = &W.sd.ctl->done;
    launch_ctl_init(W.sd.ctl, maxit, s);
    launch_op<T>(op, EPI_RESID, x, b, W.r, W.sd, done, rtol, s);
    // Singular system: keep the residual W-orthogonal to the constants.  The
    // rounding of every update leaves a null-space component in r that no
    // iteration can remove; in FP32 it grows to ~eps32 cond(A) and stalls
    // the solve, so it is deflated after every update.
    auto deflate = [&]() {
        if (!project) return;
        launch_wdot<T>(g, W.r, (const T*)nullptr, W.sd, S_TMP3, inv_sumw, done, s);
        launch_sub_scalar<T>(W.r, n, W.sd.scal + S_TMP3, done, s);
    };
    deflate();
    if (dinv) {
        launch_cg_rz<T>(g, W.r, dinv, W.z, W.sd, 1, done, s);
    } else {
        (*prec)(W.r, W.z, done, s);
        launch_cg_rz<T>(g, W.r, nullptr, W.z, W.sd, 1, done, s);
    }
    launch_copy<T>(W.z, W.p, n, s, done);
    auto body = [&]() {
        launch_op<T>(op, EPI_DOTXY, W.p, nullptr, W.q, W.sd, done, rtol, s);
        launch_cg_update<T>(g, x, W.r, W.p, W.q, W.sd, done, s);
        deflate();
        if (dinv) {
            launch_cg_rz<T>(g, W.r, dinv, W.z, W.sd, 0, done, s);
        } else {
            (*prec)(W.r, W.z, done, s);
            launch_cg_rz<T>(g, W.r, nullptr, W.z, W.sd, 0, done, s);
        }
        launch_cg_p<T>(n, W.z, W.p, W.sd, done, s);
    };
    host_loop(W, body, [](const Ctl& c) { return c.done != 0; }, predict, maxit + 2, d);
    if (project) {
        launch_wdot<T>(g, x, (const T*)nullptr, W.sd, S_TMP3, inv_sumw, nullptr, s);
        launch_sub_scalar<T>(x, n, W.sd.scal + S_TMP3, nullptr, s);
    }
    W.read_back(s);
    if (W.h_scal[S_BN] == 0.0) CAHN_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(T), s));
    SolveResult res;
    res.it = W.h_ctl->it;
    res.status = W.h_ctl->status;
    res.rel_res = W.h_scal[S_BN] > 0 ? W.h_scal[S_RES0] / W.h_scal[S_BN] : 0.0;
    predict = res.it > 0 ? res.it : 1;
    return res;
}

template <typename T>
SolveResult gmres_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                        const PrecFn<T>* prec, double rtol, int maxit, int& predict,
                        Driver& d) {
    const Grid& g = op.g;
    const size_t n = g.n();
    cudaStream_t s = d.s;
    Ctl* c = W.sd.ctl;
    const int* done = &c->done;
    const int* cyc = &c->cycle_end;
    const int* idle = &c->idle;
    const int m = W.m;
    launch_ctl_init(c, maxit, s);
    int first_chunk = predict < m ? predict : m;
    for (int cycle = 0; cycle <= maxit; ++cycle) {
        launch_op<T>(op, EPI_RESID, x, b, W.r, W.sd, done, rtol, s);
        launch_gm_start<T>(g, W.r, W.V, W.vk, W.sd, W.gm, s);
        W.read_back(s);
        if (W.h_ctl->done) break;
        auto body = [&]() {
            precondition<T>(W, dinv, prec, W.vk, W.z, cyc, d);
            launch_op<T>(op, EPI_APPLY, W.z, nullptr, W.w, W.sd, cyc, rtol, s);
            launch_gm_arnoldi<T>(g, W.w, W.V, n, W.vk, W.sd, W.gm, m, s);
        };
        host_loop(W, body, [](const Ctl& cc) { return cc.cycle_end != 0; }, first_chunk, m, d);
        first_chunk = m;
        if (dinv) {
            launch_gm_update<T>(g, W.V, n, x, dinv, W.sd, W.gm, s);
        } else {
            launch_gm_update<T>(g, W.V, n, W.u, nullptr, W.sd, W.gm, s);
            (*prec)(W.u, W.z, idle, s);
            launch_add<T>(n, x, W.z, nullptr, idle, s);
        }
        launch_gm_finish(c, s);
    }
    SolveResult res;
    res.it = W.h_ctl->it;
    res.status = W.h_ctl->status;
    res.rel_res = W.h_scal[S_BN] > 0 ? W.h_scal[S_RES0] / W.h_scal[S_BN] : 0.0;
    if (W.h_scal[S_BN] == 0.0) CAHN_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(T), s));
    predict = res.it > 0 ? res.it : 1;
    return res;
}

IrResult ir_solve(KrylovWs<double>& W, const Op& op64, double* x, const double* b, float* r32,
                  float* d32, const InnerSolve& inner, double rtol, int max_outer, bool project,
                  double inv_sumw, double anorm, Driver& d) {
    const Grid& g = op64.g;
    const size_t n = g.n();
    cudaStream_t s = d.s;
    const int* done = &W.sd.ctl->done;
    IrResult out;
    launch_ctl_init(W.sd.ctl, max_outer, s);
    int sweeps = 0, stalls = 0;
    double last = 0.0, res = 0.0, bn = 0.0;
    bool converged = false;
    const double eps64 = 1.1102230246251565e-16;
    for (;;) {
        launch_op<double>(op64, EPI_RESID, x, b, W.r, W.sd, done, rtol, s);
        launch_wdot<double>(g, x, x, W.sd, S_TMP2, 1.0, nullptr, s);
        W.read_back(s);
        res = W.h_scal[S_RES0];
        bn = W.h_scal[S_BN];
        if (W.h_ctl->status & CTL_NAN) break;
        const double floor_ = 16.0 * eps64 * (anorm * std::sqrt(W.h_scal[S_TMP2]) + bn);
        if (W.h_ctl->done || res <= floor_) {
            converged = true;
            break;
        }
        if (sweeps > 0 && res > 0.9 * last) {
            if (++stalls >= 3) break;
        } else {
            stalls = 0;
        }
        if (sweeps >= max_outer) break;
        last = res;
        launch_ir_down(n, W.r, r32, W.sd.scal, nullptr, s);
        CAHN_CUDA_TRY(cudaMemsetAsync(d32, 0, n * sizeof(float), s));
        SolveResult ri = inner(r32, d32);
        out.inner_it += ri.it;
        if (ri.status & CTL_NAN) {
            out.outer.status |= CTL_NAN;
            break;
        }
        launch_ir_up(n, x, d32, W.sd.scal, nullptr, s);
        ++sweeps;
    }
    if (project) {
        launch_wdot<double>(g, x, (const double*)nullptr, W.sd, S_TMP3, inv_sumw, nullptr, s);
        launch_sub_scalar<double>(x, n, W.sd.scal + S_TMP3, nullptr, s);
    }
    if (bn == 0.0) CAHN_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    out.outer.it = sweeps;
    out.outer.status |= W.h_ctl->status & CTL_NAN;
    if (!converged && !(out.outer.status & CTL_NAN)) out.outer.status |= CTL_NOT_CONVERGED;
    out.outer.rel_res = bn > 0 ? res / bn : 0.0;
    return out;
}

template struct KrylovWs<double>;
template struct KrylovWs<float>;
template SolveResult cg_solve<double>(KrylovWs<double>&, const Op&, double*, const double*,
                                      const double*, const PrecFn<double>*, double, int, bool,
                                      double, int&, Driver&);
template SolveResult cg_solve<float>(KrylovWs<float>&, const Op&, float*, const float*,
                                     const float*, const PrecFn<float>*, double, int, bool,
                                     double, int&, Driver&);
template SolveResult gmres_solve<double>(KrylovWs<double>&, const Op&, double*, const double*,
                                         const double*, const PrecFn<double>*, double, int, int&,
                                         Driver&);
template SolveResult gmres_solve<float>(KrylovWs<float>&, const Op&, float*, const float*,
                                        const float*, const PrecFn<float>*, double, int, int&,
                                        Driver&);

}  // namespace cahn
