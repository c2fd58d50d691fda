// Host drivers of the Krylov solves (CG, restarted GMRES) over matrix-free
// operators.  All scalars stay on the device; the host only queues kernels
// and, in host-loop mode, reads the control block to decide when to stop.
#pragma once
#include <functional>
#include <vector>
#include "internal.h"

namespace cahn {

// z = M r  (kernels must return at once while *gate != 0)
template <typename T>
using PrecFn = std::function<void(const T* r, T* z, const int* gate, cudaStream_t s)>;

// Workspace of the Krylov solves on one grid (shared by the systems).
template <typename T>
struct KrylovWs {
    Grid g{};
    size_t n = 0;
    int m = 0;                 // GMRES restart
    T *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *w = nullptr, *u = nullptr,
      *vk = nullptr, *V = nullptr;
    GmDev gm{};
    SolveDev sd{};
    Ctl* h_ctl = nullptr;      // pinned mirrors
    double* h_scal = nullptr;
    std::vector<void*> allocs;

    void alloc(const Grid& grid, int restart, bool gmres, RedWs red);
    void release();
    void read_back(cudaStream_t s);   // copies ctl + scalars to the host mirrors and syncs
};

struct SolveResult {
    int it = 0;
    int status = 0;
    double rel_res = 0.0;     // last (true or estimated) ||r||_W / ||b||_W
};

// Loop driver: runs `body` until the control flag says stop.  In host mode
// the bodies are queued `predict` at a time (each body's kernels return at
// once after the stop flag is set) and the flag is read back in between.
struct Driver {
    cudaStream_t s = nullptr;
    int64_t* launches = nullptr;   // kernel launch counter (host side estimate)
};

template <typename T>
SolveResult cg_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                     const PrecFn<T>* prec, double rtol, int maxit, bool project,
                     double inv_sumw, int& predict, Driver& d);

template <typename T>
SolveResult gmres_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                        const PrecFn<T>* prec, double rtol, int maxit, int& predict,
                        Driver& d);

// Mixed precision: FP64 iterative refinement around an FP32 inner solve.
// Each sweep forms r = b - A x in FP64 (fused with ||b||, ||r||) and stops
// when ||r||_W <= max(rtol ||b||_W, 16 eps64 (anorm ||x||_W + ||b||_W)) --
// the second term is the floor of the true residual under FP64 rounding
// (normwise backward error at unit-roundoff level), anorm an upper bound
// of ||A|| -- or when three sweeps in a row fail to reduce ||r|| by 10%;
// else it solves A d = r / ||r|| in FP32 (`inner`, zero initial guess, its
// own tolerance) and sets x += ||r|| d in FP64.
using InnerSolve = std::function<SolveResult(const float* rhs, float* sol)>;
struct IrResult {
    SolveResult outer;   // it = refinement sweeps, rel_res = last true FP64 residual
    int inner_it = 0;
};
IrResult ir_solve(KrylovWs<double>& W, const Op& op64, double* x, const double* b, float* r32,
                  float* d32, const InnerSolve& inner, double rtol, int max_outer, bool project,
                  double inv_sumw, double anorm, Driver& d);

}  // namespace cahn
