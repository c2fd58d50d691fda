// Host drivers of the Krylov solves (CG, restarted GMRES) and of the
// mixed-precision refinement over matrix-free operators.  All scalars stay
// on the device.  The same driver code runs in two modes:
//   host mode   -- kernels are queued on the stream; the host reads the
//                  control block back between chunks of iterations;
//   graph mode  -- the calls are captured into a CUDA graph; every
//                  convergence loop becomes a conditional WHILE node whose
//                  condition a kernel sets from the device flag.
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
    T* Z = nullptr;            // flexible GMRES: the preconditioned basis M V (or null)
    GmDev gm{};
    SolveDev sd{};
    Ctl* h_ctl = nullptr;      // pinned mirrors
    double* h_scal = nullptr;
    std::vector<void*> allocs;

    // flexible: keep the preconditioned basis (GMRES with a V-cycle)
    void alloc(const Grid& grid, int restart, bool gmres, RedWs red, bool flexible = false);
    void release();
    void read_back(cudaStream_t s);   // copies ctl + scalars to the host mirrors and syncs
};

struct SolveResult {
    int it = 0;
    int status = 0;
    double rel_res = 0.0;     // last (true or estimated) ||r||_W / ||b||_W
};

// Kernel executions of a captured graph: kernels outside any loop, kernels
// directly inside each loop body, and a device counter of body executions.
struct GraphCount {
    int64_t top = 0;
    std::vector<int64_t> body;
    unsigned* d_counters = nullptr;   // [capacity]
    int capacity = 0;
    int add_loop();
};

struct Driver {
    cudaStream_t s = nullptr;
    bool graph = false;
    std::vector<cudaStream_t>* pool = nullptr;   // capture streams, one per nesting depth
    int depth = 0;
    GraphCount* gc = nullptr;
};

// Run `body` while *stop == 0 (body launches on the Driver it is given).
// Host mode: `predict` bodies at a time, then `poll()` (reads the flag);
// at most `cap` bodies.  Graph mode: a conditional WHILE node.
void loop_while(Driver& d, const int* stop, const std::function<void(Driver&)>& body,
                int predict, int cap, const std::function<bool()>& poll);

// Kernel launches noted while capturing are attributed to this counter.
void set_launch_frame(int64_t* frame);

// zero_guess: start from x = 0 whatever x holds (no operator application
// for the first residual)
template <typename T>
SolveResult cg_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                     const PrecFn<T>* prec, double rtol, int maxit, bool project,
                     double inv_sumw, int& predict, Driver& d, const int* skip = nullptr,
                     bool zero_guess = false);

template <typename T>
SolveResult gmres_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                        const PrecFn<T>* prec, double rtol, int maxit, int& predict,
                        Driver& d, const int* skip = nullptr, bool zero_guess = false);

template <typename T>
SolveResult bicgstab_solve(KrylovWs<T>& W, const Op& op, T* x, const T* b, const T* dinv,
                           const PrecFn<T>* prec, double rtol, int maxit, int& predict,
                           Driver& d, const int* skip = nullptr, bool zero_guess = false);

// Mixed precision: FP64 iterative refinement around an FP32 inner solve.
// Each sweep forms r = b - A x in FP64 (fused with ||b||, ||r||) and stops
// when ||r||_W <= max(rtol ||b||_W, 16 eps64 (anorm ||x||_W + ||b||_W)) --
// the second term is the floor of the true residual under FP64 rounding
// (normwise backward error at unit-roundoff level), anorm an upper bound
// of ||A|| -- or when three sweeps in a row fail to reduce ||r|| by 10%;
// else it solves A d = r / ||r|| in FP32 (`inner`, zero initial guess, its
// own tolerance; skipped while *skip) and sets x += ||r|| d in FP64.
using InnerSolve =
    std::function<SolveResult(const float* rhs, float* sol, Driver& d, const int* skip)>;
struct IrResult {
    SolveResult outer;   // it = refinement sweeps, rel_res = last true FP64 residual
    int inner_it = 0;
};
IrResult ir_solve(KrylovWs<double>& W, const Op& op64, double* x, const double* b, float* r32,
                  float* d32, const InnerSolve& inner, double rtol, int max_outer, bool project,
                  double inv_sumw, double anorm, Driver& d);

}  // namespace cahn
