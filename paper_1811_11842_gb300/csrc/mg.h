// Geometric multigrid V-cycle used as the preconditioner of the Krylov
// solves (one hierarchy per system).  See mg.cu.
#pragma once
#include <vector>
#include "internal.h"
#include "mg_fused.h"

namespace cahn {

template <typename T>
struct MgLevel {
    Grid g{};
    Op op{};
    int semi = 0;            // coarsening to the next level: 1 = y only, 0 = x and y
    T *x = nullptr, *xt = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *dinv = nullptr,
      *a = nullptr, *dg = nullptr;   // a, dg: coefficient fields (OP_CH13: a; OP_NUT5: a, dg)
    double* lam = nullptr;   // device: upper bound of the spectrum of D^-1 A
    double* coef = nullptr;  // device: smoother Chebyshev table (c1, c2) per step
    double* coarse_coef = nullptr;   // coarsest level: whole-spectrum table
    std::vector<double> coef_h, coarse_coef_h;   // host copies (5-point levels)
};

// The coarse levels of a hierarchy run by one block (see k_tail_vcycle).
constexpr int TAIL_MAX = 6;
struct TailLevel {
    Op op;                 // the level's operator (its grid in op.g)
    int semi;              // coarsening to the next level
    int n;                 // nodes
    int off;               // offset of the level's 4 vectors in shared memory (elements)
    const double* coef;    // smoother table, or the whole-spectrum table (coarsest)
    double di_int, di_wall;   // 1 / diagonal: interior rows; Dirichlet wall rows
};
struct TailArgs {
    TailLevel lv[TAIL_MAX];
    int count, degree, coarse_iters, dz;
    const void* dense;     // the coarsest level's dense solve P (T*, row-major), or null
};

// The whole V-cycle of an FP32 5-point hierarchy in one cooperative launch
// (see k_vcycle_coop): every level's operator, transfer flag and vectors.
constexpr int COOP_MAX = 16;
struct CoopLevel {
    Op op;
    int semi;
    void *x, *xt, *b, *d, *r;     // level vectors (T*); level 0: x, b come per call
    const void* dinv;             // 1 / diagonal (T*; the single-block coarsest solve)
    const double* coef;           // smoother table; coarsest level: whole-spectrum table
};
struct CoopArgs {
    CoopLevel lv[COOP_MAX];
    int count, degree, coarse_iters, dz;
    int single_coarse;            // the coarsest level by one block (as k_coarse_solve)
    const void* dense;            // the coarsest level's dense solve P (T*), or null
    unsigned* bar;                // [0] arrivals, [1] generation (grid barrier)
    int* err;                     // set when a barrier wait gave up
};

// The dense exact solve of a constant-coefficient 5-point level (op.kind
// OP_LAP5_NEUMANN or OP_LAP5_DIRICHLET on op.g; rows held at zero by dz):
// P, n x n row-major in FP64, with x = P b; for the singular zero-flux
// operator its pseudo-inverse in the wall-weighted inner product.  False if
// the elimination fails.  Host only.
bool dense_solve_matrix(const Op& o, int dz, std::vector<double>& P);

template <typename T>
struct Multigrid {
    std::vector<MgLevel<T>> lv;
    // Chebyshev degree of pre- and post-smoothing: 3 for the FP32 hierarchies
    // (fewer Krylov iterations pay for the extra launch), 2 for the FP64 ones
    // (FP64-ALU-bound, where the extra step costs more than it saves)
    int degree = sizeof(T) == 4 ? 3 : 2;
    double alpha = 4.0;      // smoothing interval [lam/alpha, lam]
    int coarse_iters = 8;    // Chebyshev steps on the coarsest level
    double coarse_alpha = 20.0;
    bool single_block_coarse = false;
    // the coarsest level solved exactly, x = P b with the dense P of
    // dense_solve_matrix (constant-coefficient 5-point hierarchies of at
    // least two levels whose coarsest level has at most DENSE_MAX_NODES
    // nodes; CAHN_MG_DENSE=0 in the environment keeps the Chebyshev solve)
    T* dense = nullptr;
    int tail = -1;           // first level of the single-block tail (-1: none)
    bool schwarz = false;    // the domain-decomposition preconditioner on level 0 instead
    double* sw_coef = nullptr;   // its local Chebyshev table
    // coefficient kinds: the step tables for lam = 1 (smoother, coarsest
    // level, Schwarz), which the set-up launches scale by the reduced lam
    double* ntab = nullptr;
    bool coop = false;       // the whole V-cycle in one cooperative launch
    CoopArgs cargs{};
    int coop_blocks = 0;
    int coop_from = 0;       // first level of the cooperative launch
    bool fused = false;      // temporally blocked passes (mg_fused.cu), one launch per level
                             // and direction (FP32 5-point hierarchies)
    TailArgs targs{};
    size_t tail_smem = 0;
    bool dirichlet = false;
    int dz = 0;              // rows held at zero on corrections (dz_row)
    RedWs red{};
    std::vector<void*> allocs;

    // Build the hierarchy under `fine` (lap5 kinds: constant coefficients;
    // OP_CH13, OP_NUT5: coefficient fields allocated per level, filled by
    // set_coefficient / set_coefficients).  Coarsening stops at `max_levels` levels, when the
    // grid cannot be halved, or when it has <= `stop_nodes` nodes.  Each
    // level's tile height is tuned on stream s.
    void build(const Op& fine, int max_levels, size_t stop_nodes, RedWs r, cudaStream_t s);
    // run the levels from the first with at most coop_nodes() nodes down to
    // the coarsest as one cooperative launch of at most `blocks` blocks
    // (FP32 5-point hierarchies); the finer levels keep their separate
    // launches.  The caller keeps the blocks of all cooperative V-cycles
    // that may run at the same time within coop_capacity().
    void enable_coop(int blocks);
    // blocks of the cooperative V-cycle the device holds at once (0: none)
    static int coop_capacity();
    // largest level (nodes) the cooperative launch starts at
    static size_t coop_nodes();
    // apply the one-level Schwarz preconditioner of the fine level in place of
    // the V-cycle (the hierarchy must have been built with one level)
    void enable_schwarz();
    // OP_CH13 only; every launch returns at once while *gate != 0 (gate may be null)
    void set_coefficient(const T* a_fine, cudaStream_t s, const int* gate = nullptr);
    // OP_NUT5: the fine a and dg, restricted to every level
    void set_coefficients(const T* a_fine, const T* dg_fine, cudaStream_t s);
    // z = M r (z is overwritten); kernels return at once while *gate != 0.
    void vcycle(const T* r, T* z, const int* gate, cudaStream_t s);
    // One step k (0 <= k < 16) of the fine-level Chebyshev-Jacobi smoother on
    // the caller's vectors: d = c1(k) d + c2(k) D^-1 (b - A x), y = x + d,
    // the coefficients of the level's table (d is not read for k = 0).
    void fine_step(const T* x, const T* b, T* d, T* y, int k, cudaStream_t s);
    // The V-cycle's first pass on the fine level: deg steps from x = 0, then
    // the restricted residual into level 1's right-hand side.
    void down_pass(const T* b, T* x, cudaStream_t s);
    void release();
    size_t coarse_nodes() const { return lv.empty() ? 0 : lv.back().g.n(); }

   private:
    // the smoother's operands at level l: D^-1 (formed per row on 5-point
    // levels), the rows held at zero, the step table
    ChebArgs<T> cheb_args(int l, const double* coef) const;
    // the coarsest level: the single-block solve, else coarse_iters steps
    void coarse_solve(const T* b, T* x, const int* gate, cudaStream_t s);
    // C.b = R (b - A_l x) for level l and C = level l + 1
    void restrict_residual(int l, const T* x, const T* b, const int* gate, cudaStream_t s);
    // a temporally blocked pass on level l (the mode's fields set by the caller)
    FusedPass<T> fused_pass(int l, bool coarse, int steps, int halo, const T* b,
                            T* xout) const;
    // deg Chebyshev steps on level l; zero_init: from x = 0; xc: first add
    // the prolonged coarse correction P xc to x (fused into the first step)
    void smooth(int l, const T* b, T* x, bool zero_init, const int* gate, cudaStream_t s,
                int deg, const double* coef, const T* xc = nullptr);
};

}  // namespace cahn
