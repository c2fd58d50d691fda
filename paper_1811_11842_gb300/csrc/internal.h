// Host-side declarations shared by the translation units of the library.
#pragma once
#include <utility>

#include "common.cuh"

namespace cahn {

// Launch `kernel` on stream s; throws CudaError if the launch is rejected.
template <typename... P, typename... A>
inline void launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    CAHN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...));
}

// Operator kinds (matrix-free).
enum OpKind {
    OP_LAP5_NEUMANN = 0,   // c0 x + cx (2x - xw - xe) + cy (2x - xs - xn), even reflection at walls
    OP_LAP5_DIRICHLET = 1, // same on interior rows (wall neighbours as stored); c0 x on wall rows
    OP_CH13 = 2,           // idt x + 1/2 G_a (kx Lx + ky Ly + S) x  (13-point)
    OP_CH13_WADJ = 3,      // idt x + 1/2 (kx Lx + ky Ly + S) G_a x: the W-adjoint of OP_CH13
    OP_NUT5 = 4,           // dg x + sum over faces f of (a_c + a_f) g_f (x - x_f), zero flux
                           // on both walls; with nut_dtop, dg x on row ny (Dirichlet)
    OP_VISC = 5            // rho/dt v - 1/2 div(2 eta D(v)) on stacked [u; v] (visc.cu)
};

// Operator descriptor passed by value to kernels.  For OP_CH13 the
// coefficient field `a` has the element type of the solve.
struct Op {
    Grid g;
    int kind;
    double c0, cx, cy;      // lap5 (cx = nu/hx^2, cy = nu/hy^2)
    double kx, ky, S, idt;  // ch13: kappa/hx^2, kappa/hy^2, S, 1/dt
    double gx, gy;          // ch13: 1/hx^2, 1/hy^2
    const void* a;          // ch13 coefficient field; OP_NUT5: a = D_s phi_s / 4 (T*)
    const void* dg = nullptr;   // OP_NUT5: diagonal field (T*)
    int nut_dtop = 0;           // OP_NUT5: row ny is a Dirichlet row
    int ty = TILE_Y;        // output tile height (8, 16, 32) of the launches without
                            // reductions (apply, multigrid residual, Chebyshev step)
};

// Fused epilogues of the stencil kernels.
enum Epi {
    EPI_APPLY = 0,   // y = A x
    EPI_RESID = 1,   // y = b - A x; BN = ||b||_W, RR = ||y||^2_W, done if RR <= (rtol BN)^2
    EPI_DOTXY = 2,   // y = A x; PQ = <x,y>_W, ALPHA = RZ / PQ       (CG)
    EPI_NORM  = 3,   // y = A x; TMP0 = <y,y>_W                       (norms of A x)
    EPI_RPLAIN = 4,  // y = b - A x, no reduction (multigrid residual)
    EPI_CHEB = 5,    // Chebyshev-Jacobi step: d = c1 d + c2 dinv (b - A x); y = x + d
    EPI_CHEB_Z = 6,  // the same step when the previous d equals x (second step from x = 0)
    EPI_RESIDX = 7,  // EPI_RESID, plus TMP2 = <x,x>_W (the refinement's rounding floor)
    EPI_CGCG = 8     // y = A x with x = z and b = r: RZ = <r,z>_W, <z,Az>_W, then the
                     // ALPHA and BETA of the Chronopoulos-Gear CG iteration
};

// How a stencil kernel forms its input x at a node (the multigrid smoother
// fuses the step before it into the load):
enum XLoad {
    XL_PLAIN = 0,    // x as stored
    XL_ZERO = 1,     // x = c dinv b: the first Chebyshev step from x = 0 (c = coef[1])
    XL_PROLONG = 2   // x + P x_c: the coarse-grid correction, added on the fly
};

// Rows of a multigrid correction held at zero (Dirichlet rows): dz = 0
// none, 1 both wall rows, 2 the top wall row only (the nutrient operator).
__host__ __device__ inline bool dz_row(int dz, int j, int ny) {
    return dz == 1 ? (j == 0 || j == ny) : (dz == 2 && j == ny);
}

// One node of the 5-point operators, shared by the stencil and multigrid
// kernels so that both round it alike.  FP32: sums of neighbour
// differences (each exact for close values) keep ~1 ulp relative accuracy
// where the expanded form cancels O(h^-2) terms.
template <typename T>
struct Lap5C {
    T c0, cx, cy, cc;
};
template <typename T>
__host__ __device__ inline Lap5C<T> lap5_consts(const Op& op) {
    return Lap5C<T>{(T)op.c0, (T)op.cx, (T)op.cy, (T)(op.c0 + 2.0 * op.cx + 2.0 * op.cy)};
}
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ T lap5_ax(const Lap5C<T>& k, T xc, T xw, T xe, T xs, T xn) {
    if (sizeof(T) == 4)
        return fma(k.cy, (xc - xs) + (xc - xn), fma(k.cx, (xc - xw) + (xc - xe), mul_rn(k.c0, xc)));
    return fma(-k.cy, xs + xn, fma(-k.cx, xw + xe, mul_rn(k.cc, xc)));
}
#endif

// Extra operands of the multigrid epilogues.  Step k of the Chebyshev
// smoother reads its coefficients (c1, c2) = coef[2k], coef[2k+1] from a
// per-level device table (see cheb_coef).
template <typename T>
struct ChebArgs {
    const T* dinv = nullptr;
    T* d = nullptr;
    const double* coef = nullptr;
    int k = 0;
    int dirichlet_zero = 0;   // rows kept at 0 on corrections (dz_row: 1 both walls, 2 top)
    const T* xc = nullptr;    // XL_PROLONG: coarse-grid correction, its grid and
    Grid gc{};                //   the coarsening (1 = y only) of this level
    int semi = 0;
    // 5-point levels: D^-1 is one value inside and one on Dirichlet wall rows
    // (the values of the dinv array), formed instead of read
    int const_dinv = 0;
    T di_int = 0, di_wall = 0;
};

// Chebyshev coefficients of step k (d = c1 d + c2 D^-1 r).
__host__ __device__ inline void cheb_coef(double lmax, double alpha, int k, double& c1,
                                          double& c2) {
    const double lmin = lmax / alpha;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta;
    if (k == 0) {
        c1 = 0.0;
        c2 = 1.0 / theta;
        return;
    }
    double rho_old = 1.0 / sigma, rho = rho_old;
    for (int i = 1; i <= k; ++i) {
        rho_old = rho;
        rho = 1.0 / (2.0 * sigma - rho_old);
    }
    c1 = rho * rho_old;
    c2 = 2.0 * rho / delta;
}

struct SolveDev {      // device pointers of one solve's bookkeeping
    double* scal;      // [S_COUNT]
    Ctl* ctl;
    RedWs red;
    double anorm = 0.0;   // EPI_RESIDX: ||A|| for the refinement's rounding floor
};

// ---- stencil.cu
// y = A x with epilogue `epi`; kernels return at once while *gate != 0.
// Tile height (8, 16 or 32) of op's launches without reductions, picked by
// timing candidates on stream s (cached per kind, precision and grid).
template <typename T>
int tune_tile(const Op& op, cudaStream_t s);
int forced_tile_height();

template <typename T>
void launch_op(const Op& op, Epi epi, const T* x, const T* b, T* y, SolveDev sd,
               const int* gate, double rtol, cudaStream_t s);
template <typename T>
void launch_cheb(const Op& op, const T* x, const T* b, T* y, const ChebArgs<T>& ca,
                 const int* gate, cudaStream_t s, int xl = XL_PLAIN);
// ---- stencil_vec.cu: vectorised 128-column tiles of the lap5, nut5 and
// ch13 operators for fine grids (nx a multiple of 4, >= 128, 16-byte aligned
// vectors); each node is evaluated as by the general tiles of stencil.cu.
template <typename T>
bool vec_eligible(const Op& op, int epi, const void* x, const void* b, const void* y,
                  const ChebArgs<T>& ca, const SolveDev& sd);
template <typename T, int EPI, int XL>
void launch_vec(const Op& op, const T* x, const T* b, T* y, SolveDev sd, const int* gate,
                double rtol, cudaStream_t s, const ChebArgs<T>& ca);
template <typename T>
void launch_ch13_diag(const Op& op, T* diag, cudaStream_t s);
// Chebyshev step tables that the last block of a set-up launch writes from
// the spectral bound lam it reduced: up to three (steps, table), each on
// [lam/alpha, lam].  On that interval sigma = theta/delta does not depend
// on lam, so c1 does not either and c2 scales as 1/lam: the table is the one
// for lam = 1 (norm, formed on the host by cheb_coef) with every c2 divided
// by lam, entries in parallel.
struct ChebTabs {
    int n = 0;
    int count[3] = {0, 0, 0};
    const double* norm[3] = {nullptr, nullptr, nullptr};
    double* coef[3] = {nullptr, nullptr, nullptr};
    void add(const double* nt, int c, double* p) {
        norm[n] = nt;
        count[n] = c;
        coef[n] = p;
        ++n;
    }
};
// One level of a phase-field hierarchy's coefficient set-up, one launch:
// dinv = 1 / diag(A_phi) and *lam = max_i (Gershgorin row bound / D_ii)
// (exact for the checkerboard mode) by the last-block reduction; the
// coefficient op.a restricted to the next level (into ac on grid gc with
// coarsening semi; skipped when ac is null); and the tables of tabs, from
// lam, by the last block.  The launch returns at once while *gate != 0
// (gate may be null).
template <typename T>
void launch_ch13_level(const Op& op, T* dinv, double* lam, RedWs red, const Grid& gc, int semi,
                       T* ac, const ChebTabs& tabs, const int* gate, cudaStream_t s);
// the same for the nutrient operator (OP_NUT5: D = dg + S, R = dg + 2 S, S
// the face-coefficient sum; R / D = 1 on a Dirichlet row), restricting both
// coefficient fields a and dg (into ac and dgc)
template <typename T>
void launch_nut_level(const Op& op, T* dinv, double* lam, RedWs red, const Grid& gc, int semi,
                      T* ac, T* dgc, const ChebTabs& tabs, cudaStream_t s);

// GMRES small dense state (device, FP64): column-major Hessenberg H
// [(m+1) x m] with leading dimension ldh, Givens cosines / sines, the
// rotated right-hand side g and the least-squares solution y.
struct GmDev {
    double* H;
    int ldh;
    double *cs, *sn, *g, *y;
};

// ---- krylov.cu (vector kernels; all reductions W-weighted, FP64)
template <typename T>
void launch_copy(const T* x, T* y, size_t n, cudaStream_t s, const int* gate = nullptr);
template <typename Ts, typename Td>
void launch_convert(const Ts* x, Td* y, size_t n, cudaStream_t s);
void launch_fill(double* y, double v, size_t n, cudaStream_t s);
template <typename T>
void launch_zero(T* y, size_t n, const int* gate, cudaStream_t s);
// reset a solve's control block; with *gate set, mark it finished instead
void launch_ctl_init(Ctl* c, int maxit, cudaStream_t s, const int* gate = nullptr);
template <typename T>   // x = 0 if ||b|| (scal[S_BN]) is 0
void launch_zero_if_b0(size_t n, T* x, const double* scal, cudaStream_t s);
void launch_set_cond(cudaGraphConditionalHandle h, const int* stop, unsigned* counter,
                     cudaStream_t s);
template <typename T>   // x = b / c0 on the wall rows (velocity predictor)
void launch_dirichlet_walls(const Grid& g, T* x, const T* b, double inv_c0, cudaStream_t s);
template <typename T>   // scal[slot] = scale <x, y>_W   (y == nullptr: <x, 1>_W)
void launch_wdot(const Grid& g, const T* x, const T* y, SolveDev sd, int slot, double scale,
                 const int* gate, cudaStream_t s);
template <typename T>   // x -= *sc
void launch_sub_scalar(T* x, size_t n, const double* sc, const int* gate, cudaStream_t s);
template <typename T>
void launch_cg_update(const Grid& g, T* x, T* r, const T* p, const T* q, SolveDev sd,
                      const int* gate, cudaStream_t s);
template <typename T>
void launch_cgcg_update(const Grid& g, T* x, T* r, T* p, T* sv, const T* z, const T* w,
                        SolveDev sd, const int* gate, cudaStream_t s);
template <typename T>
void launch_cg_rz(const Grid& g, const T* r, const T* dinv, T* z, SolveDev sd, int first,
                  const int* gate, cudaStream_t s);
template <typename T>
void launch_cg_p(size_t n, const T* z, T* p, SolveDev sd, const int* gate, cudaStream_t s);
template <typename T>
void launch_scale_by(size_t n, const T* dinv, const T* x, T* y, const int* gate,
                     cudaStream_t s);
template <typename T>
void launch_invert(size_t n, T* d, cudaStream_t s);
template <typename T>
void launch_add(size_t n, T* x, const T* y, const T* dinv, const int* gate, cudaStream_t s);
// x = 0, r = b with the residual bookkeeping (BN, RR, RES0, TOL2, done)
template <typename T>
void launch_start_zero(const Grid& g, const T* b, T* x, T* r, SolveDev sd, double rtol,
                       const int* gate, cudaStream_t s);
// BiCGStab vector steps (see krylov.cu)
template <typename T>
void launch_bicg_init(size_t n, const T* r, T* rhat, T* p, T* v, double* scal, const int* gate,
                      cudaStream_t s);
template <typename T>
void launch_bicg_rho(const Grid& g, const T* rhat, const T* r, SolveDev sd, const int* gate,
                     cudaStream_t s);
template <typename T>
void launch_bicg_p(size_t n, const T* r, T* p, const T* v, const double* scal, const int* gate,
                   cudaStream_t s);
template <typename T>
void launch_bicg_alpha(const Grid& g, const T* rhat, const T* v, SolveDev sd, const int* gate,
                       cudaStream_t s);
template <typename T>
void launch_bicg_s(size_t n, const T* r, const T* v, T* sv, const double* scal, const int* gate,
                   cudaStream_t s);
template <typename T>
void launch_bicg_omega(const Grid& g, const T* t, const T* sv, SolveDev sd, const int* gate,
                       cudaStream_t s);
template <typename T>
void launch_bicg_x(const Grid& g, T* x, T* r, const T* phat, const T* shat, const T* sv,
                   const T* t, SolveDev sd, const int* gate, cudaStream_t s);
template <typename T>
void launch_gm_start(const Grid& g, const T* r, T* V0, T* vk, SolveDev sd, GmDev gm,
                     cudaStream_t s);
// Arnoldi step on column k (device counter); with Z (flexible GMRES) the
// iteration's preconditioned vector z is stored as column k of Z.
template <typename T>
void launch_gm_arnoldi(const Grid& g, T* w, T* V, size_t ldv, T* vk, SolveDev sd, GmDev gm,
                       int m, cudaStream_t s, const T* z = nullptr, T* Z = nullptr);
// y = R^-1 g, then out = V y; out += dinv (V y) (Jacobi); or, with add,
// out += V y (flexible GMRES: V is the preconditioned basis)
template <typename T>
void launch_gm_update(const Grid& g, const T* V, size_t ldv, T* out, const T* dinv, SolveDev sd,
                      GmDev gm, cudaStream_t s, int add = 0);
void launch_gm_finish(Ctl* c, cudaStream_t s);
void launch_ir_down(size_t n, const double* r, float* r32, const double* scal, const int* gate,
                    cudaStream_t s);
void launch_ir_up(size_t n, double* x, const float* d32, const double* scal, const int* gate,
                  cudaStream_t s);

}  // namespace cahn
