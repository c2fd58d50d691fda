// Geometric multigrid V-cycle (preconditioner of the Krylov solves).
//
// Hierarchy: vertex-centred grids, x periodic, walls kept on rows 0 and ny.
// A level is halved in y only while the y-coupling is the stronger one
// (hx > sqrt(2) hy: semicoarsening for the anisotropic 1024 x 1024 grid on
// [0,4] x [0,1]), in both directions otherwise.  Coarse operators are the
// same operators rediscretised on the coarse grid (for the phase-field
// operator with the restricted mobility coefficient, for the nutrient
// operator with its restricted diffusion and diagonal fields).  Dirichlet
// rows of the corrections are held at zero: both wall rows of the velocity
// predictor, the top wall row of the nutrient operator.
//
// Transfers: bilinear prolongation P; restriction R = W_c^-1 P^T W_f / 4
// (1/2 for semicoarsening), the W-adjoint of P scaled so that R 1 = 1.  It
// keeps the trapezoid-weighted compatibility of the singular pressure
// problem: <R r, 1>_Wc = <r, P 1>_Wf / 4 = 0 when <r, 1>_Wf = 0.
//
// Smoother: Chebyshev polynomial in D^-1 A on [lam/alpha, lam] (degree 3
// for FP32 hierarchies, 2 for FP64), with lam the Gershgorin bound (exact
// for the 5-point operators, attained by the checkerboard mode), fused into
// the stencil kernels.  FP32 hierarchies also fuse the zero-guess step and
// the prolongation into the first smoother launches, and the 5-point
// residual into the restriction; their coarse levels that fit in shared
// memory run in one block (k_tail_vcycle).  Coarsest level: solved exactly
// by a dense matrix-vector product when the operator has constant
// coefficients and the level has at most DENSE_MAX_NODES nodes (the
// pressure's 32 x 9 level: its inverse, or pseudo-inverse for the singular
// zero-flux operator, formed once on the host); otherwise a fixed number of
// Chebyshev steps over the whole spectrum, in one single-block launch when
// the grid is small.  Every piece is a fixed linear map, so the V-cycle is
// a fixed linear preconditioner.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include "mg.h"
#include "schwarz.h"
#include "mg_fused.h"
#include "stencil_dev.cuh"

namespace cahn {

__device__ __forceinline__ size_t mg_tid() { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t mg_stride() { return (size_t)gridDim.x * blockDim.x; }

// b_c = R r_f
template <typename T>
__global__ void k_restrict(Grid gf, Grid gc, int semi, int dz, const T* __restrict__ rf,
                           T* __restrict__ bc, const int* __restrict__ gate) {
    if (gate && *gate) return;
    const size_t nc = gc.n();
    const int nx = gf.nx;
    for (size_t e = mg_tid(); e < nc; e += mg_stride()) {
        const int J = (int)(e / gc.nx), I = (int)(e - (size_t)J * gc.nx);
        if (dz_row(dz, J, gc.ny)) {
            bc[e] = (T)0;
            continue;
        }
        const int c = semi ? I : 2 * I;
        auto res = [&](int j, int dx) {
            int i = c + dx;
            i = i < 0 ? nx - 1 : (i >= nx ? 0 : i);
            return rf[(size_t)j * nx + i];
        };
        bc[e] = restrict_at<T>(res, J, gf.ny, semi, gc.ny);
    }
}

// b_c = R (b_f - A_f x_f) for the 5-point operators: the fine residual at
// the 3 (semicoarsening) or 9 fine nodes of each coarse node is formed
// where it is needed, with the arithmetic of the stencil kernels, and
// restricted as in k_restrict (one launch and no residual field instead
// of two launches).
template <typename T, int KIND>
__global__ void k_resid_restrict(Op op, Grid gc, int semi, int dz, const T* __restrict__ x,
                                 const T* __restrict__ b, T* __restrict__ bc,
                                 const int* __restrict__ gate) {
    if (gate && *gate) return;
    const Grid gf = op.g;
    const int nx = gf.nx, ny = gf.ny;
    const Lap5C<T> kc = lap5_consts<T>(op);
    const size_t nc = gc.n();
    auto res = [&](int i, int j) -> T {
        const size_t e = (size_t)j * nx + i;
        const T xc = x[e];
        if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) return b[e] - mul_rn(kc.c0, xc);
        const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
        int js, jn;
        if (KIND == OP_LAP5_NEUMANN) {
            js = j > 0 ? j - 1 : 1;
            jn = j < ny ? j + 1 : ny - 1;
        } else {
            js = j - 1;
            jn = j + 1;
        }
        const size_t row = (size_t)j * nx;
        return b[e] - lap5_ax(kc, xc, x[row + im], x[row + ip], x[(size_t)js * nx + i],
                              x[(size_t)jn * nx + i]);
    };
    for (size_t e = mg_tid(); e < nc; e += mg_stride()) {
        const int J = (int)(e / gc.nx), I = (int)(e - (size_t)J * gc.nx);
        if (dz_row(dz, J, gc.ny)) {
            bc[e] = (T)0;
            continue;
        }
        const int c = semi ? I : 2 * I;
        auto rj = [&](int j, int dx) {
            int i = c + dx;
            i = i < 0 ? nx - 1 : (i >= nx ? 0 : i);
            return res(i, j);
        };
        bc[e] = restrict_at<T>(rj, J, ny, semi, gc.ny);
    }
}

// x_f += P x_c
template <typename T>
__global__ void k_prolong_add(Grid gf, Grid gc, int semi, int dz, const T* __restrict__ xc,
                              T* __restrict__ xf, const int* __restrict__ gate) {
    if (gate && *gate) return;
    const size_t nf = gf.n();
    for (size_t e = mg_tid(); e < nf; e += mg_stride()) {
        const int j = (int)(e / gf.nx), i = (int)(e - (size_t)j * gf.nx);
        if (dz_row(dz, j, gf.ny)) continue;
        int J0 = j >> 1, J1 = J0;
        T wyv = (T)1;
        if (j & 1) {
            J1 = J0 + 1;
            wyv = (T)0.5;
        }
        T v;
        if (semi) {
            v = (j & 1) ? wyv * (xc[(size_t)J0 * gc.nx + i] + xc[(size_t)J1 * gc.nx + i])
                        : xc[(size_t)J0 * gc.nx + i];
        } else {
            int I0 = i >> 1, I1 = I0;
            T wx = (T)1;
            if (i & 1) {
                I1 = I0 + 1 < gc.nx ? I0 + 1 : 0;
                wx = (T)0.5;
            }
            auto rowv = [&](int J) {
                const T* row = xc + (size_t)J * gc.nx;
                return (i & 1) ? wx * (row[I0] + row[I1]) : row[I0];
            };
            v = (j & 1) ? wyv * (rowv(J0) + rowv(J1)) : rowv(J0);
        }
        xf[e] += v;
    }
}

// First Chebyshev step from a zero initial guess: d = dinv b / theta, x = d.
template <typename T>
__global__ void k_cheb_zero(size_t n, const T* __restrict__ b, const T* __restrict__ dinv,
                            T* __restrict__ d, T* __restrict__ x, const double* __restrict__ coef,
                            const int* __restrict__ gate) {
    if (gate && *gate) return;
    const T c = (T)coef[1];
    for (size_t e = mg_tid(); e < n; e += mg_stride()) {
        const T v = c * dinv[e] * b[e];
        d[e] = v;
        x[e] = v;
    }
}

// One node of A x for the single-block coarse solver (direct evaluation).
template <typename T, int KIND>
__device__ __forceinline__ T apply_node(const Op& op, const T* __restrict__ x, int i, int j) {
    const int nx = op.g.nx, ny = op.g.ny;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    auto X = [&](int ii, int jj) { return x[(size_t)jj * nx + ii]; };
    // neighbour-difference form (accurate in FP32, see k_lap5)
    auto lap5 = [&](int js, int jn) {
        const T c = X(i, j);
        return (T)op.c0 * c + (T)op.cx * ((c - X(im, j)) + (c - X(ip, j))) +
               (T)op.cy * ((c - X(i, js)) + (c - X(i, jn)));
    };
    if (KIND == OP_LAP5_DIRICHLET) {
        if (j == 0 || j == ny) return (T)op.c0 * X(i, j);
        return lap5(j - 1, j + 1);
    } else if (KIND == OP_LAP5_NEUMANN) {
        return lap5(j > 0 ? j - 1 : 1, j < ny ? j + 1 : ny - 1);
    } else {
        const T* a = static_cast<const T*>(op.a);
        auto psi = [&](int ii, int jj) {
            const int iw = ii > 0 ? ii - 1 : nx - 1, ie = ii < nx - 1 ? ii + 1 : 0;
            const int jjs = refly(jj - 1, ny), jjn = refly(jj + 1, ny);
            const T c = X(ii, jj);
            return (T)op.S * c + (T)op.kx * ((c - X(iw, jj)) + (c - X(ie, jj))) +
                   (T)op.ky * ((c - X(ii, jjs)) + (c - X(ii, jjn)));
        };
        const int js = refly(j - 1, ny), jn = refly(j + 1, ny);
        const T pc = psi(i, j), ac = a[(size_t)j * nx + i];
        const T fx = (ac + a[(size_t)j * nx + ip]) * (psi(ip, j) - pc) -
                     (ac + a[(size_t)j * nx + im]) * (pc - psi(im, j));
        const T fy = (ac + a[(size_t)jn * nx + i]) * (psi(i, jn) - pc) -
                     (ac + a[(size_t)js * nx + i]) * (pc - psi(i, js));
        return (T)op.idt * X(i, j) - (T)(0.25 * op.gx) * fx - (T)(0.25 * op.gy) * fy;
    }
}

// Coarsest level in one block: `iters` Chebyshev steps from x = 0 over
// [lam/alpha, lam]; x and xt ping-pong, the result ends in x.  The step
// coefficients are built once (one thread, into shared memory), and for
// grids of <= SB_SMEM_NODES nodes the iterates live in shared memory.
constexpr int SB_MAX_ITERS = 512;
constexpr int MG_KTAB = 16;   // smoother table length (degree <= 16)
constexpr int SB_SMEM_NODES = 1024;

// The body of the single-block coarsest solve, run by one block of any
// size (k_coarse_solve; the cooperative V-cycle's block 0).  CG: read the
// global vectors through L2 (data another block wrote in the same launch).
template <typename T, int KIND, bool SMEM, bool CG>
__device__ __forceinline__ void coarse_solve_block(const Op& op, const T* __restrict__ b,
                                                   const T* __restrict__ dinv, T* x, T* xt, T* d,
                                                   const double* __restrict__ coef, int iters,
                                                   int dz) {
    __shared__ T s_c1[SB_MAX_ITERS], s_c2[SB_MAX_ITERS];
    __shared__ T s_x[SMEM ? SB_SMEM_NODES : 1], s_xt[SMEM ? SB_SMEM_NODES : 1],
        s_d[SMEM ? SB_SMEM_NODES : 1], s_b[SMEM ? SB_SMEM_NODES : 1],
        s_dinv[SMEM ? SB_SMEM_NODES : 1];
    const int nx = op.g.nx;
    const size_t n = op.g.n();
    auto ld = [](const T* p, size_t e) { return CG ? __ldcg(p + e) : p[e]; };
    for (int k = threadIdx.x; k < iters; k += blockDim.x) {
        s_c1[k] = (T)coef[2 * k];
        s_c2[k] = (T)coef[2 * k + 1];
    }
    T* X = x;
    T* XT = xt;
    T* D = d;
    const T* B = b;
    const T* DI = dinv;
    if (SMEM) {
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
            s_b[e] = ld(b, e);
            s_dinv[e] = ld(dinv, e);
        }
        X = s_x;
        XT = s_xt;
        D = s_d;
        B = s_b;
        DI = s_dinv;
    }
    __syncthreads();
    for (int k = 0; k < iters; ++k) {
        const T c1 = s_c1[k], c2 = s_c2[k];
        T* out = ((iters - 1 - k) % 2 == 0) ? X : XT;
        const T* in = (out == X) ? XT : X;
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
            const int j = (int)(e / nx), i = (int)(e - (size_t)j * nx);
            if (dz_row(dz, j, op.g.ny)) {
                out[e] = (T)0;
                continue;
            }
            T dn;
            if (k == 0) {
                dn = c2 * DI[e] * B[e];
                out[e] = dn;
            } else {
                const T r = B[e] - apply_node<T, KIND>(op, in, i, j);
                dn = c1 * D[e] + c2 * DI[e] * r;
                out[e] = in[e] + dn;
            }
            D[e] = dn;
        }
        __syncthreads();
    }
    if (SMEM)
        for (size_t e = threadIdx.x; e < n; e += blockDim.x) x[e] = s_x[e];
}

template <typename T, int KIND, bool SMEM>
__global__ void __launch_bounds__(1024) k_coarse_solve(Op op, const T* __restrict__ b,
                                                       const T* __restrict__ dinv, T* x, T* xt,
                                                       T* d, const double* __restrict__ coef,
                                                       int iters, int dz,
                                                       const int* __restrict__ gate) {
    if (gate && *gate) return;
    coarse_solve_block<T, KIND, SMEM, false>(op, b, dinv, x, xt, d, coef, iters, dz);
}

// ------------------------------------------------- dense coarsest solve
// The coarsest level of a constant-coefficient 5-point hierarchy solved
// exactly: x = P b, P the n x n matrix of dense_solve_matrix (row-major, the
// level's node order).  One warp per row: an fma chain over the columns
// lane, lane + 32, ..., then a butterfly, after which every lane holds the
// same sum; the order depends neither on the caller nor on where b lives,
// so k_coarse_dense, the single-block tail and the cooperative V-cycle give
// the same bits.  CG: b was written by another block of the same launch
// (read through L2).
constexpr int DENSE_MAX_NODES = 512;

template <typename T, bool CG>
__device__ __forceinline__ T dense_row(const T* __restrict__ P, const T* b, int row, int n,
                                       int lane) {
    const T* pr = P + (size_t)row * n;
    T acc = (T)0;
    for (int k = lane; k < n; k += 32) acc = fma(__ldg(pr + k), CG ? __ldcg(b + k) : b[k], acc);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_coarse_dense(const T* __restrict__ P,
                                                      const T* __restrict__ b, T* __restrict__ x,
                                                      int n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    const int row = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;   // warp-uniform
    const T v = dense_row<T, false>(P, b, row, n, lane);
    if (lane == 0) x[row] = v;
}

// Tail of the V-cycle in one block (FP32 5-point hierarchies): the levels
// from the first tail level -- its right-hand side in global memory,
// restricted by the level above -- down to the coarsest, with every vector
// in shared memory: Chebyshev smoothing from zero, the fine residual formed
// where the restriction needs it, the whole-spectrum coarsest solve,
// prolongation and post-smoothing, each pass followed by a block barrier.
// The arithmetic per node is that of the multi-launch path (lap5_ax, the
// fused zero-guess step, the restriction and prolongation weights).  One
// launch replaces about 13 on the pressure hierarchy's coarse levels.
template <typename T, int KIND>
__global__ void __launch_bounds__(1024) k_tail_vcycle(TailArgs ta, const T* __restrict__ bg,
                                                      T* __restrict__ xg,
                                                      const int* __restrict__ gate) {
    if (gate && *gate) return;
    extern __shared__ unsigned char tail_smem[];
    T* sm = reinterpret_cast<T*>(tail_smem);
    const int nl = ta.count, tid = threadIdx.x, nt = blockDim.x;
    auto X = [&](int l) { return sm + ta.lv[l].off; };
    auto XT = [&](int l) { return sm + ta.lv[l].off + ta.lv[l].n; };
    auto Bv = [&](int l) { return sm + ta.lv[l].off + 2 * ta.lv[l].n; };
    auto Dv = [&](int l) { return sm + ta.lv[l].off + 3 * ta.lv[l].n; };
    auto dinv_at = [&](int l, int j) {
        const TailLevel& tl = ta.lv[l];
        return (T)((KIND == OP_LAP5_DIRICHLET && (j == 0 || j == tl.op.g.ny)) ? tl.di_wall : tl.di_int);
    };
    // A v at node (i, j) of level l (v in shared memory)
    auto ax_at = [&](int l, const T* v, int i, int j) {
        const Op& o = ta.lv[l].op;
        const int nx = o.g.nx, ny = o.g.ny;
        const Lap5C<T> kc = lap5_consts<T>(o);
        const T c = v[j * nx + i];
        if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) return mul_rn(kc.c0, c);
        const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
        int js, jn;
        if (KIND == OP_LAP5_NEUMANN) {
            js = j > 0 ? j - 1 : 1;
            jn = j < ny ? j + 1 : ny - 1;
        } else {
            js = j - 1;
            jn = j + 1;
        }
        return lap5_ax(kc, c, v[j * nx + im], v[j * nx + ip], v[js * nx + i], v[jn * nx + i]);
    };
    // deg Chebyshev steps on level l with table coef; from zero (x = 0) or
    // from the current x; the result ends in X(l)
    auto smooth = [&](int l, const double* coef, int deg, bool zero) {
        const Grid g = ta.lv[l].op.g;
        const int n = (int)g.n();
        T* cur = X(l);
        T* nxt = XT(l);
        T* d = Dv(l);
        const T* b = Bv(l);
        for (int k = 0; k < deg; ++k) {
            const T c1 = (T)coef[2 * k], c2 = (T)coef[2 * k + 1];
            for (int e = tid; e < n; e += nt) {
                const int j = e / g.nx, i = e - j * g.nx;
                if (ta.dz && (j == 0 || j == g.ny)) {
                    nxt[e] = (T)0;
                    continue;
                }
                const T di = dinv_at(l, j);
                T dn, xv;
                if (zero && k == 0) {
                    dn = mul_rn(mul_rn(c2, di), b[e]);
                    xv = (T)0;
                } else {
                    const T r = b[e] - ax_at(l, cur, i, j);
                    dn = fma(mul_rn(c2, di), r, c1 != (T)0 ? mul_rn(c1, d[e]) : (T)0);
                    xv = cur[e];
                }
                d[e] = dn;
                nxt[e] = xv + dn;
            }
            __syncthreads();
            T* t = cur;
            cur = nxt;
            nxt = t;
        }
        if (cur != X(l)) {
            for (int e = tid; e < n; e += nt) X(l)[e] = cur[e];
            __syncthreads();
        }
    };
    // b_{l+1} = R (b_l - A_l x_l)
    auto resid_restrict = [&](int l) {
        const Grid gf = ta.lv[l].op.g, gc = ta.lv[l + 1].op.g;
        const int semi = ta.lv[l].semi, nc = (int)gc.n();
        const T* x = X(l);
        const T* b = Bv(l);
        T* bc = Bv(l + 1);
        auto res = [&](int i, int j) { return b[j * gf.nx + i] - ax_at(l, x, i, j); };
        for (int e = tid; e < nc; e += nt) {
            const int J = e / gc.nx, I = e - J * gc.nx;
            if (ta.dz && (J == 0 || J == gc.ny)) {
                bc[e] = (T)0;
                continue;
            }
            const int c = semi ? I : 2 * I;
            auto rj = [&](int j, int dx) {
                int i = c + dx;
                i = i < 0 ? gf.nx - 1 : (i >= gf.nx ? 0 : i);
                return res(i, j);
            };
            bc[e] = restrict_at<T>(rj, J, gf.ny, semi, gc.ny);
        }
        __syncthreads();
    };
    // x_l += P x_{l+1}
    auto prolong_add = [&](int l) {
        const Grid gf = ta.lv[l].op.g, gc = ta.lv[l + 1].op.g;
        const int semi = ta.lv[l].semi, n = (int)gf.n();
        const T* xc = X(l + 1);
        T* x = X(l);
        for (int e = tid; e < n; e += nt) {
            const int j = e / gf.nx, i = e - j * gf.nx;
            if (ta.dz && (j == 0 || j == gf.ny)) continue;
            const int J0 = j >> 1, J1 = (j & 1) ? J0 + 1 : J0;
            auto rowv = [&](int J) {
                const T* row = xc + J * gc.nx;
                if (semi) return row[i];
                const int I0 = i >> 1;
                if (!(i & 1)) return row[I0];
                const int I1 = I0 + 1 < gc.nx ? I0 + 1 : 0;
                return (T)0.5 * (row[I0] + row[I1]);
            };
            x[e] += (j & 1) ? (T)0.5 * (rowv(J0) + rowv(J1)) : rowv(J0);
        }
        __syncthreads();
    };
    {
        const int n0 = (int)ta.lv[0].op.g.n();
        for (int e = tid; e < n0; e += nt) Bv(0)[e] = bg[e];
        __syncthreads();
    }
    for (int l = 0; l < nl - 1; ++l) {
        smooth(l, ta.lv[l].coef, ta.degree, true);
        resid_restrict(l);
    }
    if (ta.dense) {   // x = P b, a warp per row
        const int n = ta.lv[nl - 1].n;
        const T* P = static_cast<const T*>(ta.dense);
        for (int row = tid >> 5; row < n; row += nt >> 5) {
            const T v = dense_row<T, false>(P, Bv(nl - 1), row, n, tid & 31);
            if ((tid & 31) == 0) X(nl - 1)[row] = v;
        }
        __syncthreads();
    } else {
        smooth(nl - 1, ta.lv[nl - 1].coef, ta.coarse_iters, true);
    }
    for (int l = nl - 2; l >= 0; --l) {
        prolong_add(l);
        smooth(l, ta.lv[l].coef, ta.degree, false);
    }
    {
        const int n0 = (int)ta.lv[0].op.g.n();
        for (int e = tid; e < n0; e += nt) xg[e] = X(0)[e];
    }
}

// ------------------------------------------------- cooperative V-cycle
// The whole V-cycle of an FP32 5-point hierarchy (all levels) in one
// cooperative launch: one block of COOP_THREADS per SM walks every pass of
// the multi-launch path -- the fused zero-guess smoother step, the further
// Chebyshev steps, the residual formed at the restriction points, the
// coarsest level's steps, the smoother steps with the prolongation fused
// into their loads -- with the same per-node operations (lap5_ax, the
// step formulas, the restriction and prolongation weights), so the result
// is bit for bit that of the separate launches.  Passes are separated by a
// grid barrier; data written by an earlier pass is read through L2
// (ld.global.cg), since L1 is not coherent between SMs.

constexpr int COOP_THREADS = 512;
// The cooperative launch starts at the first level with at most COOP_NODES
// nodes (CAHN_COOP_NODES overrides): finer levels run the vectorised tiles
// as separate launches, which use the SMs better than grid-stride passes.
constexpr size_t COOP_NODES = 1u << 17;
constexpr int COOP_NODES_PER_THREAD = 2;
// A barrier wait gives up after COOP_SPIN polls (about a second), sets the
// error word and lets the kernel run to its end: the V-cycle then returns
// NaN, which the Krylov solve reports as CAHN_ERR_NAN.  Nothing waits
// without a bound.
constexpr unsigned COOP_SPIN = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void coop_sync(unsigned* bar, int* err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire_u32(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else if (!*(volatile int*)err) {
            unsigned it = 0;
            while (ld_acquire_u32(bar + 1) == gen) {
                if (++it > COOP_SPIN) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T ldg_cg(const T* p, size_t e) {
    return __ldcg(p + e);
}

template <typename T, int KIND>
__global__ void __launch_bounds__(COOP_THREADS) k_vcycle_coop(CoopArgs A, const T* __restrict__ r0,
                                                              T* __restrict__ z0,
                                                              const int* __restrict__ gate) {
    if (gate && *gate) return;
    const int nl = A.count, dz = A.dz;
    const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gs = (size_t)gridDim.x * blockDim.x;
    auto Xp = [&](int l) { return l == 0 ? z0 : static_cast<T*>(A.lv[l].x); };
    auto XTp = [&](int l) { return static_cast<T*>(A.lv[l].xt); };
    auto Bp = [&](int l) -> const T* { return l == 0 ? r0 : static_cast<const T*>(A.lv[l].b); };
    auto sync = [&]() { coop_sync(A.bar, A.err); };

    // One Chebyshev step (index k of table coef) on level l: y = in + d',
    // d' = c1 d + c2 D^-1 (b - A in), with `in` formed as XL says (XL_ZERO:
    // c2(0) D^-1 b; XL_PROLONG: in + P xc); CHZ: the step after the zero
    // guess (d = in).  The per-node arithmetic of k_lap5 and load_x.
    auto cheb_pass = [&](int l, int xl, bool chz, const T* in, T* y, int k, const double* coef,
                         const T* xc) {
        const CoopLevel& Lv = A.lv[l];
        const Op& op = Lv.op;
        const int nx = op.g.nx, ny = op.g.ny;
        const size_t n = op.g.n();
        const Lap5C<T> kc = lap5_consts<T>(op);
        const T c1 = (T)coef[2 * k], c2 = (T)coef[2 * k + 1], cz = (T)coef[1];
        const T di_int = (T)(1.0 / (op.c0 + 2 * op.cx + 2 * op.cy));
        const T di_wall = op.c0 != 0.0 ? (T)(1.0 / op.c0) : (T)0;
        const T* b = Bp(l);
        T* d = static_cast<T*>(Lv.d);
        auto di_of = [&](int j) {
            return (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) ? di_wall : di_int;
        };
        Grid gc{};
        if (xl == XL_PROLONG) gc = A.lv[l + 1].op.g;
        auto prolong = [&](int i, int j) -> T {
            if (dz_row(dz, j, ny)) return (T)0;
            const int ncx = gc.nx;
            const int J0 = j >> 1, J1 = (j & 1) ? J0 + 1 : J0;
            auto rowv = [&](int J) {
                const size_t r = (size_t)J * ncx;
                if (Lv.semi) return ldg_cg(xc, r + i);
                const int I0 = i >> 1;
                if (!(i & 1)) return ldg_cg(xc, r + I0);
                const int I1 = I0 + 1 < ncx ? I0 + 1 : 0;
                return (T)0.5 * (ldg_cg(xc, r + I0) + ldg_cg(xc, r + I1));
            };
            return (j & 1) ? (T)0.5 * (rowv(J0) + rowv(J1)) : rowv(J0);
        };
        auto X = [&](int i, int j) -> T {
            const size_t e = (size_t)j * nx + i;
            if (xl == XL_ZERO) return mul_rn(mul_rn(cz, di_of(j)), ldg_cg(b, e));
            if (xl == XL_PROLONG) return ldg_cg(in, e) + prolong(i, j);
            return ldg_cg(in, e);
        };
        for (size_t e = gt; e < n; e += gs) {
            const int j = (int)(e / nx), i = (int)(e - (size_t)j * nx);
            const T xcv = X(i, j);
            T ax;
            if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) {
                if (dz) {
                    y[e] = (T)0;
                    continue;
                }
                ax = mul_rn(kc.c0, xcv);
            } else {
                const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
                int js, jn;
                if (KIND == OP_LAP5_NEUMANN) {
                    js = j > 0 ? j - 1 : 1;
                    jn = j < ny ? j + 1 : ny - 1;
                } else {
                    js = j - 1;
                    jn = j + 1;
                }
                ax = lap5_ax(kc, xcv, X(im, j), X(ip, j), X(i, js), X(i, jn));
            }
            const T r = ldg_cg(b, e) - ax;
            const T di = di_of(j);
            T dn;
            if (chz)
                dn = fma(mul_rn(c2, di), r, mul_rn(c1, xcv));
            else
                dn = fma(mul_rn(c2, di), r, c1 != (T)0 ? mul_rn(c1, ldg_cg(d, e)) : (T)0);
            d[e] = dn;
            y[e] = xcv + dn;
        }
        sync();
    };
    // deg steps on level l (smooth() of the multi-launch path)
    auto smooth = [&](int l, bool zero, int deg, const double* coef, const T* xc) {
        T* x = Xp(l);
        T* xt = XTp(l);
        auto out_of = [&](int k) { return ((deg - 1 - k) % 2 == 0) ? x : xt; };
        int k0 = 0;
        if (zero) {
            cheb_pass(l, XL_ZERO, true, nullptr, out_of(1), 1, coef, nullptr);
            k0 = 2;
        } else {
            if (out_of(0) != x) {
                cheb_pass(l, XL_PROLONG, false, x, out_of(0), 0, coef, xc);
                k0 = 1;
            } else {
                T* r = static_cast<T*>(A.lv[l].r);
                cheb_pass(l, XL_PROLONG, false, x, r, 0, coef, xc);
                cheb_pass(l, XL_PLAIN, false, r, out_of(1), 1, coef, nullptr);
                k0 = 2;
            }
        }
        for (int k = k0; k < deg; ++k) {
            T* o = out_of(k);
            cheb_pass(l, XL_PLAIN, false, (o == x) ? xt : x, o, k, coef, nullptr);
        }
    };
    // b_{l+1} = R (b_l - A_l x_l) (k_resid_restrict)
    auto resid_restrict = [&](int l) {
        const Op& op = A.lv[l].op;
        const Grid gf = op.g, gc = A.lv[l + 1].op.g;
        const int nx = gf.nx, ny = gf.ny, semi = A.lv[l].semi;
        const Lap5C<T> kc = lap5_consts<T>(op);
        const T* x = Xp(l);
        const T* b = Bp(l);
        T* bc = static_cast<T*>(A.lv[l + 1].b);
        const size_t nc = gc.n();
        auto res = [&](int i, int j) -> T {
            const size_t e = (size_t)j * nx + i;
            const T xcv = ldg_cg(x, e);
            if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny))
                return ldg_cg(b, e) - mul_rn(kc.c0, xcv);
            const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
            int js, jn;
            if (KIND == OP_LAP5_NEUMANN) {
                js = j > 0 ? j - 1 : 1;
                jn = j < ny ? j + 1 : ny - 1;
            } else {
                js = j - 1;
                jn = j + 1;
            }
            const size_t row = (size_t)j * nx;
            return ldg_cg(b, e) - lap5_ax(kc, xcv, ldg_cg(x, row + im), ldg_cg(x, row + ip),
                                          ldg_cg(x, (size_t)js * nx + i),
                                          ldg_cg(x, (size_t)jn * nx + i));
        };
        for (size_t e = gt; e < nc; e += gs) {
            const int J = (int)(e / gc.nx), I = (int)(e - (size_t)J * gc.nx);
            if (dz_row(dz, J, gc.ny)) {
                bc[e] = (T)0;
                continue;
            }
            const int c = semi ? I : 2 * I;
            auto rj = [&](int j, int dx) {
                int i = c + dx;
                i = i < 0 ? nx - 1 : (i >= nx ? 0 : i);
                return res(i, j);
            };
            bc[e] = restrict_at<T>(rj, J, ny, semi, gc.ny);
        }
        sync();
    };
    for (int l = 0; l < nl - 1; ++l) {
        smooth(l, true, A.degree, A.lv[l].coef, nullptr);
        resid_restrict(l);
    }
    if (A.single_coarse) {
        // the coarsest solve of the separate launches: the dense solve over
        // the grid's warps, else the single-block Chebyshev steps in block 0
        const CoopLevel& C = A.lv[nl - 1];
        if (A.dense) {   // x = P b, the grid's warps over the rows
            const int n = (int)C.op.g.n();
            const T* P = static_cast<const T*>(A.dense);
            for (int row = (int)(gt >> 5); row < n; row += (int)(gs >> 5)) {
                const T v = dense_row<T, true>(P, Bp(nl - 1), row, n, (int)(gt & 31));
                if ((gt & 31) == 0) Xp(nl - 1)[row] = v;
            }
        } else if (blockIdx.x == 0) {
            if (C.op.g.n() <= (size_t)SB_SMEM_NODES)
                coarse_solve_block<T, KIND, true, true>(C.op, Bp(nl - 1), static_cast<const T*>(C.dinv),
                                                        Xp(nl - 1), XTp(nl - 1), static_cast<T*>(C.d),
                                                        C.coef, A.coarse_iters, dz);
            else
                coarse_solve_block<T, KIND, false, true>(C.op, Bp(nl - 1), static_cast<const T*>(C.dinv),
                                                         Xp(nl - 1), XTp(nl - 1), static_cast<T*>(C.d),
                                                         C.coef, A.coarse_iters, dz);
        }
        sync();
    } else {
        smooth(nl - 1, true, A.coarse_iters, A.lv[nl - 1].coef, nullptr);
    }
    for (int l = nl - 2; l >= 0; --l) smooth(l, false, A.degree, A.lv[l].coef, Xp(l + 1));
    if (*(volatile int*)A.err) {
        const size_t n0 = A.lv[0].op.g.n();
        for (size_t e = gt; e < n0; e += gs) z0[e] = (T)NAN;
    }
}

// ------------------------------------------------------------------ host
template <typename T>
static T* mg_alloc(std::vector<void*>& list, size_t count) {
    void* p = nullptr;
    CAHN_CUDA_TRY(cudaMalloc(&p, count * sizeof(T)));
    list.push_back(p);
    return static_cast<T*>(p);
}

// Chebyshev step table (c1, c2) for k < count, computed on the host (also
// returned, for the kernels that take the coefficients as arguments).
static std::vector<double> host_table(double lmax, double alpha, int count, double* dev) {
    std::vector<double> t(2 * (size_t)count);
    for (int k = 0; k < count; ++k) cheb_coef(lmax, alpha, k, t[2 * k], t[2 * k + 1]);
    CAHN_CUDA_TRY(cudaMemcpy(dev, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    return t;
}

// In-place Gauss-Jordan elimination with partial pivoting: inv = M^-1 (M is
// destroyed); false at a pivot below 1e-12 of the largest entry.
static bool gauss_jordan_inverse(std::vector<double>& M, int n, std::vector<double>& inv) {
    inv.assign((size_t)n * n, 0.0);
    double big = 0.0;
    for (int e = 0; e < n; ++e) inv[(size_t)e * n + e] = 1.0;
    for (double v : M) big = std::max(big, std::fabs(v));
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)p * n + c])) p = r;
        if (!(std::fabs(M[(size_t)p * n + c]) > 1e-12 * big)) return false;
        if (p != c)
            for (int k = 0; k < n; ++k) {
                std::swap(M[(size_t)p * n + k], M[(size_t)c * n + k]);
                std::swap(inv[(size_t)p * n + k], inv[(size_t)c * n + k]);
            }
        double* mc = &M[(size_t)c * n];
        double* ic = &inv[(size_t)c * n];
        const double d = 1.0 / mc[c];
        for (int k = c; k < n; ++k) mc[k] *= d;
        for (int k = 0; k < n; ++k) ic[k] *= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double* mr = &M[(size_t)r * n];
            const double f = mr[c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) mr[k] -= f * mc[k];
            double* ir = &inv[(size_t)r * n];
            for (int k = 0; k < n; ++k) ir[k] -= f * ic[k];
        }
    }
    return true;
}

// The dense solve of a 5-point level (op.kind OP_LAP5_NEUMANN or
// OP_LAP5_DIRICHLET, its own grid op.g): P (n x n, row-major) such that
// x = P b is the level's exact solution.  Rows held at zero (dz_row) are
// dropped from the system: their rows and columns of P are zero.  The
// zero-flux operator without a diagonal term (c0 = 0, nothing held) is
// singular, its null space the constants.  A is self-adjoint in the inner
// product weighted by W (1/2 on the wall rows, 1 inside; the rows there
// carry twice the coupling to their neighbour row), so b = A x is solvable
// exactly when sum_e W_e b_e = 0.  With s = sum_e W_e and sigma > 0,
// M = A + sigma 1 (W 1)^T / s is invertible, and for such b, M^-1 b is the
// solution with sum_e W_e x_e = 0; M^-1 1 = 1 / sigma.  So P = M^-1 -
// 1 (W 1)^T / (sigma s) is the W-pseudo-inverse: it maps the constants to
// zero.  Returns false if the elimination fails.
bool dense_solve_matrix(const Op& o, int dz, std::vector<double>& P) {
    const int nx = o.g.nx, ny = o.g.ny, n = nx * (ny + 1);
    const bool neumann = o.kind == OP_LAP5_NEUMANN;
    if (!neumann && o.kind != OP_LAP5_DIRICHLET) return false;
    std::vector<double> M((size_t)n * n, 0.0);
    auto held = [&](int j) { return dz_row(dz, j, ny); };
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int e = j * nx + i;
            double* row = &M[(size_t)e * n];
            if (held(j)) {   // decoupled; its row and column of P are cleared below
                row[e] = 1.0;
                continue;
            }
            if (!neumann && (j == 0 || j == ny)) {
                row[e] = o.c0;
                continue;
            }
            const int js = neumann ? (j > 0 ? j - 1 : 1) : j - 1;
            const int jn = neumann ? (j < ny ? j + 1 : ny - 1) : j + 1;
            const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
            row[e] += o.c0 + 2.0 * o.cx + 2.0 * o.cy;
            row[j * nx + im] -= o.cx;
            row[j * nx + ip] -= o.cx;
            if (!held(js)) row[js * nx + i] -= o.cy;
            if (!held(jn)) row[jn * nx + i] -= o.cy;
        }
    const bool singular = neumann && o.c0 == 0.0 && dz == 0;
    std::vector<double> w;
    double sw = 0.0, sigma = 0.0;
    if (singular) {
        w.resize(n);
        for (int e = 0; e < n; ++e) {
            const int j = e / nx;
            w[e] = (j == 0 || j == ny) ? 0.5 : 1.0;
            sw += w[e];
        }
        sigma = 2.0 * (o.cx + o.cy);
        for (int e = 0; e < n; ++e)
            for (int f = 0; f < n; ++f) M[(size_t)e * n + f] += sigma * w[f] / sw;
    }
    if (!gauss_jordan_inverse(M, n, P)) return false;
    if (singular)
        for (int e = 0; e < n; ++e)
            for (int f = 0; f < n; ++f) P[(size_t)e * n + f] -= w[f] / (sigma * sw);
    for (int e = 0; e < n; ++e)
        if (held(e / nx))
            for (int f = 0; f < n; ++f) P[(size_t)e * n + f] = P[(size_t)f * n + e] = 0.0;
    return true;
}

// dense_solve_matrix, computed once per distinct level in the process
static bool dense_solve_cached(const Op& o, int dz, std::vector<double>& P) {
    static std::mutex mu;
    static std::map<std::vector<double>, std::vector<double>> cache;
    const std::vector<double> key{(double)o.kind, (double)o.g.nx, (double)o.g.ny, (double)dz,
                                  o.c0, o.cx, o.cy};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            P = it->second;
            return true;
        }
    }
    if (!dense_solve_matrix(o, dz, P)) return false;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = P;
    return true;
}

template <typename T>
void Multigrid<T>::build(const Op& fine, int max_levels, size_t stop_nodes, RedWs r,
                         cudaStream_t s) {
    red = r;
    dirichlet = fine.kind == OP_LAP5_DIRICHLET;
    dz = dirichlet ? 1 : ((fine.kind == OP_NUT5 && fine.nut_dtop) ? 2 : 0);
    if constexpr (sizeof(T) == 4) {
        // CAHN_MG_DEGREE=2..8 in the environment: the FP32 smoother's degree
        const char* deg_env = std::getenv("CAHN_MG_DEGREE");
        if (deg_env && deg_env[0]) {
            const int d = std::atoi(deg_env);
            if (d >= 2 && d <= 8) degree = d;
        }
    }
    const bool coef_kind = fine.kind == OP_CH13 || fine.kind == OP_NUT5;
    Grid g = fine.g;
    for (int l = 0;; ++l) {
        MgLevel<T> L;
        L.g = g;
        L.op = fine;
        L.op.g = g;
        const double sx = (fine.g.hx * fine.g.hx) / (g.hx * g.hx);
        const double sy = (fine.g.hy * fine.g.hy) / (g.hy * g.hy);
        if (fine.kind == OP_CH13) {
            L.op.kx = fine.kx * sx;
            L.op.ky = fine.ky * sy;
            L.op.gx = fine.gx * sx;
            L.op.gy = fine.gy * sy;
        } else if (fine.kind == OP_NUT5) {
            L.op.gx = fine.gx * sx;
            L.op.gy = fine.gy * sy;
        } else {
            L.op.cx = fine.cx * sx;
            L.op.cy = fine.cy * sy;
        }
        const size_t n = g.n();
        if (l > 0) {
            L.x = mg_alloc<T>(allocs, n);
            L.b = mg_alloc<T>(allocs, n);
        }
        L.xt = mg_alloc<T>(allocs, n);
        L.r = mg_alloc<T>(allocs, n);
        L.d = mg_alloc<T>(allocs, n);
        L.dinv = mg_alloc<T>(allocs, n);
        L.lam = mg_alloc<double>(allocs, 1);
        L.coef = mg_alloc<double>(allocs, 2 * MG_KTAB);
        if (coef_kind) {
            if (l > 0) {
                L.a = mg_alloc<T>(allocs, n);
                CAHN_CUDA_TRY(cudaMemset(L.a, 0, n * sizeof(T)));
                if (fine.kind == OP_NUT5) {
                    L.dg = mg_alloc<T>(allocs, n);
                    CAHN_CUDA_TRY(cudaMemset(L.dg, 0, n * sizeof(T)));
                }
            }
        } else {
            // constant-coefficient operator: diagonal and exact spectral bound
            const Op& o = L.op;
            const double Dint = o.c0 + 2 * o.cx + 2 * o.cy;
            std::vector<T> h(n);
            for (int j = 0; j <= g.ny; ++j)
                for (int i = 0; i < g.nx; ++i)
                    h[(size_t)j * g.nx + i] =
                        (T)((dirichlet && (j == 0 || j == g.ny)) ? 1.0 / o.c0 : 1.0 / Dint);
            CAHN_CUDA_TRY(cudaMemcpy(L.dinv, h.data(), n * sizeof(T), cudaMemcpyHostToDevice));
            double lm = (o.c0 + 4 * o.cx + 4 * o.cy) / Dint * 1.01;
            CAHN_CUDA_TRY(cudaMemcpy(L.lam, &lm, sizeof(double), cudaMemcpyHostToDevice));
            L.coef_h = host_table(lm, alpha, MG_KTAB, L.coef);
        }
        // decide the next coarsening
        const bool can_y = g.ny % 2 == 0 && g.ny / 2 >= 2;
        const bool can_x = g.nx % 2 == 0 && g.nx / 2 >= 4;
        const bool last = (l + 1 >= max_levels) || !can_y || n <= stop_nodes;
        if (last) {
            lv.push_back(L);
            break;
        }
        L.semi = (g.hx > 1.41421356 * g.hy || !can_x) ? 1 : 0;
        lv.push_back(L);
        Grid c = g;
        c.ny = g.ny / 2;
        c.hy = 2 * g.hy;
        if (!L.semi) {
            c.nx = g.nx / 2;
            c.hx = 2 * g.hx;
        }
        g = c;
    }
    // coarsest-level solve: whole-spectrum Chebyshev
    const MgLevel<T>& C = lv.back();
    const Op& o = C.op;
    const double pi = 3.14159265358979323846;
    if (coef_kind) {
        coarse_alpha = 40.0;
    } else {
        const double Dint = o.c0 + 2 * o.cx + 2 * o.cy;
        const double lx1 = 4 * o.cx * std::pow(std::sin(pi / C.g.nx), 2);
        const double ly1 = 4 * o.cy * std::pow(std::sin(pi / (2.0 * C.g.ny)), 2);
        const double lmin = (o.c0 > 0) ? o.c0 + (dirichlet ? ly1 : 0.0)
                                       : std::min(lx1, ly1);   // singular: smallest nonzero mode
        const double lmax = (o.c0 + 4 * o.cx + 4 * o.cy) * 1.01;
        coarse_alpha = std::max(2.0, lmax / lmin);
        (void)Dint;
    }
    coarse_iters = (int)std::ceil(std::sqrt(coarse_alpha) * 4.0);
    if (coarse_iters < 4) coarse_iters = 4;
    if (coarse_iters > SB_MAX_ITERS) coarse_iters = SB_MAX_ITERS;
    lv.back().coarse_coef = mg_alloc<double>(allocs, 2 * SB_MAX_ITERS);
    if (!coef_kind) {
        const double Dint = o.c0 + 2 * o.cx + 2 * o.cy;
        lv.back().coarse_coef_h = host_table((o.c0 + 4 * o.cx + 4 * o.cy) / Dint * 1.01,
                                             coarse_alpha, SB_MAX_ITERS, lv.back().coarse_coef);
    }
    // (the single-block coarse solver evaluates the 5-point and 13-point
    // operators only; the nutrient's coarsest level takes the multi-launch path)
    single_block_coarse = C.g.n() <= 2048 && fine.kind != OP_NUT5;
    if (!single_block_coarse && coarse_iters > 6) coarse_iters = 6;
    if (coef_kind) {
        // the lam = 1 tables: smoother, coarsest level (a later, smaller
        // coarse_iters reads a prefix), Schwarz (see enable_schwarz)
        ntab = mg_alloc<double>(allocs, 2 * (MG_KTAB + SB_MAX_ITERS + MG_KTAB));
        host_table(1.0, alpha, MG_KTAB, ntab);
        host_table(1.0, coarse_alpha, coarse_iters, ntab + 2 * MG_KTAB);
    }
    // the dense coarsest solve (CAHN_MG_DENSE=0 in the environment keeps the
    // Chebyshev steps, to check one against the other)
    dense = nullptr;
    const char* dense_env = std::getenv("CAHN_MG_DENSE");
    if (!coef_kind && lv.size() >= 2 && C.g.n() <= (size_t)DENSE_MAX_NODES &&
        !(dense_env && dense_env[0] == '0')) {
        std::vector<double> pd;
        if (dense_solve_cached(C.op, dz, pd)) {
            const std::vector<T> ph(pd.begin(), pd.end());
            dense = mg_alloc<T>(allocs, ph.size());
            CAHN_CUDA_TRY(cudaMemcpy(dense, ph.data(), ph.size() * sizeof(T), cudaMemcpyHostToDevice));
        }
    }
    // tile heights
    for (size_t l = 0; l < lv.size(); ++l) {
        MgLevel<T>& L = lv[l];
        Op o = L.op;
        if (coef_kind && L.a) o.a = L.a;
        if (fine.kind == OP_NUT5 && L.dg) o.dg = L.dg;
        L.op.ty = tune_tile<T>(o, s);
    }
    // single-block tail: FP32 5-point hierarchies, from the first level (>= 1)
    // whose remaining levels (4 vectors each) fit in TAIL_SMEM_BYTES of
    // shared memory, when that covers at least two levels
    // (CAHN_MG_TAIL=0 in the environment keeps the multi-launch tail, to
    // check one against the other)
    constexpr size_t TAIL_SMEM_BYTES = 150 * 1024;
    // temporally blocked passes: FP32 5-point hierarchies (CAHN_MG_FUSED=0 in
    // the environment keeps the separate launches, to check one against the
    // other)
    const char* fused_env = std::getenv("CAHN_MG_FUSED");
    if constexpr (sizeof(T) == 4) {
        if (fine.kind != OP_NUT5 && degree >= FUSED_DEG_MIN && degree <= FUSED_DEG_MAX &&
            !(fused_env && fused_env[0] == '0')) {
            fused_prepare<T>(fine.kind, degree);
            fused = true;
        }
    }
    // the tail serves the separate launches; with the fused passes the
    // coarse levels are cheaper as fused launches (measured: 148.9 against
    // 145.0 steps/s on the 1024^2 workload).  CAHN_MG_TAIL=1 or 0 forces it
    // on or off.
    const char* tail_env = std::getenv("CAHN_MG_TAIL");
    const bool tail_on = tail_env && tail_env[0] ? tail_env[0] != '0' : !fused;
    if (tail_on && sizeof(T) == 4 && !coef_kind) {
        const int nl = (int)lv.size();
        size_t bytes = 0;
        int t = nl;
        for (int l = nl - 1; l >= 1 && nl - l <= TAIL_MAX; --l) {
            const size_t add = 4 * lv[l].g.n() * sizeof(T);
            if (bytes + add > TAIL_SMEM_BYTES) break;
            bytes += add;
            t = l;
        }
        if (nl - t >= 2) {
            tail = t;
            tail_smem = bytes;
            targs.count = nl - t;
            targs.degree = degree;
            targs.coarse_iters = coarse_iters;
            targs.dz = dirichlet ? 1 : 0;
            targs.dense = dense;
            int off = 0;
            for (int l = t; l < nl; ++l) {
                TailLevel& tl = targs.lv[l - t];
                tl.op = lv[l].op;
                tl.semi = lv[l].semi;
                tl.n = (int)lv[l].g.n();
                tl.off = off;
                tl.coef = (l + 1 == nl) ? lv[l].coarse_coef : lv[l].coef;
                // as the level's dinv array: 1 / D in FP64, rounded to T in the kernel
                const Op& o = lv[l].op;
                tl.di_int = 1.0 / (o.c0 + 2 * o.cx + 2 * o.cy);
                tl.di_wall = o.c0 != 0.0 ? 1.0 / o.c0 : 0.0;
                off += 4 * tl.n;
            }
            // the limit is per kernel, shared by every hierarchy of the
            // process: set it to the largest tail any hierarchy may launch
            auto k = dirichlet ? k_tail_vcycle<T, OP_LAP5_DIRICHLET> : k_tail_vcycle<T, OP_LAP5_NEUMANN>;
            CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)TAIL_SMEM_BYTES));
        }
    }
}

template <typename T>
FusedPass<T> Multigrid<T>::fused_pass(int l, bool coarse, int steps, int halo, const T* b,
                                      T* xout) const {
    const MgLevel<T>& L = lv[l];
    if (steps > FUSED_MAXK) throw ArgError("fused multigrid pass: too many steps");
    FusedPass<T> fp{};
    fp.op = L.op;
    fp.ca = cheb_args(l, coarse ? L.coarse_coef : L.coef);
    // constants rounded to T on the host, as the separate launches round
    // them on the device
    if (L.op.kind == OP_CH13) {
        // the step table is refreshed on the device every time step: the
        // kernel reads it from ca.coef
        fp.k13 = C13<T>{(T)L.op.kx, (T)L.op.ky, (T)L.op.S, (T)(0.25 * L.op.gx),
                        (T)(0.25 * L.op.gy), (T)L.op.idt};
    } else {
        const std::vector<double>& tab = coarse ? L.coarse_coef_h : L.coef_h;
        if ((int)tab.size() < 2 * steps) throw ArgError("fused multigrid pass: no host step table");
        fp.kc = lap5_consts<T>(L.op);
        for (int k = 0; k < steps; ++k) {
            fp.c1[k] = (T)tab[2 * k];
            fp.c2[k] = (T)tab[2 * k + 1];
        }
    }
    fp.steps = steps;
    fp.halo = halo;
    fp.b = b;
    fp.xout = xout;
    return fp;
}

template <typename T>
void Multigrid<T>::set_coefficient(const T* a_fine, cudaStream_t s, const int* gate) {
    // one launch per level: its D^-1, spectral bound and step tables, and
    // the coefficient restricted to the next level
    lv[0].a = const_cast<T*>(a_fine);
    for (size_t l = 0; l < lv.size(); ++l) {
        MgLevel<T>& L = lv[l];
        L.op.a = L.a;
        const bool last = l + 1 == lv.size();
        ChebTabs tabs;
        tabs.add(ntab, MG_KTAB, L.coef);
        if (schwarz && l == 0) tabs.add(ntab + 2 * (MG_KTAB + SB_MAX_ITERS), MG_KTAB, sw_coef);
        if (last) tabs.add(ntab + 2 * MG_KTAB, coarse_iters, L.coarse_coef);
        launch_ch13_level<T>(L.op, L.dinv, L.lam, red, last ? Grid{} : lv[l + 1].g, L.semi,
                             last ? nullptr : lv[l + 1].a, tabs, gate, s);
    }
}

template <typename T>
void Multigrid<T>::set_coefficients(const T* a_fine, const T* dg_fine, cudaStream_t s) {
    // one launch per level, as set_coefficient
    lv[0].a = const_cast<T*>(a_fine);
    lv[0].dg = const_cast<T*>(dg_fine);
    for (size_t l = 0; l < lv.size(); ++l) {
        MgLevel<T>& L = lv[l];
        L.op.a = L.a;
        L.op.dg = L.dg;
        const bool last = l + 1 == lv.size();
        ChebTabs tabs;
        tabs.add(ntab, MG_KTAB, L.coef);
        if (schwarz && l == 0) tabs.add(ntab + 2 * (MG_KTAB + SB_MAX_ITERS), MG_KTAB, sw_coef);
        if (last) tabs.add(ntab + 2 * MG_KTAB, coarse_iters, L.coarse_coef);
        launch_nut_level<T>(L.op, L.dinv, L.lam, red, last ? Grid{} : lv[l + 1].g, L.semi,
                            last ? nullptr : lv[l + 1].a, last ? nullptr : lv[l + 1].dg, tabs, s);
    }
}

template <typename T>
ChebArgs<T> Multigrid<T>::cheb_args(int l, const double* coef) const {
    const MgLevel<T>& L = lv[l];
    ChebArgs<T> ca;
    ca.dinv = L.dinv;
    ca.d = L.d;
    ca.coef = coef;
    ca.dirichlet_zero = dz;
    if (L.op.kind == OP_LAP5_NEUMANN || L.op.kind == OP_LAP5_DIRICHLET) {
        // the values of L.dinv (1 / D in FP64, rounded to T), formed in the kernels
        const Op& o = L.op;
        ca.const_dinv = 1;
        ca.di_int = (T)(1.0 / (o.c0 + 2 * o.cx + 2 * o.cy));
        ca.di_wall = o.c0 != 0.0 ? (T)(1.0 / o.c0) : (T)0;
    }
    return ca;
}

template <typename T>
void Multigrid<T>::fine_step(const T* x, const T* b, T* d, T* y, int k, cudaStream_t s) {
    ChebArgs<T> ca = cheb_args(0, lv[0].coef);
    ca.d = d;
    ca.k = k;
    launch_cheb<T>(lv[0].op, x, b, y, ca, nullptr, s);
}

template <typename T>
void Multigrid<T>::smooth(int l, const T* b, T* x, bool zero_init, const int* gate,
                          cudaStream_t s, int deg, const double* coef, const T* xc) {
    MgLevel<T>& L = lv[l];
    ChebArgs<T> ca = cheb_args(l, coef);
    // step k writes to x when (deg - 1 - k) is even, so the last step lands in x
    auto out_of = [&](int k) { return ((deg - 1 - k) % 2 == 0) ? x : L.xt; };
    int k0 = 0;
    // Fused first steps for the FP32 hierarchies (latency-bound); the FP64
    // kernels are FP64-ALU-bound, where recomputing x in every load costs
    // more than the launch it saves.
    constexpr bool fuse = sizeof(T) == 4;
    if (fuse && zero_init && deg >= 2) {
        // steps 0 and 1 in one launch: step 0 (x = c dinv b) is formed in the loads
        ca.k = 1;
        launch_cheb<T>(L.op, b, b, out_of(1), ca, gate, s, XL_ZERO);
        k0 = 2;
    } else if (zero_init) {
        T* o = out_of(0);
        note_launch(); launch_k(k_cheb_zero<T>, vec_blocks(L.g.n()), RED_THREADS, 0, s, L.g.n(), b, L.dinv, L.d, o, coef, gate);
        k0 = 1;
    } else if (fuse && xc) {
        // step 0 on x + P xc: the coarse-grid correction is added in the loads
        ca.xc = xc;
        ca.gc = lv[l + 1].g;
        ca.semi = L.semi;
        ca.k = 0;
        if (out_of(0) != x) {
            launch_cheb<T>(L.op, x, b, out_of(0), ca, gate, s, XL_PROLONG);
            k0 = 1;
        } else {
            // odd degree: step 0 cannot write x in place; it writes the
            // level's residual buffer (free on the way up), step 1 reads it
            launch_cheb<T>(L.op, x, b, L.r, ca, gate, s, XL_PROLONG);
            if (deg == 1) {
                launch_copy<T>(L.r, x, L.g.n(), s, gate);
                return;
            }
            ca.k = 1;
            launch_cheb<T>(L.op, L.r, b, out_of(1), ca, gate, s);
            k0 = 2;
        }
    } else {
        if (xc) {
            const MgLevel<T>& C = lv[l + 1];
            note_launch(); launch_k(k_prolong_add<T>, vec_blocks(L.g.n()), RED_THREADS, 0, s, L.g, C.g, L.semi, ca.dirichlet_zero, xc, x, gate);
        }
        if (out_of(0) == x) launch_copy<T>(x, L.xt, L.g.n(), s, gate);   // odd degree: read from the copy
    }
    for (int k = k0; k < deg; ++k) {
        T* o = out_of(k);
        const T* in = (o == x) ? L.xt : x;
        ca.k = k;
        launch_cheb<T>(L.op, in, b, o, ca, gate, s);
    }
}

template <typename T>
int Multigrid<T>::coop_capacity() {
    if constexpr (sizeof(T) != 4) {
        return 0;
    } else {
        // opt-in (CAHN_MG_COOP=1): measured on the 1024^2 workload, the grid
        // barrier between passes costs more than the kernel boundary of a
        // graph, at every starting level tried
        const char* env = std::getenv("CAHN_MG_COOP");
        if (!env || env[0] != '1') return 0;
        int dev = 0, sms = 0, per_d = 0, per_n = 0, coop_ok = 0;
        CAHN_CUDA_TRY(cudaGetDevice(&dev));
        CAHN_CUDA_TRY(cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, dev));
        CAHN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        CAHN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_d, k_vcycle_coop<T, OP_LAP5_DIRICHLET>, COOP_THREADS, 0));
        CAHN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_n, k_vcycle_coop<T, OP_LAP5_NEUMANN>, COOP_THREADS, 0));
        return coop_ok ? sms * std::min(per_d, per_n) : 0;
    }
}

template <typename T>
size_t Multigrid<T>::coop_nodes() {
    const char* env = std::getenv("CAHN_COOP_NODES");
    if (env && env[0]) return (size_t)std::strtoull(env, nullptr, 10);
    return COOP_NODES;
}

template <typename T>
void Multigrid<T>::enable_coop(int blocks) {
    if constexpr (sizeof(T) != 4) {
        return;
    } else {
        const Op& f = lv[0].op;
        if (blocks < 1 || schwarz) return;
        if (f.kind != OP_LAP5_NEUMANN && f.kind != OP_LAP5_DIRICHLET) return;
        const int nall = (int)lv.size();
        const size_t cap_nodes = coop_nodes();
        int from = 0;
        while (from < nall && lv[from].g.n() > cap_nodes) ++from;
        const int nl = nall - from;
        if (nl > COOP_MAX || nl < 2) return;
        // about COOP_NODES_PER_THREAD nodes per thread on the first level:
        // fewer blocks make a cheaper grid barrier
        const size_t per_block = (size_t)COOP_THREADS * COOP_NODES_PER_THREAD;
        const size_t need = (lv[from].g.n() + per_block - 1) / per_block;
        coop_blocks = (int)std::max<size_t>(1, std::min<size_t>((size_t)blocks, need));
        coop_from = from;
        cargs.count = nl;
        cargs.degree = degree;
        cargs.coarse_iters = coarse_iters;
        cargs.dz = dz;
        cargs.single_coarse = single_block_coarse ? 1 : 0;
        cargs.dense = dense;
        for (int k = 0; k < nl; ++k) {
            const MgLevel<T>& L = lv[from + k];
            CoopLevel& c = cargs.lv[k];
            c.op = L.op;
            c.semi = L.semi;
            c.x = L.x;
            c.xt = L.xt;
            c.b = L.b;
            c.d = L.d;
            c.r = L.r;
            c.dinv = L.dinv;
            c.coef = (k + 1 == nl) ? L.coarse_coef : L.coef;
        }
        cargs.bar = mg_alloc<unsigned>(allocs, 2);
        cargs.err = mg_alloc<int>(allocs, 1);
        CAHN_CUDA_TRY(cudaMemset(cargs.bar, 0, 2 * sizeof(unsigned)));
        CAHN_CUDA_TRY(cudaMemset(cargs.err, 0, sizeof(int)));
        coop = true;
    }
}

template <typename T>
void Multigrid<T>::enable_schwarz() {
    schwarz = true;
    sw_coef = mg_alloc<double>(allocs, 2 * MG_KTAB);
    const Op& o = lv[0].op;
    if (o.kind == OP_LAP5_NEUMANN || o.kind == OP_LAP5_DIRICHLET) {
        const double Dint = o.c0 + 2 * o.cx + 2 * o.cy;
        host_table((o.c0 + 4 * o.cx + 4 * o.cy) / Dint * 1.01, SW_ALPHA, MG_KTAB, sw_coef);
    } else if (ntab) {
        // coefficient kinds: refreshed with lam by set_coefficient(s)
        host_table(1.0, SW_ALPHA, MG_KTAB, ntab + 2 * (MG_KTAB + SB_MAX_ITERS));
    }
}

template <typename T>
void Multigrid<T>::vcycle(const T* r0, T* z0, const int* gate, cudaStream_t s) {
    const int nl = (int)lv.size();
    if (schwarz) {
        launch_schwarz<T>(lv[0].op, r0, z0, lv[0].dinv, sw_coef, dz, gate, s);
        return;
    }
    auto bptr = [&](int l) -> const T* { return l == 0 ? r0 : lv[l].b; };
    auto xptr = [&](int l) -> T* { return l == 0 ? z0 : lv[l].x; };
    // levels coop_from .. nl-1 in one cooperative launch
    auto launch_coop = [&]() {
      if constexpr (sizeof(T) == 4) {
        auto k = dirichlet ? k_vcycle_coop<T, OP_LAP5_DIRICHLET> : k_vcycle_coop<T, OP_LAP5_NEUMANN>;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)coop_blocks);
        cfg.blockDim = dim3(COOP_THREADS);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        note_launch();
        CAHN_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, cargs, bptr(coop_from), xptr(coop_from), gate));
      }
    };
    if (coop && coop_from == 0) {
        launch_coop();
        return;
    }
    // the level the down pass stops at
    const int last = coop ? coop_from : (tail >= 0 ? tail : nl - 1);
    if constexpr (sizeof(T) == 4) if (fused && !coop) {
        // one launch per level and direction; the down pass keeps its x in
        // the level's xt until the up pass (which reads it around its tile)
        for (int l = 0; l < last; ++l) {
            FusedPass<T> fp = fused_pass(l, false, degree, degree + 1, bptr(l), lv[l].xt);
            fp.bc = lv[l + 1].b;
            fp.gc = lv[l + 1].g;
            fp.semi = lv[l].semi;
            launch_fused<T>(FUSED_DOWN, fp, gate, s);
        }
        const int c = nl - 1;
        if (tail >= 0) {
            auto k = dirichlet ? k_tail_vcycle<T, OP_LAP5_DIRICHLET> : k_tail_vcycle<T, OP_LAP5_NEUMANN>;
            note_launch(); launch_k(k, 1, 1024, tail_smem, s, targs, (const T*)lv[tail].b, lv[tail].x, gate);
        } else if (!single_block_coarse && fused_coarse_steps(lv[c].op.kind, coarse_iters)) {
            FusedPass<T> fp = fused_pass(c, true, coarse_iters, 0, bptr(c), xptr(c));
            launch_fused<T>(FUSED_COARSE, fp, gate, s);
        } else {
            coarse_solve(bptr(c), xptr(c), gate, s);
        }
        for (int l = last - 1; l >= 0; --l) {
            FusedPass<T> fp = fused_pass(l, false, degree, degree, bptr(l), xptr(l));
            fp.xin = lv[l].xt;
            fp.ca.xc = lv[l + 1].x;
            fp.ca.gc = lv[l + 1].g;
            fp.ca.semi = lv[l].semi;
            launch_fused<T>(FUSED_UP, fp, gate, s);
        }
        return;
    }
    for (int l = 0; l < last; ++l) {
        smooth(l, bptr(l), xptr(l), true, gate, s, degree, lv[l].coef);
        restrict_residual(l, xptr(l), bptr(l), gate, s);
    }
    if (coop) {
        launch_coop();
    } else if (tail >= 0) {
        // levels tail .. nl-1 in one block
        auto k = dirichlet ? k_tail_vcycle<T, OP_LAP5_DIRICHLET> : k_tail_vcycle<T, OP_LAP5_NEUMANN>;
        note_launch(); launch_k(k, 1, 1024, tail_smem, s, targs, (const T*)lv[tail].b, lv[tail].x, gate);
    } else {
        coarse_solve(bptr(nl - 1), xptr(nl - 1), gate, s);
    }
    for (int l = last - 1; l >= 0; --l) {
        MgLevel<T>& L = lv[l];
        const MgLevel<T>& C = lv[l + 1];
        smooth(l, bptr(l), xptr(l), false, gate, s, degree, L.coef, C.x);
    }
}

template <typename T>
void Multigrid<T>::coarse_solve(const T* b, T* x, const int* gate, cudaStream_t s) {
    {
        MgLevel<T>& C = lv.back();
        if (dense) {
            // one warp per row, eight rows per block
            const int n = (int)C.g.n();
            note_launch(); launch_k(k_coarse_dense<T>, (n + 7) / 8, 256, 0, s, (const T*)dense, b, x, n, gate);
        } else if (single_block_coarse) {
            const bool sm = C.g.n() <= (size_t)SB_SMEM_NODES;
            // one node per thread where the level allows (a 32x9 coarsest level
            // takes 288 threads): the barrier of every step waits for no idle
            // warps; each node's arithmetic does not depend on the block size
            const int nthr = (int)std::min<size_t>(1024, (C.g.n() + 31) / 32 * 32);
#define CAHN_COARSE(KIND, SM) \
    launch_k(k_coarse_solve<T, KIND, SM>, 1, nthr, 0, s, C.op, b, C.dinv, x, C.xt, C.d, C.coarse_coef, coarse_iters, dz, gate)
            note_launch();
            switch (C.op.kind) {
                case OP_LAP5_NEUMANN:
                    if (sm) CAHN_COARSE(OP_LAP5_NEUMANN, true); else CAHN_COARSE(OP_LAP5_NEUMANN, false);
                    break;
                case OP_LAP5_DIRICHLET:
                    if (sm) CAHN_COARSE(OP_LAP5_DIRICHLET, true); else CAHN_COARSE(OP_LAP5_DIRICHLET, false);
                    break;
                default:
                    CAHN_COARSE(OP_CH13, false);
                    break;
            }
#undef CAHN_COARSE
        } else {
            smooth((int)lv.size() - 1, b, x, true, gate, s, coarse_iters, C.coarse_coef);
        }
    }
}

template <typename T>
void Multigrid<T>::restrict_residual(int l, const T* x, const T* b, const int* gate,
                                     cudaStream_t s) {
    MgLevel<T>& L = lv[l];
    const MgLevel<T>& C = lv[l + 1];
    if (sizeof(T) == 4 && L.op.kind == OP_LAP5_NEUMANN) {
        note_launch(); launch_k(k_resid_restrict<T, OP_LAP5_NEUMANN>, vec_blocks(C.g.n()), RED_THREADS, 0, s, L.op, C.g, L.semi, dz, x, b, C.b, gate);
    } else if (sizeof(T) == 4 && L.op.kind == OP_LAP5_DIRICHLET) {
        note_launch(); launch_k(k_resid_restrict<T, OP_LAP5_DIRICHLET>, vec_blocks(C.g.n()), RED_THREADS, 0, s, L.op, C.g, L.semi, dz, x, b, C.b, gate);
    } else {
        launch_op<T>(L.op, EPI_RPLAIN, x, b, L.r, SolveDev{}, gate, 0.0, s);
        note_launch(); launch_k(k_restrict<T>, vec_blocks(C.g.n()), RED_THREADS, 0, s, L.g, C.g, L.semi, dz, L.r, C.b, gate);
    }
}

template <typename T>
void Multigrid<T>::down_pass(const T* b, T* x, cudaStream_t s) {
    if (lv.size() < 2) throw ArgError("down_pass: one-level hierarchy");
    if constexpr (sizeof(T) == 4) {
        if (fused) {
            FusedPass<T> fp = fused_pass(0, false, degree, degree + 1, b, x);
            fp.bc = lv[1].b;
            fp.gc = lv[1].g;
            fp.semi = lv[0].semi;
            launch_fused<T>(FUSED_DOWN, fp, nullptr, s);
            return;
        }
    }
    smooth(0, b, x, true, nullptr, s, degree, lv[0].coef);
    restrict_residual(0, x, b, nullptr, s);
}

template <typename T>
void Multigrid<T>::release() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    lv.clear();
    dense = nullptr;
    ntab = nullptr;
}

template struct Multigrid<double>;
template struct Multigrid<float>;

}  // namespace cahn
