// Device helpers shared by the stencil kernels (stencil.cu: the general
// tiles; stencil_vec.cu: the vectorised fine-grid tiles): the fused
// epilogues at one node, the W-weighted reductions that finish them, and
// how a kernel forms its input x at a node (XLoad).  Both kernel families
// evaluate a node through these functions, so they round it alike.
#pragma once
#include "internal.h"

namespace cahn {

template <typename T>
struct EpiAcc {
    WSum<T> s0, s1, s2;
};

// Epilogue at one node: returns the stored value and accumulates.  ax is
// A x at the node in the kernel's precision T.
template <typename T, int EPI>
__device__ __forceinline__ T epi_node(T ax, T xc, const T* __restrict__ b, size_t e,
                                      T w, EpiAcc<T>& acc, const ChebArgs<T>& ca, T c1,
                                      T c2, T di) {
    if (EPI == EPI_RPLAIN) {
        return b[e] - ax;
    } else if (EPI == EPI_CHEB_Z) {
        const T r = b[e] - ax;
        const T dn = fma(mul_rn(c2, di), r, mul_rn(c1, xc));
        ca.d[e] = dn;
        return xc + dn;
    } else if (EPI == EPI_CHEB) {
        const T r = b[e] - ax;
        const T dn = fma(mul_rn(c2, di), r, c1 != (T)0 ? mul_rn(c1, ca.d[e]) : (T)0);
        ca.d[e] = dn;
        return xc + dn;
    } else if (EPI == EPI_RESID || EPI == EPI_RESIDX) {
        const T bv = b[e];
        const T r = bv - ax;
        acc.s0.add(w, bv, bv);
        acc.s1.add(w, r, r);
        if (EPI == EPI_RESIDX) acc.s2.add(w, xc, xc);
        return r;
    } else if (EPI == EPI_DOTXY) {
        acc.s0.add(w, xc, ax);
        return ax;
    } else if (EPI == EPI_CGCG) {
        acc.s0.add(w, b[e], xc);
        acc.s1.add(w, xc, ax);
        return ax;
    } else if (EPI == EPI_NORM) {
        acc.s0.add(w, ax, ax);
        return ax;
    }
    return ax;
}

// The refinement's test after the FP64 residual (run by one thread: the
// last block of the residual launch, EPI_RESIDX): stop at the rounding floor
// 16 eps64 (||A|| ||x||_W + ||b||_W), on three stalled sweeps or at maxit;
// else count the sweep.
__device__ __forceinline__ void ir_check_dev(SolveDev sd, double anorm) {
    Ctl* c = sd.ctl;
    if (c->done) return;
    double* sc = sd.scal;
    const double res = sc[S_RES0], bn = sc[S_BN];
    const double eps64 = 1.1102230246251565e-16;
    const double floor_ = 16.0 * eps64 * (anorm * sqrt(sc[S_TMP2]) + bn);
    if (res <= floor_) {
        c->done = 1;
        return;
    }
    if (c->it > 0 && res > 0.9 * sc[S_IRLAST]) {
        if (++c->cycles >= 3) {
            c->done = 1;
            c->status |= CTL_NOT_CONVERGED;
            return;
        }
    } else {
        c->cycles = 0;
    }
    if (c->it >= c->maxit) {
        c->done = 1;
        c->status |= CTL_NOT_CONVERGED;
        return;
    }
    sc[S_IRLAST] = res;
    c->it += 1;
    c->total += 1;
}

template <typename T, int EPI>
__device__ __forceinline__ void epi_finish(const EpiAcc<T>& acc, SolveDev sd, double rtol) {
    if (EPI == EPI_APPLY || EPI == EPI_RPLAIN || EPI == EPI_CHEB || EPI == EPI_CHEB_Z) return;
    __shared__ double sh[32];
    publish_wsum<T>(sd.red, 0, acc.s0, sh);
    constexpr bool RES = EPI == EPI_RESID || EPI == EPI_RESIDX;
    if (RES || EPI == EPI_CGCG) publish_wsum<T>(sd.red, 1, acc.s1, sh);
    if (EPI == EPI_RESIDX) publish_wsum<T>(sd.red, 2, acc.s2, sh);
    if (!last_block(sd.red)) return;
    double t0 = final_wsum<T>(sd.red, 0, sh);
    double t1 = (RES || EPI == EPI_CGCG) ? final_wsum<T>(sd.red, 1, sh) : 0.0;
    double t2 = (EPI == EPI_RESIDX) ? final_wsum<T>(sd.red, 2, sh) : 0.0;
    if (flat_tid() == 0) {
        double* sc = sd.scal;
        if (EPI == EPI_RESIDX) sc[S_TMP2] = t2;
        if (RES) {
            sc[S_BN] = sqrt(t0);
            sc[S_RR] = t1;
            sc[S_RES0] = sqrt(t1);
            sc[S_TOL2] = rtol * rtol * t0;
            if (!isfinite(t1) || !isfinite(t0)) {
                sd.ctl->status |= CTL_NAN;
                sd.ctl->done = 1;
            } else if (t1 <= rtol * rtol * t0 || t0 == 0.0) {
                sd.ctl->done = 1;
            }
            if (EPI == EPI_RESIDX) ir_check_dev(sd, sd.anorm);   // the refinement's sweep test
        } else if (EPI == EPI_DOTXY) {
            sc[S_PQ] = t0;
            if (!isfinite(t0)) {
                sd.ctl->status |= CTL_NAN;
                sd.ctl->done = 1;
                sc[S_ALPHA] = 0.0;
            } else {
                sc[S_ALPHA] = (t0 != 0.0) ? sc[S_RZ] / t0 : 0.0;
            }
        } else if (EPI == EPI_NORM) {
            sc[S_TMP0] = t0;
        } else if (EPI == EPI_CGCG) {
            // Chronopoulos-Gear: gamma = <r,z>, delta = <z,Az>; beta = gamma /
            // gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
            // (beta = 0, alpha = gamma / delta in the first iteration)
            const double gam = t0, del = t1;
            const bool first = sd.ctl->it == 0;
            double beta = 0.0, den = del;
            if (!first) {
                beta = sc[S_RZ] != 0.0 ? gam / sc[S_RZ] : 0.0;
                den = sc[S_ALPHA] != 0.0 ? del - beta * gam / sc[S_ALPHA] : del;
            }
            if (!isfinite(gam) || !isfinite(del)) {
                sd.ctl->status |= CTL_NAN;
                sd.ctl->done = 1;
                sc[S_ALPHA] = 0.0;
                sc[S_BETA] = 0.0;
            } else {
                sc[S_BETA] = beta;
                sc[S_ALPHA] = den != 0.0 ? gam / den : 0.0;
            }
            sc[S_RZ] = gam;
            sc[S_PQ] = del;
        }
        reset_counter(sd.red);
    }
}

template <typename T>
__device__ __forceinline__ void cheb_consts(const ChebArgs<T>& ca, T& c1, T& c2) {
    c1 = (T)ca.coef[2 * ca.k];
    c2 = (T)ca.coef[2 * ca.k + 1];
}

// Coarse-grid correction (P x_c)(i, j) at a fine node: bilinear, wall rows
// untouched on Dirichlet levels.  Every weight is 1 or 1/2, so the products
// are exact and the value does not depend on FMA contraction.
template <typename T>
__device__ __forceinline__ T prolong_at(const ChebArgs<T>& ca, int ny, int i, int j) {
    if (dz_row(ca.dirichlet_zero, j, ny)) return (T)0;
    const int ncx = ca.gc.nx;
    const int J0 = j >> 1, J1 = (j & 1) ? J0 + 1 : J0;
    auto rowv = [&](int J) {
        const T* row = ca.xc + (size_t)J * ncx;
        if (ca.semi) return row[i];
        const int I0 = i >> 1;
        if (!(i & 1)) return row[I0];
        const int I1 = I0 + 1 < ncx ? I0 + 1 : 0;
        return (T)0.5 * (row[I0] + row[I1]);
    };
    return (j & 1) ? (T)0.5 * (rowv(J0) + rowv(J1)) : rowv(J0);
}

// The restriction R = W_c^-1 P^T W_f / 4 (/ 2 with semicoarsening) at coarse
// row J: the bilinear weights 1 and 1/2, the half weight of the fine wall
// rows, then the coarse wall weight and the ratio.  res(j, dx) is the fine
// value at row j and column c + dx, c the coarse node's fine column (2I, or
// I with semicoarsening), the column wrapped periodically.  Every weight is
// a power of two, so each product is exact; the sum is taken in T with
// explicit fma, and every kernel that restricts rounds it alike.  (FP32
// levels sum in FP32: GB300's FP64 pipe issues 2 operations per clock and SM,
// and an FP64 sum here bounded the fused multigrid passes.)
template <typename T, typename F>
__device__ __forceinline__ T restrict_at(const F& res, int J, int nyf, int semi, int nyc) {
    T sum = (T)0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int j = 2 * J + dy;
        if (j < 0 || j > nyf) continue;
        const T wy = (dy == 0 ? (T)1 : (T)0.5) * ((j == 0 || j == nyf) ? (T)0.5 : (T)1);
        const T t = semi ? res(j, 0) : fma((T)0.5, res(j, -1) + res(j, 1), res(j, 0));
        sum = fma(wy, t, sum);
    }
    // the ratio 1/2 (1/4) over the coarse weight 1/2 on wall rows: a power of two
    return sum * ((semi ? (T)0.5 : (T)0.25) * ((J == 0 || J == nyc) ? (T)2 : (T)1));
}

// D^-1 at node (j, e) of an operator of kind KIND (formed for 5-point levels)
template <typename T, int KIND>
__device__ __forceinline__ T dinv_at(const ChebArgs<T>& ca, int ny, int j, size_t e) {
    if (KIND != OP_CH13 && ca.const_dinv)
        return (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) ? ca.di_wall : ca.di_int;
    return ca.dinv[e];
}

// Input x of a stencil kernel at node (i, j), flat index e (see XLoad).
template <typename T, int XL, int KIND>
__device__ __forceinline__ T load_x(const T* __restrict__ x, const T* __restrict__ b,
                                    const ChebArgs<T>& ca, T cz, int ny, int i, int j,
                                    size_t e) {
    if (XL == XL_ZERO) return mul_rn(mul_rn(cz, dinv_at<T, KIND>(ca, ny, j, e)), b[e]);
    if (XL == XL_PROLONG) return x[e] + prolong_at(ca, ny, i, j);
    return x[e];
}

// The tables of tabs for the bound lam (see ChebTabs), by the threads of one
// block.
__device__ inline void cheb_tables_dev(const ChebTabs& tabs, double lam, int t, int nt) {
    for (int q = 0; q < tabs.n; ++q)
        for (int k = t; k < tabs.count[q]; k += nt) {
            tabs.coef[q][2 * k] = tabs.norm[q][2 * k];
            tabs.coef[q][2 * k + 1] = tabs.norm[q][2 * k + 1] / lam;
        }
}

}  // namespace cahn
