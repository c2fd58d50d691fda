// Matrix-free stencil operators of the four per-step systems, FP64 and FP32.
//
//   OP_LAP5_NEUMANN    c0 x + cx(2x - x_w - x_e) + cy(2x - x_s - x_n), ghost
//                      rows by even reflection (zero normal derivative,
//                      Eq. 4.6-4.7): the pressure operator L_h of Eq. 4.4,
//                      whose interior row is Listing 3's (4,-1,-1,-1,-1).
//   OP_LAP5_DIRICHLET  the velocity predictor H of Eq. 4.3: the same row on
//                      interior rows with the stored wall values as
//                      neighbours, c0 x on the wall rows.
//   OP_CH13            idt x + 1/2 G_a (kappa L_h + S) x, the Crank-Nicolson
//                      matrix of Eq. 2.4 with the degenerate mobility a: a
//                      13-point, two-deep stencil (Eq. 4.7).
//   OP_CH13_WADJ       idt x + 1/2 (kappa L_h + S) G_a x, the same factors in
//                      the other order.  L_h and G_a are self-adjoint in the
//                      W inner product, so this is W^-1 A_phi^T W: the
//                      transposed phase-field solve of the discrete adjoint
//                      (FP64 only).
//   OP_NUT5            the nutrient matrix of Eq. 2.6 (Crank-Nicolson):
//                      dg x + 1/2 G_k x with face coefficients k_f = (k_c +
//                      k_n)/2, stored as a = k/4 so that the face weight is
//                      a_c + a_n; zero flux on both walls, or a Dirichlet
//                      row ny (op.nut_dtop).
//
// Each block computes a 32-column output tile of TY = 8, 16 or 32 rows with
// 32 x 8 threads (TY / 8 consecutive rows per thread); the tile height of
// the launches without reductions is picked per operator by the autotuner
// at the end of this file.  OP_CH13 stages x (halo 2) and a (halo 1) in
// shared memory and forms psi = kappa L_h x + S x once per node of the tile
// plus a one-node ring, then applies G_a to psi; each thread keeps its
// column of psi and a in registers.  FP64 arithmetic, not HBM, bounds the
// FP64 kernels, so no intermediate is computed twice.
//
// Fused epilogues: W-weighted reductions (trapezoid weights, 1/2 on the
// wall rows) finished by the last block, which also derives the Krylov
// scalars the next kernel needs; the multigrid residual; the Chebyshev
// smoother step.  The smoother's first steps fuse the step before them into
// the loads of x (XLoad): the zero-guess step c D^-1 b, or the prolonged
// coarse-grid correction.  Every multiply-add is an explicit fma or a
// separately rounded product, so all instantiations round a node alike.
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "stencil_dev.cuh"
#include "visc.h"

namespace cahn {

// -------------------------------------------------------------- 5-point
template <typename T, int KIND, int EPI, int TY, int XL>
__global__ void __launch_bounds__(256) k_lap5(Op op, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ y,
                                              SolveDev sd, const int* __restrict__ gate,
                                              double rtol, ChebArgs<T> ca) {
    if (gate && *gate) return;
    T c1 = 0, c2 = 0, cz = 0;
    if (EPI == EPI_CHEB || EPI == EPI_CHEB_Z) cheb_consts(ca, c1, c2);
    if (XL == XL_ZERO) cz = (T)ca.coef[1];
    const int nx = op.g.nx, ny = op.g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    const Lap5C<T> kc = lap5_consts<T>(op);
    const T c0 = kc.c0;
    EpiAcc<T> acc;
    if (i < nx) {
        const int im = i > 0 ? i - 1 : nx - 1;
        const int ip = i < nx - 1 ? i + 1 : 0;
#pragma unroll
        for (int r = 0; r < TY / 8; ++r) {
            const int j = blockIdx.y * TY + threadIdx.y + 8 * r;
            if (j > ny) continue;   // predicated (no break), so loads can be hoisted
            const size_t e = (size_t)j * nx + i;
            const T xc = load_x<T, XL, KIND>(x, b, ca, cz, ny, i, j, e);
            T ax;
            if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) {
                ax = mul_rn(c0, xc);
                if ((EPI == EPI_CHEB || EPI == EPI_CHEB_Z) && ca.dirichlet_zero) {
                    y[e] = (T)0;
                    continue;
                }
            } else {
                int js, jn;
                if (KIND == OP_LAP5_NEUMANN) {
                    js = j > 0 ? j - 1 : 1;
                    jn = j < ny ? j + 1 : ny - 1;
                } else {
                    js = j - 1;
                    jn = j + 1;
                }
                const size_t row = (size_t)j * nx;
                const T xw = load_x<T, XL, KIND>(x, b, ca, cz, ny, im, j, row + im);
                const T xe = load_x<T, XL, KIND>(x, b, ca, cz, ny, ip, j, row + ip);
                const T xs = load_x<T, XL, KIND>(x, b, ca, cz, ny, i, js, (size_t)js * nx + i);
                const T xn = load_x<T, XL, KIND>(x, b, ca, cz, ny, i, jn, (size_t)jn * nx + i);
                ax = lap5_ax(kc, xc, xw, xe, xs, xn);
            }
            const T w = (j == 0 || j == ny) ? (T)0.5 : (T)1;
            y[e] = epi_node<T, EPI>(ax, xc, b, e, w, acc, ca, c1, c2,
                                   (EPI == EPI_CHEB || EPI == EPI_CHEB_Z) ? dinv_at<T, KIND>(ca, ny, j, e) : (T)0);
        }
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

// ------------------------------------------------ nutrient (5-point, variable)
// y = dg x + gx [(a_c + a_e)(x - x_e) + (a_c + a_w)(x - x_w)]
//          + gy [(a_c + a_n)(x - x_n) + (a_c + a_s)(x - x_s)],
// the neighbours beyond the walls reflected (x_{-1} = x_1, a_{-1} = a_1,
// likewise at row ny); with op.nut_dtop row ny is y = dg x instead.  Sums of
// neighbour differences keep FP32 accurate where the expanded form cancels
// O(h^-2) terms.
template <typename T, int EPI, int TY, int XL>
__global__ void __launch_bounds__(256) k_nut5(Op op, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ y,
                                              SolveDev sd, const int* __restrict__ gate,
                                              double rtol, ChebArgs<T> ca) {
    if (gate && *gate) return;
    constexpr bool CH = EPI == EPI_CHEB || EPI == EPI_CHEB_Z;
    T c1 = 0, c2 = 0, cz = 0;
    if (CH) cheb_consts(ca, c1, c2);
    if (XL == XL_ZERO) cz = (T)ca.coef[1];
    const int nx = op.g.nx, ny = op.g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const T* __restrict__ dg = static_cast<const T*>(op.dg);
    const T gx = (T)op.gx, gy = (T)op.gy;
    EpiAcc<T> acc;
    if (i < nx) {
        const int im = i > 0 ? i - 1 : nx - 1;
        const int ip = i < nx - 1 ? i + 1 : 0;
#pragma unroll
        for (int r = 0; r < TY / 8; ++r) {
            const int j = blockIdx.y * TY + threadIdx.y + 8 * r;
            if (j > ny) continue;
            const size_t e = (size_t)j * nx + i;
            const T xc = load_x<T, XL, OP_NUT5>(x, b, ca, cz, ny, i, j, e);
            T ax;
            if (op.nut_dtop && j == ny) {
                if (CH && dz_row(ca.dirichlet_zero, j, ny)) {
                    y[e] = (T)0;
                    continue;
                }
                ax = mul_rn(dg[e], xc);
            } else {
                const int js = j > 0 ? j - 1 : 1;
                const int jn = j < ny ? j + 1 : ny - 1;
                const size_t row = (size_t)j * nx;
                const size_t es = (size_t)js * nx + i, en = (size_t)jn * nx + i;
                const T xe = load_x<T, XL, OP_NUT5>(x, b, ca, cz, ny, ip, j, row + ip);
                const T xw = load_x<T, XL, OP_NUT5>(x, b, ca, cz, ny, im, j, row + im);
                const T xn = load_x<T, XL, OP_NUT5>(x, b, ca, cz, ny, i, jn, en);
                const T xs = load_x<T, XL, OP_NUT5>(x, b, ca, cz, ny, i, js, es);
                const T ac = a[e];
                const T ce = ac + a[row + ip], cw = ac + a[row + im];
                const T cn = ac + a[en], cs = ac + a[es];
                const T sxv = fma(ce, xc - xe, mul_rn(cw, xc - xw));
                const T syv = fma(cn, xc - xn, mul_rn(cs, xc - xs));
                ax = fma(gx, sxv, fma(gy, syv, mul_rn(dg[e], xc)));
            }
            const T w = (j == 0 || j == ny) ? (T)0.5 : (T)1;
            y[e] = epi_node<T, EPI>(ax, xc, b, e, w, acc, ca, c1, c2,
                                   CH ? dinv_at<T, OP_NUT5>(ca, ny, j, e) : (T)0);
        }
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

// -------------------------------------------------------------- 13-point
template <typename T, int EPI, int TY, int XL>
__global__ void __launch_bounds__(256) k_ch13(Op op, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ y,
                                              SolveDev sd, const int* __restrict__ gate,
                                              double rtol, ChebArgs<T> ca) {
    if (gate && *gate) return;
    T c1 = 0, c2 = 0, cz = 0;
    if (EPI == EPI_CHEB || EPI == EPI_CHEB_Z) cheb_consts(ca, c1, c2);
    if (XL == XL_ZERO) cz = (T)ca.coef[1];
    constexpr int XW = TILE_X + 4, XH = TY + 4;   // x with halo 2
    constexpr int PW = TILE_X + 2, PH = TY + 2;   // psi, a with halo 1
    __shared__ T sx[XH][XW];
    __shared__ T sp[PH][PW];
    __shared__ T sa[PH][PW];
    const int nx = op.g.nx, ny = op.g.ny;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * TY;
    // Tile loads by fixed rows and columns: thread (tx, ty) loads rows
    // ty + 8r (reflected once per row) at column tx and, for the halo,
    // column 32 + tx (wrapped once per thread).  All loads are issued before
    // any shared-memory store, so a thread has them in flight at once.
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool wide = nx >= 2 * TILE_X;   // tile + halo wraps at most once
    auto wrapc = [&](int gi) { return wide ? wrapx_near(gi, nx) : wrapx(gi, nx); };
    const int gx0 = wrapc(i0 + tx - 2), gx1 = wrapc(i0 + TILE_X + tx - 2);   // x columns
    const int ga0 = wrapc(i0 + tx - 1), ga1 = wrapc(i0 + TILE_X + tx - 1);   // a columns
    constexpr int R = (XH + 7) / 8;   // passes of 8 rows cover the XH rows of x, PH of a
    T vx0[R], vx1[R], va0[R], va1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = ty + 8 * r;
        if (ly < XH) {
            const int jr = refly(j0 + ly - 2, ny);
            const size_t row = (size_t)jr * nx;
            vx0[r] = load_x<T, XL, OP_CH13>(x, b, ca, cz, ny, gx0, jr, row + gx0);
            if (tx < XW - TILE_X) vx1[r] = load_x<T, XL, OP_CH13>(x, b, ca, cz, ny, gx1, jr, row + gx1);
        }
        if (ly < PH) {
            const T* row = a + (size_t)refly(j0 + ly - 1, ny) * nx;
            va0[r] = row[ga0];
            if (tx < PW - TILE_X) va1[r] = row[ga1];
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = ty + 8 * r;
        if (ly < XH) {
            sx[ly][tx] = vx0[r];
            if (tx < XW - TILE_X) sx[ly][TILE_X + tx] = vx1[r];
        }
        if (ly < PH) {
            sa[ly][tx] = va0[r];
            if (tx < PW - TILE_X) sa[ly][TILE_X + tx] = va1[r];
        }
    }
    __syncthreads();
    // psi = kappa L_h x + S x on the tile and a one-node ring; ghost rows of
    // psi come out evenly reflected because x is.
    const T kx = (T)op.kx, ky = (T)op.ky;
    const T kc = (T)(2.0 * op.kx + 2.0 * op.ky + op.S);
    // psi of centre c, vertical neighbours v0, v2 and horizontal h0, h2
    auto psi_val = [&](T c, T v0, T v2, T h0, T h2) {
        if (sizeof(T) == 4)
            return fma(ky, (c - v0) + (c - v2), fma(kx, (c - h0) + (c - h2), mul_rn((T)op.S, c)));
        return fma(-ky, v0 + v2, fma(-kx, h0 + h2, mul_rn(kc, c)));
    };
    auto psi_at = [&](int ly, int lx) {
        return psi_val(sx[ly + 1][lx + 1], sx[ly][lx + 1], sx[ly + 2][lx + 1], sx[ly + 1][lx],
                       sx[ly + 1][lx + 2]);
    };
    // Register blocking in y: thread (tx, ty) forms the psi column strip of
    // rows RPT ty .. RPT ty + RPT - 1 (RPT = TY / 8) with the strip's column
    // of x held in registers (each x value loaded once); the two ring rows
    // TY, TY + 1 go to the threads ty < 2, the ring columns 32, 33 to tx < 2.
    constexpr int RPT = TY / 8;
    auto psi_strip = [&](int lx) {
        T col[RPT + 2];
#pragma unroll
        for (int k = 0; k < RPT + 2; ++k) col[k] = sx[ty * RPT + k][lx + 1];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int ly = ty * RPT + k;
            sp[ly][lx] = psi_val(col[k + 1], col[k], col[k + 2], sx[ly + 1][lx], sx[ly + 1][lx + 2]);
        }
    };
    psi_strip(tx);
    if (tx < PW - TILE_X) psi_strip(TILE_X + tx);
    if (ty < PH - TY) {
        sp[TY + ty][tx] = psi_at(TY + ty, tx);
        if (tx < PW - TILE_X) sp[TY + ty][TILE_X + tx] = psi_at(TY + ty, TILE_X + tx);
    }
    __syncthreads();
    const T gxq = (T)(0.25 * op.gx), gyq = (T)(0.25 * op.gy);   // 1/2 (CN) x 1/2 (face mean)
    const T idt = (T)op.idt;
    EpiAcc<T> acc;
    const int i = i0 + tx;
    // the same blocking for the output rows: the column of psi and a from
    // row RPT ty - 1 to RPT ty + RPT stays in registers
    const int px = tx + 1;
    T pcol[RPT + 2], acol[RPT + 2];
#pragma unroll
    for (int k = 0; k < RPT + 2; ++k) {
        pcol[k] = sp[ty * RPT + k][px];
        acol[k] = sa[ty * RPT + k][px];
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int oy = ty * RPT + k, j = j0 + oy;
        if (i < nx && j <= ny) {
            const int py = oy + 1;
            const T pc = pcol[k + 1], ac = acol[k + 1];
            const T fx = fma(ac + sa[py][px + 1], sp[py][px + 1] - pc,
                             -mul_rn(ac + sa[py][px - 1], pc - sp[py][px - 1]));
            const T fy = fma(ac + acol[k + 2], pcol[k + 2] - pc,
                             -mul_rn(ac + acol[k], pc - pcol[k]));
            const T xc = sx[oy + 2][tx + 2];
            const T ax = fma(-gyq, fy, fma(-gxq, fx, mul_rn(idt, xc)));
            const size_t e = (size_t)j * nx + i;
            const T w = (j == 0 || j == ny) ? (T)0.5 : (T)1;
            y[e] = epi_node<T, EPI>(ax, xc, b, e, w, acc, ca, c1, c2,
                                   (EPI == EPI_CHEB || EPI == EPI_CHEB_Z) ? ca.dinv[e] : (T)0);
        }
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

// W-adjoint of the 13-point operator: t = G_a x on the tile and a one-node
// ring (x and a staged with halo 2), then idt x + 1/2 (kappa L_h + S) t.
// Ghost rows of t come out evenly reflected because x and a are.
template <typename T, int EPI, int TY>
__global__ void __launch_bounds__(256) k_ch13_wadj(Op op, const T* __restrict__ x,
                                                   const T* __restrict__ b, T* __restrict__ y,
                                                   SolveDev sd, const int* __restrict__ gate,
                                                   double rtol, ChebArgs<T> ca) {
    if (gate && *gate) return;
    T c1 = 0, c2 = 0;
    if (EPI == EPI_CHEB) cheb_consts(ca, c1, c2);
    constexpr int XW = TILE_X + 4, XH = TY + 4;   // x, a with halo 2
    constexpr int PW = TILE_X + 2, PH = TY + 2;   // t with halo 1
    __shared__ T sx[XH][XW];
    __shared__ T sa[XH][XW];
    __shared__ T st[PH][PW];
    const int nx = op.g.nx, ny = op.g.ny;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const int i0 = blockIdx.x * TILE_X, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool wide = nx >= 2 * TILE_X;
    auto wrapc = [&](int gi) { return wide ? wrapx_near(gi, nx) : wrapx(gi, nx); };
    const int gx0 = wrapc(i0 + tx - 2), gx1 = wrapc(i0 + TILE_X + tx - 2);
    constexpr int R = (XH + 7) / 8;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = ty + 8 * r;
        if (ly < XH) {
            const size_t row = (size_t)refly(j0 + ly - 2, ny) * nx;
            sx[ly][tx] = x[row + gx0];
            sa[ly][tx] = a[row + gx0];
            if (tx < XW - TILE_X) {
                sx[ly][TILE_X + tx] = x[row + gx1];
                sa[ly][TILE_X + tx] = a[row + gx1];
            }
        }
    }
    __syncthreads();
    const T hgx = (T)(0.5 * op.gx), hgy = (T)(0.5 * op.gy);   // face mean x 1/h^2
    auto t_at = [&](int ly, int lx) {   // G_a x at smem node (ly + 1, lx + 1)
        const int cy = ly + 1, cx = lx + 1;
        const T xc = sx[cy][cx], ac = sa[cy][cx];
        const T fx = fma(ac + sa[cy][cx + 1], sx[cy][cx + 1] - xc,
                         -mul_rn(ac + sa[cy][cx - 1], xc - sx[cy][cx - 1]));
        const T fy = fma(ac + sa[cy + 1][cx], sx[cy + 1][cx] - xc,
                         -mul_rn(ac + sa[cy - 1][cx], xc - sx[cy - 1][cx]));
        return -fma(hgy, fy, mul_rn(hgx, fx));
    };
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = ty + 8 * r;
        if (ly < PH) {
            st[ly][tx] = t_at(ly, tx);
            if (tx < PW - TILE_X) st[ly][TILE_X + tx] = t_at(ly, TILE_X + tx);
        }
    }
    __syncthreads();
    const T kx = (T)op.kx, ky = (T)op.ky, S = (T)op.S, idt = (T)op.idt, h = (T)0.5;
    EpiAcc<T> acc;
    const int i = i0 + tx;
#pragma unroll
    for (int r = 0; r < TY / 8; ++r) {
        const int oy = ty + 8 * r, j = j0 + oy;
        if (i < nx && j <= ny) {
            const int py = oy + 1, px = tx + 1;
            const T tc = st[py][px];
            const T lt = fma(ky, (tc - st[py - 1][px]) + (tc - st[py + 1][px]),
                             mul_rn(kx, (tc - st[py][px - 1]) + (tc - st[py][px + 1])));
            const T xc = sx[oy + 2][tx + 2];
            const T ax = fma(h, fma(S, tc, lt), mul_rn(idt, xc));
            const size_t e = (size_t)j * nx + i;
            const T w = (j == 0 || j == ny) ? (T)0.5 : (T)1;
            y[e] = epi_node<T, EPI>(ax, xc, b, e, w, acc, ca, c1, c2,
                                   (EPI == EPI_CHEB || EPI == EPI_CHEB_Z) ? ca.dinv[e] : (T)0);
        }
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

// The maximum of v over every thread of the launch (block maxima, then the
// last block to finish, which resets the counter): true in every thread of
// the last block, each of which receives it in m.
__device__ __forceinline__ bool max_last(double v, RedWs red, double& m) {
    __shared__ double sh[32];
    __shared__ double s_m;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int t = flat_tid();
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        double w = t < 8 ? sh[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (t == 0) red.partials[flat_bid()] = w;
    }
    if (!last_block(red)) return false;
    double mb = 0.0;
    for (int b = t; b < nblocks(); b += 256) mb = fmax(mb, __ldcg(red.partials + b));
    for (int o = 16; o > 0; o >>= 1) mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    __syncthreads();
    if ((t & 31) == 0) sh[t >> 5] = mb;
    __syncthreads();
    if (t == 0) {
        double r = 0.0;
        for (int k = 0; k < 8; ++k) r = fmax(r, sh[k]);
        s_m = r;
        reset_counter(red);
    }
    __syncthreads();
    m = s_m;
    return true;
}
// *out = that maximum
__device__ __forceinline__ void max_to(double v, double* out, RedWs red) {
    double m;
    if (max_last(v, red, m) && flat_tid() == 0) *out = m;
}

// Exact diagonal of A_phi (Jacobi scaling and smoother):
// idt + 1/2 [ G_ii (kappa L_ii + S) + kappa sum_{k != i} G_ik L_ki ].
template <typename T>
__global__ void __launch_bounds__(256) k_ch13_diag(Op op, T* __restrict__ d) {
    const int nx = op.g.nx, ny = op.g.ny;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const int js = refly(j - 1, ny), jn = refly(j + 1, ny);
        const double ac = a[(size_t)j * nx + i];
        const double fe = 0.5 * (ac + (double)a[(size_t)j * nx + ip]);
        const double fw = 0.5 * (ac + (double)a[(size_t)j * nx + im]);
        const double fn = 0.5 * (ac + (double)a[(size_t)jn * nx + i]);
        const double fs = 0.5 * (ac + (double)a[(size_t)js * nx + i]);
        // weight of the wall row's own Laplacian row on its interior neighbour
        const double cn = (j + 1 == ny) ? 2.0 : 1.0;
        const double cs = (j - 1 == 0) ? 2.0 : 1.0;
        const double gii = (fe + fw) * op.gx + (fn + fs) * op.gy;
        const double off = (fe + fw) * op.gx * op.kx + (fn * cn + fs * cs) * op.gy * op.ky;
        d[(size_t)j * nx + i] = (T)(op.idt + 0.5 * (gii * (2.0 * op.kx + 2.0 * op.ky + op.S) + off));
    }
}

// dinv = 1 / diag(A_phi); lam = max_i R_i / D_ii with the Gershgorin row
// bound R_i = idt + G_ii (2 kappa d_L + S) (d_L = 2/hx^2 + 2/hy^2; every
// row of L_h has absolute sum 2 d_L and every row of G_a 2 G_ii).  For a
// constant coefficient the bound is attained by the checkerboard mode.
// The same launch restricts the coefficient to the next level (ac, when
// given: grid-stride over its nodes, as k_restrict) and, in the last block,
// writes the level's Chebyshev tables from lam.  Arithmetic in the solve's
// precision, with the operator's constants rounded to T on the host (FP64
// arithmetic is 58x slower here); the maximum is taken in T and widened
// once (exact).
template <typename T>
struct Ch13DiagC {
    T gx, gy, kx, ky, S, idt;
};
template <typename T>
__global__ void __launch_bounds__(256) k_ch13_level(Op op, Ch13DiagC<T> c, T* __restrict__ dinv,
                                                    double* __restrict__ lam, RedWs red, Grid gc,
                                                    int semi, T* __restrict__ ac, ChebTabs tabs,
                                                    const int* __restrict__ gate) {
    if (gate && *gate) return;   // uniform: no block reaches the reduction
    const int nx = op.g.nx, ny = op.g.ny;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    T mx = (T)0;
    if (i < nx) {
        const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
        for (int r = 0; r < TILE_Y / 8; ++r) {
            const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
            if (j > ny) break;
            const int js = refly(j - 1, ny), jn = refly(j + 1, ny);
            const T ac0 = a[(size_t)j * nx + i];
            const T h = (T)0.5;
            const T fe = h * (ac0 + a[(size_t)j * nx + ip]);
            const T fw = h * (ac0 + a[(size_t)j * nx + im]);
            const T fn = h * (ac0 + a[(size_t)jn * nx + i]);
            const T fs = h * (ac0 + a[(size_t)js * nx + i]);
            const T cn = (j + 1 == ny) ? (T)2 : (T)1;
            const T cs = (j - 1 == 0) ? (T)2 : (T)1;
            const T gii = (fe + fw) * c.gx + (fn + fs) * c.gy;
            const T off = (fe + fw) * c.gx * c.kx + (fn * cn + fs * cs) * c.gy * c.ky;
            const T D = c.idt + h * (gii * ((T)2 * c.kx + (T)2 * c.ky + c.S) + off);
            const T R = c.idt + gii * ((T)4 * c.kx + (T)4 * c.ky + c.S);
            dinv[(size_t)j * nx + i] = (T)1 / D;
            mx = fmax(mx, R / D);
        }
    }
    if (ac) {
        const size_t nc = gc.n(), ts = (size_t)nblocks() * 256;
        for (size_t e = (size_t)flat_bid() * 256 + flat_tid(); e < nc; e += ts) {
            const int J = (int)(e / gc.nx), I = (int)(e - (size_t)J * gc.nx);
            const int cc = semi ? I : 2 * I;
            auto fine = [&](int jj, int dx) {
                int ii = cc + dx;
                ii = ii < 0 ? nx - 1 : (ii >= nx ? 0 : ii);
                return a[(size_t)jj * nx + ii];
            };
            ac[e] = restrict_at<T>(fine, J, ny, semi, gc.ny);
        }
    }
    double m;
    if (max_last((double)mx, red, m)) {
        if (flat_tid() == 0) *lam = m;
        cheb_tables_dev(tabs, m, flat_tid(), 256);
    }
}

// dinv = 1 / diag(K) and *lam = max_i (Gershgorin row bound / D_ii) of the
// nutrient operator: D = dg + S, R = dg + 2 S with S = gx (c_e + c_w) +
// gy (c_n + c_s) (a wall row's reflected neighbour adds its weight to the
// row inside), R / D = 1 on a Dirichlet row.
// The same launch restricts a and dg to the next level (ac, dgc, when
// given) and, in its last block, writes the level's Chebyshev tables from
// lam; the maximum is taken in T and widened once (exact).
template <typename T>
__global__ void __launch_bounds__(256) k_nut_level(Op op, T gxT, T gyT, T* __restrict__ dinv,
                                                   double* __restrict__ lam, RedWs red, Grid gc,
                                                   int semi, T* __restrict__ ac,
                                                   T* __restrict__ dgc, ChebTabs tabs) {
    const int nx = op.g.nx, ny = op.g.ny;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const T* __restrict__ dg = static_cast<const T*>(op.dg);
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    T mx = (T)0;
    if (i < nx) {
        const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
        for (int r = 0; r < TILE_Y / 8; ++r) {
            const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
            if (j > ny) break;
            const size_t e = (size_t)j * nx + i;
            if (op.nut_dtop && j == ny) {
                dinv[e] = (T)1 / dg[e];
                mx = fmax(mx, (T)1);
                continue;
            }
            const int js = j > 0 ? j - 1 : 1, jn = j < ny ? j + 1 : ny - 1;
            const T a0 = a[e];
            const T S = gxT * ((a0 + a[(size_t)j * nx + ip]) + (a0 + a[(size_t)j * nx + im])) +
                        gyT * ((a0 + a[(size_t)jn * nx + i]) + (a0 + a[(size_t)js * nx + i]));
            const T D = dg[e] + S;
            dinv[e] = (T)1 / D;
            mx = fmax(mx, (D + S) / D);
        }
    }
    if (ac) {
        const size_t nc = gc.n(), ts = (size_t)nblocks() * 256;
        for (size_t e = (size_t)flat_bid() * 256 + flat_tid(); e < nc; e += ts) {
            const int J = (int)(e / gc.nx), I = (int)(e - (size_t)J * gc.nx);
            const int cc = semi ? I : 2 * I;
            auto at = [&](const T* f) {
                return [&, f](int jj, int dx) {
                    int ii = cc + dx;
                    ii = ii < 0 ? nx - 1 : (ii >= nx ? 0 : ii);
                    return f[(size_t)jj * nx + ii];
                };
            };
            ac[e] = restrict_at<T>(at(a), J, ny, semi, gc.ny);
            dgc[e] = restrict_at<T>(at(dg), J, ny, semi, gc.ny);
        }
    }
    double m;
    if (max_last((double)mx, red, m)) {
        if (flat_tid() == 0) *lam = m;
        cheb_tables_dev(tabs, m, flat_tid(), 256);
    }
}

// ---------------------------------------------------------------- launch
template <typename T, int EPI, int TY, int XL>
static void launch_tile(const Op& op, const T* x, const T* b, T* y, SolveDev sd,
                        const int* gate, double rtol, cudaStream_t s, const ChebArgs<T>& ca) {
    dim3 grid = tile_grid(op.g.nx, op.g.ny, TY), blk(32, 8);
    switch (op.kind) {
        case OP_LAP5_NEUMANN:
            note_launch(); launch_k(k_lap5<T, OP_LAP5_NEUMANN, EPI, TY, XL>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol, ca);
            break;
        case OP_LAP5_DIRICHLET:
            note_launch(); launch_k(k_lap5<T, OP_LAP5_DIRICHLET, EPI, TY, XL>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol, ca);
            break;
        case OP_NUT5:
            note_launch(); launch_k(k_nut5<T, EPI, TY, XL>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol, ca);
            break;
        case OP_CH13_WADJ:
            if constexpr (sizeof(T) == 8 && XL == XL_PLAIN) {
                note_launch(); launch_k(k_ch13_wadj<T, EPI, TY>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol, ca);
            } else {
                throw ArgError("OP_CH13_WADJ: FP64 plain applies only");
            }
            break;
        default:
            note_launch(); launch_k(k_ch13<T, EPI, TY, XL>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol, ca);
            break;
    }
}

// Launches with a block reduction keep the 32-row tile, so the order of
// every reduction is fixed whatever tile the operator was tuned to.
template <typename T, int EPI, int XL>
static void launch_ty(const Op& op, const T* x, const T* b, T* y, SolveDev sd,
                      const int* gate, double rtol, cudaStream_t s, const ChebArgs<T>& ca) {
    // fine grids: the vectorised tiles of stencil_vec.cu (same value at every node)
    constexpr bool VEC = (XL == XL_PLAIN && EPI != EPI_CHEB_Z) ||
                         (XL == XL_PROLONG && EPI == EPI_CHEB) ||
                         (XL == XL_ZERO && EPI == EPI_CHEB_Z);
    if constexpr (VEC) {
        if (vec_eligible<T>(op, EPI, x, b, y, ca, sd)) {
            launch_vec<T, EPI, XL>(op, x, b, y, sd, gate, rtol, s, ca);
            return;
        }
    }
    if constexpr (EPI == EPI_APPLY || EPI == EPI_RPLAIN || EPI == EPI_CHEB ||
                  EPI == EPI_CHEB_Z) {
        switch (op.ty) {
            case 8: launch_tile<T, EPI, 8, XL>(op, x, b, y, sd, gate, rtol, s, ca); return;
            case 16: launch_tile<T, EPI, 16, XL>(op, x, b, y, sd, gate, rtol, s, ca); return;
            default: break;
        }
    }
    launch_tile<T, EPI, TILE_Y, XL>(op, x, b, y, sd, gate, rtol, s, ca);
}

template <typename T, int EPI>
static void launch_op_epi(const Op& op, const T* x, const T* b, T* y, SolveDev sd,
                          const int* gate, double rtol, cudaStream_t s,
                          const ChebArgs<T>& ca = ChebArgs<T>(), int xl = XL_PLAIN) {
    if constexpr (EPI == EPI_CHEB) {
        if (xl == XL_ZERO) {
            launch_ty<T, EPI_CHEB_Z, XL_ZERO>(op, x, b, y, sd, gate, rtol, s, ca);
            return;
        }
        if (xl == XL_PROLONG) {
            launch_ty<T, EPI_CHEB, XL_PROLONG>(op, x, b, y, sd, gate, rtol, s, ca);
            return;
        }
    }
    launch_ty<T, EPI, XL_PLAIN>(op, x, b, y, sd, gate, rtol, s, ca);
}

template <typename T>
void launch_op(const Op& op, Epi epi, const T* x, const T* b, T* y, SolveDev sd,
               const int* gate, double rtol, cudaStream_t s) {
    if (op.kind == OP_VISC) {   // the coupled momentum operator (visc.cu)
        launch_visc<T>(op, epi, x, b, y, sd, gate, rtol, s);
        return;
    }
    switch (epi) {
        case EPI_APPLY: launch_op_epi<T, EPI_APPLY>(op, x, b, y, sd, gate, rtol, s); break;
        case EPI_RESID: launch_op_epi<T, EPI_RESID>(op, x, b, y, sd, gate, rtol, s); break;
        case EPI_RESIDX: launch_op_epi<T, EPI_RESIDX>(op, x, b, y, sd, gate, rtol, s); break;
        case EPI_DOTXY: launch_op_epi<T, EPI_DOTXY>(op, x, b, y, sd, gate, rtol, s); break;
        case EPI_CGCG: launch_op_epi<T, EPI_CGCG>(op, x, b, y, sd, gate, rtol, s); break;
        case EPI_RPLAIN: launch_op_epi<T, EPI_RPLAIN>(op, x, b, y, sd, gate, rtol, s); break;
        default: launch_op_epi<T, EPI_NORM>(op, x, b, y, sd, gate, rtol, s); break;
    }
}

template <typename T>
void launch_cheb(const Op& op, const T* x, const T* b, T* y, const ChebArgs<T>& ca,
                 const int* gate, cudaStream_t s, int xl) {
    launch_op_epi<T, EPI_CHEB>(op, x, b, y, SolveDev{}, gate, 0.0, s, ca, xl);
}

template <typename T>
void launch_ch13_diag(const Op& op, T* diag, cudaStream_t s) {
    note_launch(); launch_k(k_ch13_diag<T>, tile_grid(op.g.nx, op.g.ny), dim3(32, 8), 0, s, op, diag);
}

template void launch_op<double>(const Op&, Epi, const double*, const double*, double*, SolveDev,
                                const int*, double, cudaStream_t);
template void launch_op<float>(const Op&, Epi, const float*, const float*, float*, SolveDev,
                               const int*, double, cudaStream_t);
template void launch_cheb<double>(const Op&, const double*, const double*, double*,
                                  const ChebArgs<double>&, const int*, cudaStream_t, int);
template void launch_cheb<float>(const Op&, const float*, const float*, float*,
                                 const ChebArgs<float>&, const int*, cudaStream_t, int);
template <typename T>
void launch_ch13_level(const Op& op, T* dinv, double* lam, RedWs red, const Grid& gc, int semi,
                       T* ac, const ChebTabs& tabs, const int* gate, cudaStream_t s) {
    const Ch13DiagC<T> c{(T)op.gx, (T)op.gy, (T)op.kx, (T)op.ky, (T)op.S, (T)op.idt};
    note_launch(); launch_k(k_ch13_level<T>, tile_grid(op.g.nx, op.g.ny), dim3(32, 8), 0, s, op, c, dinv, lam, red, gc, semi, ac, tabs, gate);
}
template void launch_ch13_level<double>(const Op&, double*, double*, RedWs, const Grid&, int, double*,
                                        const ChebTabs&, const int*, cudaStream_t);
template void launch_ch13_level<float>(const Op&, float*, double*, RedWs, const Grid&, int, float*,
                                       const ChebTabs&, const int*, cudaStream_t);
template <typename T>
void launch_nut_level(const Op& op, T* dinv, double* lam, RedWs red, const Grid& gc, int semi,
                      T* ac, T* dgc, const ChebTabs& tabs, cudaStream_t s) {
    note_launch(); launch_k(k_nut_level<T>, tile_grid(op.g.nx, op.g.ny), dim3(32, 8), 0, s, op, (T)op.gx, (T)op.gy, dinv, lam, red, gc, semi, ac, dgc, tabs);
}
template void launch_nut_level<double>(const Op&, double*, double*, RedWs, const Grid&, int, double*,
                                       double*, const ChebTabs&, cudaStream_t);
template void launch_nut_level<float>(const Op&, float*, double*, RedWs, const Grid&, int, float*,
                                      float*, const ChebTabs&, cudaStream_t);
template void launch_ch13_diag<double>(const Op&, double*, cudaStream_t);
template void launch_ch13_diag<float>(const Op&, float*, cudaStream_t);

// ------------------------------------------------------------- autotuner
// Tile height of an operator's launches without reductions, picked by
// timing: each candidate (32, 16, 8 rows per 32-column block) runs the
// multigrid residual y = b - A x 20 times between CUDA events on the
// context's stream; a shorter tile is taken only when it is at least 3%
// faster than the best taller one.  Short tiles give small (coarse-level)
// grids more blocks; tall ones amortise the halo rows on large grids.
// Every candidate computes each node with the same arithmetic, so the pick
// changes timing only.  Results are cached per (device, kind, precision,
// grid);
// CAHN_TILE=8|16|32 in the environment forces one height.
int forced_tile_height() {
    const char* e = std::getenv("CAHN_TILE");
    if (!e) return 0;
    const int v = std::atoi(e);
    return (v == 8 || v == 16 || v == 32) ? v : 0;
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune_cache;
}  // namespace

template <typename T>
int tune_tile(const Op& op, cudaStream_t s) {
    if (const int f = forced_tile_height()) return f;
    int dev = 0;
    CAHN_CUDA_TRY(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, op.kind, (int)sizeof(T), op.g.nx, op.g.ny);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
    const size_t n = op.g.n();
    T *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best = TILE_Y;
    try {
        CAHN_CUDA_TRY(cudaMalloc(&x, n * sizeof(T)));
        CAHN_CUDA_TRY(cudaMalloc(&y, n * sizeof(T)));
        CAHN_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(T), s));
        CAHN_CUDA_TRY(cudaEventCreate(&e0));
        CAHN_CUDA_TRY(cudaEventCreate(&e1));
        float best_ms = 0.0f;
        const int cand[3] = {32, 16, 8};
        for (int c = 0; c < 3; ++c) {
            Op o = op;
            o.ty = cand[c];
            for (int k = 0; k < 3; ++k)
                launch_op_epi<T, EPI_RPLAIN>(o, x, x, y, SolveDev{}, nullptr, 0.0, s);
            CAHN_CUDA_TRY(cudaEventRecord(e0, s));
            for (int k = 0; k < 20; ++k)
                launch_op_epi<T, EPI_RPLAIN>(o, x, x, y, SolveDev{}, nullptr, 0.0, s);
            CAHN_CUDA_TRY(cudaEventRecord(e1, s));
            CAHN_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CAHN_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (c == 0 || ms < 0.97f * best_ms) {
                best = cand[c];
                best_ms = ms;
            }
        }
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(x);
        cudaFree(y);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    g_tune_cache[key] = best;
    return best;
}
template int tune_tile<double>(const Op&, cudaStream_t);
template int tune_tile<float>(const Op&, cudaStream_t);

}  // namespace cahn
