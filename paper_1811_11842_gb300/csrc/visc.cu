// Fully implicit variable-viscosity momentum (the stress of Eq. 4.1 without
// the eta_bar split of Eq. 4.2): Crank-Nicolson on
//   div(2 eta D(v)) = ( d/dx(2 eta u_x) + d/dy(eta u_y) + d/dy(eta v_x),
//                       d/dx(eta u_y) + d/dx(eta v_x) + d/dy(2 eta v_y) ),
// eta = phi eta_b + (1 - phi) eta_w at phi^{n+1/2}.  The normal and
// tangential second derivatives take the compact face-mean form (face value
// the mean of the two nodes), the cross derivatives central differences of
// central differences, so the 9-point block matrix
//   rho/dt - 1/2 div(2 eta D(.))
// is symmetric and, on the fields that vanish on the (Dirichlet) walls,
// bounded below by rho/dt: the discrete viscous form
// sum 2 eta (D_h v : D_h v) is positive semi-definite because a central
// difference is the mean of the two compact differences beside it.
#include "stencil_dev.cuh"
#include "visc.h"

namespace cahn {

// div(2 eta D(v)) at interior node (i, j) of a component grid; E, U, V give
// eta, u and v at (i, j).
template <typename T, typename FE, typename FU, typename FV>
__device__ __forceinline__ void visc_div(int i, int j, int nx, const FE& E, const FU& U,
                                         const FV& V, T gx, T gy, T gxy, T& tu, T& tv) {
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const int js = j - 1, jn = j + 1;
    const T ec = E(i, j), ee = E(ip, j), ew = E(im, j), en = E(i, jn), es = E(i, js);
    const T uc = U(i, j), vc = V(i, j);
    const T fxe = ec + ee, fxw = ec + ew, fyn = ec + en, fys = ec + es;   // 2 x face means
    const T half = (T)0.5;
    const T du_x = fxe * (U(ip, j) - uc) - fxw * (uc - U(im, j));
    const T du_y = fyn * (U(i, jn) - uc) - fys * (uc - U(i, js));
    const T dv_x = fxe * (V(ip, j) - vc) - fxw * (vc - V(im, j));
    const T dv_y = fyn * (V(i, jn) - vc) - fys * (vc - V(i, js));
    const T cross_u = en * (V(ip, jn) - V(im, jn)) - es * (V(ip, js) - V(im, js));
    const T cross_v = ee * (U(ip, jn) - U(ip, js)) - ew * (U(im, jn) - U(im, js));
    tu = gx * du_x + half * gy * du_y + gxy * cross_u;
    tv = gxy * cross_v + half * gx * dv_x + gy * dv_y;
}

__global__ void __launch_bounds__(256) k_mom_rhs_impl(Grid g, PhysDev P, const double* __restrict__ u,
                                                      const double* __restrict__ v, MomWs W,
                                                      double* __restrict__ bu,
                                                      double* __restrict__ bv) {
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double ihx2 = 0.5 / g.hx, ihy2 = 0.5 / g.hy;
    const double gx = 1.0 / (g.hx * g.hx), gy = 1.0 / (g.hy * g.hy);
    const double gxy = 0.25 / (g.hx * g.hy);
    auto E = [&](int a, int b) { return W.ep[(size_t)b * nx + a]; };
    auto U = [&](int a, int b) { return u[(size_t)b * nx + a]; };
    auto V = [&](int a, int b) { return v[(size_t)b * nx + a]; };
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const size_t e = (size_t)j * nx + i;
        if (j == 0 || j == ny) {
            bu[e] = P.rho * P.idt * (j == 0 ? P.u_wall0 : P.u_wall1);
            bv[e] = 0.0;
            continue;
        }
        const size_t ew = (size_t)j * nx + im, ee = (size_t)j * nx + ip;
        const size_t es = (size_t)(j - 1) * nx + i, en = (size_t)(j + 1) * nx + i;
        const double gam = P.gamma_cap;
        const double cxf = -gam * ((W.txx[ee] - W.txx[ew]) * ihx2 + (W.txy[en] - W.txy[es]) * ihy2);
        const double cyf = -gam * ((W.txy[ee] - W.txy[ew]) * ihx2 + (W.tyy[en] - W.tyy[es]) * ihy2);
        const double usc = W.us[e], vsc = W.vs[e];
        const double us_x = (W.us[ee] - W.us[ew]) * ihx2, us_y = (W.us[en] - W.us[es]) * ihy2;
        const double vs_x = (W.vs[ee] - W.vs[ew]) * ihx2, vs_y = (W.vs[en] - W.vs[es]) * ihy2;
        const double conv_u = usc * us_x + vsc * us_y;
        const double conv_v = usc * vs_x + vsc * vs_y;
        double tu, tv;
        visc_div<double>(i, j, nx, E, U, V, gx, gy, gxy, tu, tv);
        bu[e] = P.rho * u[e] * P.idt - P.rho * conv_u + 0.5 * tu + cxf + P.fx;
        bv[e] = P.rho * v[e] * P.idt - P.rho * conv_v + 0.5 * tv + cyf;
    }
}

// y = A [u; v] with epilogue EPI, one thread per node of the component grid
// (both components); the trapezoid weights are those of the stacked grid
// (every Krylov vector vanishes on the wall rows, where they differ).
template <typename T, int EPI>
__global__ void __launch_bounds__(256) k_visc(Op op, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ y,
                                              SolveDev sd, const int* __restrict__ gate,
                                              double rtol) {
    if (gate && *gate) return;
    const int nx = op.g.nx, ny = (op.g.ny - 1) / 2;
    const size_t nc = (size_t)nx * (ny + 1);
    const T* __restrict__ eta = static_cast<const T*>(op.a);
    const T c0 = (T)op.c0, gx = (T)op.gx, gy = (T)op.gy, gxy = (T)op.kx, half = (T)0.5;
    const ChebArgs<T> ca{};
    EpiAcc<T> acc;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    auto E = [&](int a, int c) { return eta[(size_t)c * nx + a]; };
    auto U = [&](int a, int c) { return x[(size_t)c * nx + a]; };
    auto V = [&](int a, int c) { return x[nc + (size_t)c * nx + a]; };
    if (i < nx) {
        for (int r = 0; r < TILE_Y / 8; ++r) {
            const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
            if (j > ny) break;
            const size_t e = (size_t)j * nx + i;
            const T uc = x[e], vc = x[nc + e];
            T au, av;
            if (j == 0 || j == ny) {
                au = c0 * uc;
                av = c0 * vc;
            } else {
                T tu, tv;
                visc_div<T>(i, j, nx, E, U, V, gx, gy, gxy, tu, tv);
                au = c0 * uc - half * tu;
                av = c0 * vc - half * tv;
            }
            const T wu = j == 0 ? (T)0.5 : (T)1, wv = j == ny ? (T)0.5 : (T)1;
            y[e] = epi_node<T, EPI>(au, uc, b, e, wu, acc, ca, (T)0, (T)0, (T)0);
            y[nc + e] = epi_node<T, EPI>(av, vc, b, nc + e, wv, acc, ca, (T)0, (T)0, (T)0);
        }
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

template <typename T>
__global__ void __launch_bounds__(256) k_visc_dinv(Op op, T* __restrict__ dinv) {
    const int nx = op.g.nx, ny = (op.g.ny - 1) / 2;
    const size_t nc = (size_t)nx * (ny + 1);
    const T* __restrict__ eta = static_cast<const T*>(op.a);
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double c0 = op.c0, gx = op.gx, gy = op.gy;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const size_t e = (size_t)j * nx + i;
        if (j == 0 || j == ny) {
            dinv[e] = dinv[nc + e] = (T)(1.0 / c0);
            continue;
        }
        const double ec = eta[e];
        const double sx = 2.0 * ec + eta[(size_t)j * nx + ip] + eta[(size_t)j * nx + im];
        const double sy = 2.0 * ec + eta[(size_t)(j + 1) * nx + i] + eta[(size_t)(j - 1) * nx + i];
        dinv[e] = (T)(1.0 / (c0 + 0.5 * (gx * sx + 0.5 * gy * sy)));
        dinv[nc + e] = (T)(1.0 / (c0 + 0.5 * (0.5 * gx * sx + gy * sy)));
    }
}

// ---------------------------------------------------------------- launch
static dim3 comp_grid(const Op& op) { return tile_grid(op.g.nx, (op.g.ny - 1) / 2); }

void launch_mom_rhs_impl(const Grid& g, const PhysDev& P, const double* u, const double* v,
                         const MomWs& W, double* bu, double* bv, cudaStream_t s) {
    note_launch(); launch_k(k_mom_rhs_impl, tile_grid(g.nx, g.ny), dim3(32, 8), 0, s, g, P, u, v, W, bu, bv);
}

template <typename T>
void launch_visc(const Op& op, Epi epi, const T* x, const T* b, T* y, SolveDev sd,
                 const int* gate, double rtol, cudaStream_t s) {
    const dim3 grid = comp_grid(op), blk(32, 8);
    note_launch();
    switch (epi) {
        case EPI_APPLY: launch_k(k_visc<T, EPI_APPLY>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        case EPI_RESID: launch_k(k_visc<T, EPI_RESID>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        case EPI_RESIDX: launch_k(k_visc<T, EPI_RESIDX>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        case EPI_DOTXY: launch_k(k_visc<T, EPI_DOTXY>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        case EPI_CGCG: launch_k(k_visc<T, EPI_CGCG>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        case EPI_RPLAIN: launch_k(k_visc<T, EPI_RPLAIN>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        case EPI_NORM: launch_k(k_visc<T, EPI_NORM>, grid, blk, 0, s, op, x, b, y, sd, gate, rtol); break;
        default: throw ArgError("OP_VISC: no smoother epilogue");
    }
}

template <typename T>
void launch_visc_dinv(const Op& op, T* dinv, cudaStream_t s) {
    note_launch(); launch_k(k_visc_dinv<T>, comp_grid(op), dim3(32, 8), 0, s, op, dinv);
}

template void launch_visc<double>(const Op&, Epi, const double*, const double*, double*, SolveDev,
                                  const int*, double, cudaStream_t);
template void launch_visc<float>(const Op&, Epi, const float*, const float*, float*, SolveDev,
                                 const int*, double, cudaStream_t);
template void launch_visc_dinv<double>(const Op&, double*, cudaStream_t);
template void launch_visc_dinv<float>(const Op&, float*, cudaStream_t);

}  // namespace cahn
