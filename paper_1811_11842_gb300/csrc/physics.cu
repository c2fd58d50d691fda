// Explicit parts of one time step (FP64): the right-hand sides of the
// phase-field and velocity-predictor systems, the mass correction, the
// divergence of the predicted velocity and the projection update.
//
//   CH   (Eq. 2.4, CN + extrapolation, §4):
//        b = phi^n/dt - G_a( 1/2 (kappa L_h + S) phi^n + F'(phi*) - S phi* )
//            - D_c(phi* v*),     a = M phi*,  q* = (3 q^n - q^{n-1}) / 2
//   momentum (Eq. 4.1-4.3), interior rows:
//        b = rho u^n/dt - rho (v*.grad) u* - eta_bar/2 L_h u^n + R + f
//        R = -Gamma div(grad phi grad phi) + div(eta' grad v*)
//            + (grad v*)^T grad eta',  eta' = eta(phi^{n+1/2}) - eta_bar
//   pressure rhs (Eq. 4.4): d = rho D_c(u), projected on <d,1>_W = 0
//   correction (Eq. 4.5):   v = u + grad_c(p) / rho on interior rows.
//
// Walls: even reflection (zero flux, Eq. 4.6-4.7) for phi, a, chemical
// potential and pressure; the wall-normal flux phi v_y is odd (it vanishes).
#include "physics.h"

namespace cahn {

// Grid constants of the explicit kernels, formed once on the host: a
// division on GB300's FP64 pipe (2 lanes per clock and SM) per thread cost
// more than the node work it served, and IEEE division rounds alike on the
// host and the device, so the values are those the kernels formed.
struct GridK {
    double ihx2, ihy2;   // 1/(2h)
    double gx, gy;       // 1/h^2
    double kx, ky;       // kappa/h^2
};
static GridK grid_k(const Grid& g, const PhysDev& P) {
    GridK k;
    k.ihx2 = 0.5 / g.hx;
    k.ihy2 = 0.5 / g.hy;
    k.gx = 1.0 / (g.hx * g.hx);
    k.gy = 1.0 / (g.hy * g.hy);
    k.kx = P.kappa / (g.hx * g.hx);
    k.ky = P.kappa / (g.hy * g.hy);
    return k;
}

__device__ __forceinline__ double f_prime(const PhysDev& P, double ph) {
    if (P.energy == 1) return 2.0 * P.gamma2 * ph * (1.0 - ph) * (1.0 - 2.0 * ph);
    return (log(ph) + 1.0) * P.inv_npoly - log(1.0 - ph) - 1.0 + P.chi * (1.0 - 2.0 * ph);
}

// a = M phi* (and its FP32 copy a32, when given), wr = 1/2 (kappa L_h + S) phi^n
// + F'(phi*) - S phi*; domain check into status.  Returns at once while *gate != 0.
__global__ void __launch_bounds__(256) k_ch_prep(Grid g, PhysDev P, GridK K, const double* __restrict__ phi,
                                                 const double* __restrict__ phi_prev,
                                                 double* __restrict__ a, float* __restrict__ a32,
                                                 double* __restrict__ wr, int* __restrict__ status,
                                                 const int* __restrict__ gate) {
    if (gate && *gate) return;
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double kx = K.kx, ky = K.ky;
    int bad = 0;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const int js = j > 0 ? j - 1 : 1, jn = j < ny ? j + 1 : ny - 1;
        const size_t e = (size_t)j * nx + i;
        const double pc = phi[e];
        const double ps = 1.5 * pc - 0.5 * phi_prev[e];
        if (P.energy == 0 ? !(ps > 0.0 && ps < 1.0) : !(ps >= 0.0)) bad = 1;
        const double av = P.mobility * ps;
        a[e] = av;
        if (a32) a32[e] = (float)av;   // the FP32 hierarchy's copy
        const double lap = kx * (2.0 * pc - phi[(size_t)j * nx + im] - phi[(size_t)j * nx + ip]) +
                           ky * (2.0 * pc - phi[(size_t)js * nx + i] - phi[(size_t)jn * nx + i]);
        const double psc = fmin(fmax(ps, 1e-300), 1.0 - 1e-16);
        wr[e] = 0.5 * (lap + P.S * pc) + f_prime(P, P.energy == 0 ? psc : ps) - P.S * ps;
    }
    if (bad) atomicOr(status, CTL_DOMAIN);
}

__device__ __forceinline__ double extrap(const double* q, const double* qp, size_t e) {
    return 1.5 * q[e] - 0.5 * qp[e];
}

// b = phi/dt - G_a wr - D_c(phi* u*, phi* v*).  fold (when given): the
// domain check of the coefficient's launch, moved into status and cleared.
__global__ void __launch_bounds__(256) k_ch_rhs(Grid g, PhysDev P, GridK K, const double* __restrict__ phi,
                                                const double* __restrict__ phi_prev,
                                                const double* __restrict__ u, const double* __restrict__ u_prev,
                                                const double* __restrict__ v, const double* __restrict__ v_prev,
                                                const double* __restrict__ a, const double* __restrict__ wr,
                                                double* __restrict__ b, int* __restrict__ fold,
                                                int* __restrict__ status) {
    if (fold && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        const int f = *fold;
        if (f) atomicOr(status, f);
        *fold = 0;
    }
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double gx = K.gx, gy = K.gy;
    const double ihx2 = K.ihx2, ihy2 = K.ihy2;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const int js = j > 0 ? j - 1 : 1, jn = j < ny ? j + 1 : ny - 1;
        const size_t e = (size_t)j * nx + i, ew = (size_t)j * nx + im, ee = (size_t)j * nx + ip;
        const size_t es = (size_t)js * nx + i, en = (size_t)jn * nx + i;
        const double ac = a[e], wc = wr[e];
        const double fxp = 0.5 * (ac + a[ee]) * (wr[ee] - wc) - 0.5 * (ac + a[ew]) * (wc - wr[ew]);
        const double fyp = 0.5 * (ac + a[en]) * (wr[en] - wc) - 0.5 * (ac + a[es]) * (wc - wr[es]);
        const double gaw = -(fxp * gx + fyp * gy);
        // advective flux divergence, F_y odd about the walls
        const double fx_e = extrap(phi, phi_prev, ee) * extrap(u, u_prev, ee);
        const double fx_w = extrap(phi, phi_prev, ew) * extrap(u, u_prev, ew);
        double fy_n, fy_s;
        if (j == 0) {
            fy_n = extrap(phi, phi_prev, en) * extrap(v, v_prev, en);
            fy_s = -fy_n;
        } else if (j == ny) {
            fy_s = extrap(phi, phi_prev, es) * extrap(v, v_prev, es);
            fy_n = -fy_s;
        } else {
            fy_n = extrap(phi, phi_prev, en) * extrap(v, v_prev, en);
            fy_s = extrap(phi, phi_prev, es) * extrap(v, v_prev, es);
        }
        const double div = (fx_e - fx_w) * ihx2 + (fy_n - fy_s) * ihy2;
        b[e] = phi[e] * P.idt - gaw - div;
    }
}

// phi += (m0 - <phi,1>_W) / <1,1>_W   (scal[S_MASS] holds <phi,1>_W)
__global__ void k_mass_fix(size_t n, double* __restrict__ phi, const double* __restrict__ scal,
                           double m0, double inv_sumw) {
    const double shift = (m0 - scal[S_MASS]) * inv_sumw;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        phi[e] += shift;
}

// Nodal intermediates of the momentum rhs: T = grad phi_h (x) grad phi_h
// (central, zero normal derivative on the walls), eta', u*, v*.
__global__ void __launch_bounds__(256) k_mom_prep(Grid g, PhysDev P, GridK K, const double* __restrict__ phi_new,
                                                  const double* __restrict__ phi,
                                                  const double* __restrict__ u, const double* __restrict__ u_prev,
                                                  const double* __restrict__ v, const double* __restrict__ v_prev,
                                                  MomWs W) {
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double ihx2 = K.ihx2, ihy2 = K.ihy2;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const size_t e = (size_t)j * nx + i;
        auto ph = [&](size_t k) { return 0.5 * (phi_new[k] + phi[k]); };
        const double gxv = (ph((size_t)j * nx + ip) - ph((size_t)j * nx + im)) * ihx2;
        double gyv = 0.0;
        if (j > 0 && j < ny) gyv = (ph((size_t)(j + 1) * nx + i) - ph((size_t)(j - 1) * nx + i)) * ihy2;
        W.txx[e] = gxv * gxv;
        W.txy[e] = gxv * gyv;
        W.tyy[e] = gyv * gyv;
        const double pc = ph(e);
        W.ep[e] = pc * P.eta_b + (1.0 - pc) * P.eta_w - P.eta_bar;
        W.us[e] = extrap(u, u_prev, e);
        W.vs[e] = extrap(v, v_prev, e);
    }
}

__global__ void __launch_bounds__(256) k_mom_rhs(Grid g, PhysDev P, GridK K, const double* __restrict__ u,
                                                 const double* __restrict__ v, MomWs W,
                                                 double* __restrict__ bu, double* __restrict__ bv) {
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double ihx2 = K.ihx2, ihy2 = K.ihy2;
    const double gx = K.gx, gy = K.gy;
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
        // capillary force -Gamma div(T)
        const double cxf = -gam * ((W.txx[ee] - W.txx[ew]) * ihx2 + (W.txy[en] - W.txy[es]) * ihy2);
        const double cyf = -gam * ((W.txy[ee] - W.txy[ew]) * ihx2 + (W.tyy[en] - W.tyy[es]) * ihy2);
        // viscous remainder
        const double epc = W.ep[e];
        const double fe = 0.5 * (epc + W.ep[ee]), fw = 0.5 * (epc + W.ep[ew]);
        const double fn = 0.5 * (epc + W.ep[en]), fs = 0.5 * (epc + W.ep[es]);
        const double usc = W.us[e], vsc = W.vs[e];
        const double us_x = (W.us[ee] - W.us[ew]) * ihx2, us_y = (W.us[en] - W.us[es]) * ihy2;
        const double vs_x = (W.vs[ee] - W.vs[ew]) * ihx2, vs_y = (W.vs[en] - W.vs[es]) * ihy2;
        const double ep_x = (W.ep[ee] - W.ep[ew]) * ihx2, ep_y = (W.ep[en] - W.ep[es]) * ihy2;
        const double visc_u = (fe * (W.us[ee] - usc) - fw * (usc - W.us[ew])) * gx +
                              (fn * (W.us[en] - usc) - fs * (usc - W.us[es])) * gy +
                              ep_x * us_x + ep_y * vs_x;
        const double visc_v = (fe * (W.vs[ee] - vsc) - fw * (vsc - W.vs[ew])) * gx +
                              (fn * (W.vs[en] - vsc) - fs * (vsc - W.vs[es])) * gy +
                              ep_x * us_y + ep_y * vs_y;
        const double conv_u = usc * us_x + vsc * us_y;
        const double conv_v = usc * vs_x + vsc * vs_y;
        const double uc = u[e], vc = v[e];
        const double lap_u = (2.0 * uc - u[ew] - u[ee]) * gx + (2.0 * uc - u[es] - u[en]) * gy;
        const double lap_v = (2.0 * vc - v[ew] - v[ee]) * gx + (2.0 * vc - v[es] - v[en]) * gy;
        bu[e] = P.rho * uc * P.idt - P.rho * conv_u - P.nu * lap_u + cxf + visc_u + P.fx;
        bv[e] = P.rho * vc * P.idt - P.rho * conv_v - P.nu * lap_v + cyf + visc_v;
    }
}

// d = rho D_c(u, v), v odd about the walls
__global__ void __launch_bounds__(256) k_div(Grid g, GridK K, double rho, const double* __restrict__ u,
                                             const double* __restrict__ v, double* __restrict__ d) {
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double ihx2 = K.ihx2, ihy2 = K.ihy2;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const size_t e = (size_t)j * nx + i;
        double vn, vs;
        if (j == 0) {
            vn = v[(size_t)1 * nx + i];
            vs = -vn;
        } else if (j == ny) {
            vs = v[(size_t)(ny - 1) * nx + i];
            vn = -vs;
        } else {
            vn = v[(size_t)(j + 1) * nx + i];
            vs = v[(size_t)(j - 1) * nx + i];
        }
        d[e] = rho * ((u[(size_t)j * nx + ip] - u[(size_t)j * nx + im]) * ihx2 + (vn - vs) * ihy2);
    }
}

// interior rows: u += p_x / rho, v += p_y / rho
__global__ void __launch_bounds__(256) k_correct(Grid g, GridK K, double inv_rho, const double* __restrict__ p,
                                                 double* __restrict__ u, double* __restrict__ v) {
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double ihx2 = K.ihx2, ihy2 = K.ihy2;
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        if (j == 0 || j == ny) continue;
        const size_t e = (size_t)j * nx + i;
        u[e] += inv_rho * (p[(size_t)j * nx + ip] - p[(size_t)j * nx + im]) * ihx2;
        v[e] += inv_rho * (p[(size_t)(j + 1) * nx + i] - p[(size_t)(j - 1) * nx + i]) * ihy2;
    }
}

// ---------------------------------------------------------------- launch
static dim3 tg(const Grid& g) { return tile_grid(g.nx, g.ny); }
static const dim3 TB(32, 8);

void launch_ch_prep(const Grid& g, const PhysDev& P, const double* phi, const double* phi_prev,
                    double* a, float* a32, double* wr, int* status, const int* gate,
                    cudaStream_t s) {
    note_launch(); launch_k(k_ch_prep, tg(g), TB, 0, s, g, P, grid_k(g, P), phi, phi_prev, a, a32, wr, status, gate);
}
void launch_ch_rhs(const Grid& g, const PhysDev& P, const double* phi, const double* phi_prev,
                   const double* u, const double* u_prev, const double* v, const double* v_prev,
                   const double* a, const double* wr, double* b, int* fold, int* status, cudaStream_t s) {
    note_launch(); launch_k(k_ch_rhs, tg(g), TB, 0, s, g, P, grid_k(g, P), phi, phi_prev, u, u_prev, v, v_prev, a, wr, b, fold, status);
}
void launch_mass_fix(size_t n, double* phi, const double* scal, double m0, double inv_sumw,
                     cudaStream_t s) {
    note_launch(); launch_k(k_mass_fix, vec_blocks(n), RED_THREADS, 0, s, n, phi, scal, m0, inv_sumw);
}
void launch_mom_prep(const Grid& g, const PhysDev& P, const double* phi_new, const double* phi,
                     const double* u, const double* u_prev, const double* v, const double* v_prev,
                     const MomWs& W, cudaStream_t s) {
    note_launch(); launch_k(k_mom_prep, tg(g), TB, 0, s, g, P, grid_k(g, P), phi_new, phi, u, u_prev, v, v_prev, W);
}
void launch_mom_rhs(const Grid& g, const PhysDev& P, const double* u, const double* v,
                    const MomWs& W, double* bu, double* bv, cudaStream_t s) {
    note_launch(); launch_k(k_mom_rhs, tg(g), TB, 0, s, g, P, grid_k(g, P), u, v, W, bu, bv);
}
void launch_div(const Grid& g, double rho, const double* u, const double* v, double* d,
                cudaStream_t s) {
    note_launch(); launch_k(k_div, tg(g), TB, 0, s, g, grid_k(g, PhysDev{}), rho, u, v, d);
}
void launch_correct(const Grid& g, double inv_rho, const double* p, double* u, double* v,
                    cudaStream_t s) {
    note_launch(); launch_k(k_correct, tg(g), TB, 0, s, g, grid_k(g, PhysDev{}), inv_rho, p, u, v);
}

}  // namespace cahn
