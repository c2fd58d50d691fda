// Explicit parts of the nutrient transport (Eq. 2.6-2.7) and of the network
// production g_n (Eq. 2.5), FP64.
//
//   phi_s = 1 - phi, phi^{n+1/2} = (phi^{n+1} + phi^n)/2, q* = (3 q^n - q^{n-1})/2
//   K c = dg c + 1/2 G_k c, with
//     dg = phi_s^{n+1}/dt + A/2 phi^{n+1/2},  k = D_s phi_s^{n+1/2}
//     G_k c = -div_h(k grad_h c), face values means of the two nodes,
//     zero total flux on both walls (c and k evenly reflected)
//   b = (phi_s^n/dt - A/2 phi^{n+1/2}) c^n - 1/2 G_k c^n - D_c(c* phi_s* v*)
//     (the wall-normal advective flux odd about the walls)
//   with c = c_bulk on the top wall (N.dtop): K c = c/dt and b = c_bulk/dt on
//     row ny, whose value row ny-1 takes as its neighbour
//   g_n = eps mu phi* max(c*, 0) / (K_c + max(c*, 0))
//
// The operator stores a = k/4 (the face weight of 1/2 G_k is a_c + a_f), so
// the prep kernel forms a at the centre and the four neighbours from phi.
#include "nutrient.h"

namespace cahn {

__device__ __forceinline__ double extrap_n(const double* q, const double* qp, size_t e) {
    return 1.5 * q[e] - 0.5 * qp[e];
}

__global__ void __launch_bounds__(256) k_nut_prep(
    Grid g, NutDev N, const double* __restrict__ phi_new, const double* __restrict__ phi,
    const double* __restrict__ phi_prev, const double* __restrict__ c,
    const double* __restrict__ c_prev, const double* __restrict__ u,
    const double* __restrict__ u_prev, const double* __restrict__ v,
    const double* __restrict__ v_prev, double* __restrict__ a, double* __restrict__ dg,
    double* __restrict__ dinv, double* __restrict__ b, double* __restrict__ x0,
    float* __restrict__ a32, float* __restrict__ dg32, float* __restrict__ dinv32,
    int* __restrict__ status) {
    const int nx = g.nx, ny = g.ny;
    const int i = blockIdx.x * TILE_X + threadIdx.x;
    if (i >= nx) return;
    bool bad = false;
    const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
    const double gx = 1.0 / (g.hx * g.hx), gy = 1.0 / (g.hy * g.hy);
    const double ihx2 = 0.5 / g.hx, ihy2 = 0.5 / g.hy;
    const double qd = 0.25 * N.diff_s;
    auto half = [&](size_t k) { return 0.5 * (phi_new[k] + phi[k]); };
    auto acoef = [&](size_t k) { return qd * (1.0 - half(k)); };
    for (int r = 0; r < TILE_Y / 8; ++r) {
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;
        if (j > ny) break;
        const size_t e = (size_t)j * nx + i;
        const double ac = acoef(e);
        bad |= !(1.0 - phi_new[e] > 0.0) || !(ac >= 0.0);
        double d, di;
        if (N.dtop && j == ny) {
            d = N.idt;
            di = N.dt;
            if (b) {
                b[e] = N.c_bulk * N.idt;
                x0[e] = N.c_bulk;
            }
        } else {
            const int js = j > 0 ? j - 1 : 1, jn = j < ny ? j + 1 : ny - 1;
            const size_t ew = (size_t)j * nx + im, ee = (size_t)j * nx + ip;
            const size_t es = (size_t)js * nx + i, en = (size_t)jn * nx + i;
            const double ph = half(e);
            d = (1.0 - phi_new[e]) * N.idt + 0.5 * N.consume_a * ph;
            const double ce = ac + acoef(ee), cw = ac + acoef(ew);
            const double cn = ac + acoef(en), cs = ac + acoef(es);
            di = 1.0 / (d + gx * (ce + cw) + gy * (cn + cs));
            if (b) {
                const double cc = c[e];
                const double gk = gx * (ce * (cc - c[ee]) + cw * (cc - c[ew])) +
                                  gy * (cn * (cc - c[en]) + cs * (cc - c[es]));
                // advective flux F = c* phi_s* v*, F_y odd about the walls
                auto flux = [&](size_t k, const double* w, const double* wp) {
                    return extrap_n(c, c_prev, k) * (1.0 - extrap_n(phi, phi_prev, k)) *
                           extrap_n(w, wp, k);
                };
                double fy_n, fy_s;
                if (j == 0) {
                    fy_n = flux(en, v, v_prev);
                    fy_s = -fy_n;
                } else if (j == ny) {
                    fy_s = flux(es, v, v_prev);
                    fy_n = -fy_s;
                } else {
                    fy_n = flux(en, v, v_prev);
                    fy_s = flux(es, v, v_prev);
                }
                const double div = (flux(ee, u, u_prev) - flux(ew, u, u_prev)) * ihx2 +
                                   (fy_n - fy_s) * ihy2;
                b[e] = ((1.0 - phi[e]) * N.idt - 0.5 * N.consume_a * ph) * cc - gk - div;
                x0[e] = cc;
            }
        }
        a[e] = ac;
        dg[e] = d;
        dinv[e] = di;
        if (a32) {
            a32[e] = (float)ac;
            dg32[e] = (float)d;
            dinv32[e] = (float)di;
        }
    }
    if (bad && status) atomicOr(status, CTL_DOMAIN);
}

__global__ void __launch_bounds__(256) k_growth(Grid g, NutDev N, const double* __restrict__ phi,
                                                const double* __restrict__ phi_prev,
                                                const double* __restrict__ c,
                                                const double* __restrict__ c_prev,
                                                double* __restrict__ b, double* __restrict__ gr) {
    const size_t n = g.n();
    const double k = N.eps_g * N.mu;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x) {
        const double cs = fmax(extrap_n(c, c_prev, e), 0.0);
        const double gn = k * extrap_n(phi, phi_prev, e) * cs / (N.kc + cs);
        gr[e] = gn;
        b[e] += gn;
    }
}

__global__ void k_mass_fix_grow(size_t n, double* __restrict__ phi, double* __restrict__ scal,
                                const double* __restrict__ m, double inv_sumw) {
    const double target = m[0] + scal[S_TMP1];
    const double shift = (target - scal[S_MASS]) * inv_sumw;
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_TMP0] = target;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        phi[e] += shift;
}

__global__ void k_nut_top(int nx, size_t off, double* __restrict__ x,
                          const double* __restrict__ b, double dt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x)
        x[off + i] = b[off + i] * dt;
}

void launch_nut_prep(const Grid& g, const NutDev& N, const double* phi_new, const double* phi,
                     const double* phi_prev, const double* c, const double* c_prev,
                     const double* u, const double* u_prev, const double* v,
                     const double* v_prev, double* a, double* dg, double* dinv, double* b,
                     double* x0, float* a32, float* dg32, float* dinv32, int* status,
                     cudaStream_t s) {
    note_launch();
    launch_k(k_nut_prep, tile_grid(g.nx, g.ny), dim3(32, 8), 0, s, g, N, phi_new, phi, phi_prev,
             c, c_prev, u, u_prev, v, v_prev, a, dg, dinv, b, x0, a32, dg32, dinv32, status);
}

void launch_growth(const Grid& g, const NutDev& N, const double* phi, const double* phi_prev,
                   const double* c, const double* c_prev, double* b, double* gr,
                   cudaStream_t s) {
    note_launch();
    launch_k(k_growth, vec_blocks(g.n()), RED_THREADS, 0, s, g, N, phi, phi_prev, c, c_prev, b, gr);
}

void launch_mass_fix_grow(size_t n, double* phi, double* scal, const double* m,
                          double inv_sumw, cudaStream_t s) {
    note_launch();
    launch_k(k_mass_fix_grow, vec_blocks(n), RED_THREADS, 0, s, n, phi, scal, m, inv_sumw);
}

void launch_nut_top(const Grid& g, double* x, const double* b, double dt, cudaStream_t s) {
    note_launch();
    launch_k(k_nut_top, vec_blocks((size_t)g.nx), RED_THREADS, 0, s, g.nx, (size_t)g.ny * g.nx, x,
             b, dt);
}

}  // namespace cahn
