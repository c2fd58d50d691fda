// Discrete adjoint of one time step (FP64): the exact reverse of every
// operation of the step in physics.cu / api.cu, in the Euclidean inner
// product of the flattened fields.  The three linear solves are reversed
// with transposed solves (A_phi^T through its W-adjoint, H on the interior,
// the projected pressure map through W S W^-1); the explicit parts are
// gathered node by node (each transpose written as the sum of the
// contributions a node received in the forward pass).
#include "adjoint.h"

namespace cahn {

namespace {

struct Nb {   // neighbour indices of node (i, j) with even reflection in y
    int i, j, im, ip, js, jn;
};

__device__ __forceinline__ Nb nb_of(const Grid& g, int i, int j) {
    Nb n;
    n.i = i;
    n.j = j;
    n.im = i > 0 ? i - 1 : g.nx - 1;
    n.ip = i < g.nx - 1 ? i + 1 : 0;
    n.js = j > 0 ? j - 1 : 1;
    n.jn = j < g.ny ? j + 1 : g.ny - 1;
    return n;
}

__device__ __forceinline__ double at(const double* f, const Grid& g, int i, int j) {
    return f[(size_t)j * g.nx + i];
}
__device__ __forceinline__ int wx(const Grid& g, int i) {
    return i < 0 ? i + g.nx : (i >= g.nx ? i - g.nx : i);
}
__device__ __forceinline__ double wgt_row(const Grid& g, int j) {
    return (j == 0 || j == g.ny) ? 0.5 : 1.0;
}
__device__ __forceinline__ bool interior(const Grid& g, int j) { return j >= 1 && j <= g.ny - 1; }

// transposes at node (i, j) of a field given by a functor F(i, j)
template <typename F>
__device__ __forceinline__ double dxcT(F f, const Grid& g, int i, int j) {
    return (f(wx(g, i - 1), j) - f(wx(g, i + 1), j)) / (2.0 * g.hx);
}
template <typename F>
__device__ __forceinline__ double dycT(F f, const Grid& g, int i, int j) {
    const double lo = (j - 1 >= 1 && j - 1 <= g.ny - 1) ? f(i, j - 1) : 0.0;
    const double hi = (j + 1 >= 1 && j + 1 <= g.ny - 1) ? f(i, j + 1) : 0.0;
    return (lo - hi) / (2.0 * g.hy);
}
template <typename F>
__device__ __forceinline__ double dyoddT(F f, const Grid& g, int i, int j) {
    double v = 0.0;
    if (j >= 2) v += f(i, j - 1) / (2.0 * g.hy);
    if (j <= g.ny - 2) v -= f(i, j + 1) / (2.0 * g.hy);
    if (j == 1) v += f(i, 0) / g.hy;
    if (j == g.ny - 1) v -= f(i, g.ny) / g.hy;
    return v;
}
// G_a x at (i, j) with even reflection (x, a given as functors)
template <typename FA, typename FX>
__device__ __forceinline__ double ga_at(FA a, FX x, const Grid& g, int i, int j) {
    const Nb n = nb_of(g, i, j);
    const double ac = a(i, j), xc = x(i, j);
    const double fx = 0.5 * (ac + a(n.ip, j)) * (x(n.ip, j) - xc) - 0.5 * (ac + a(n.im, j)) * (xc - x(n.im, j));
    const double fy = 0.5 * (ac + a(i, n.jn)) * (x(i, n.jn) - xc) - 0.5 * (ac + a(i, n.js)) * (xc - x(i, n.js));
    return -(fx / (g.hx * g.hx) + fy / (g.hy * g.hy));
}
// L_h x at (i, j) (Neumann)
template <typename FX>
__device__ __forceinline__ double lap_at(FX x, const Grid& g, int i, int j) {
    const Nb n = nb_of(g, i, j);
    const double c = x(i, j);
    return (2.0 * c - x(n.im, j) - x(n.ip, j)) / (g.hx * g.hx) +
           (2.0 * c - x(i, n.js) - x(i, n.jn)) / (g.hy * g.hy);
}

// Transpose of a -> G_a z at node k = (i, j) applied to lam (see the face
// bookkeeping: the four face coefficients of each node, each the mean of
// two nodes, with the reflected ghost at the walls).
template <typename FZ, typename FL>
__device__ double gacoefT(FZ z, FL lam, const Grid& g, int i, int j) {
    const double hx2 = g.hx * g.hx, hy2 = g.hy * g.hy;
    auto dze = [&](int ii, int jj) { return z(wx(g, ii + 1), jj) - z(ii, jj); };
    auto dzw = [&](int ii, int jj) { return z(ii, jj) - z(wx(g, ii - 1), jj); };
    auto dzn = [&](int ii, int jj) {
        const int jn = jj < g.ny ? jj + 1 : g.ny - 1;
        return z(ii, jn) - z(ii, jj);
    };
    auto dzs = [&](int ii, int jj) {
        const int js = jj > 0 ? jj - 1 : 1;
        return z(ii, jj) - z(ii, js);
    };
    auto ae_b = [&](int ii, int jj) { return -lam(ii, jj) * dze(ii, jj) / hx2; };
    auto aw_b = [&](int ii, int jj) { return lam(ii, jj) * dzw(ii, jj) / hx2; };
    auto an_b = [&](int ii, int jj) { return -lam(ii, jj) * dzn(ii, jj) / hy2; };
    auto as_b = [&](int ii, int jj) { return lam(ii, jj) * dzs(ii, jj) / hy2; };
    double v = 0.5 * (ae_b(i, j) + ae_b(wx(g, i - 1), j)) + 0.5 * (aw_b(i, j) + aw_b(wx(g, i + 1), j));
    double nt = an_b(i, j);
    if (j >= 1) nt += an_b(i, j - 1);
    if (j == g.ny - 1) nt += an_b(i, g.ny);
    double st = as_b(i, j);
    if (j <= g.ny - 1) st += as_b(i, j + 1);
    if (j == 1) st += as_b(i, 0);
    return v + 0.5 * nt + 0.5 * st;
}

// (c_bar, f_bar) of dxx_face(c, f) and dyy_face(c, f) against lam, at node k
template <typename FC, typename FF, typename FL>
__device__ void dxxT(FC c, FF f, FL lam, const Grid& g, int i, int j, double& cb, double& fb) {
    const double hx2 = g.hx * g.hx;
    const int im = wx(g, i - 1), ip = wx(g, i + 1);
    auto t = [&](int ii) { return lam(ii, j) / hx2; };
    auto ce = [&](int ii) { return 0.5 * (c(ii, j) + c(wx(g, ii + 1), j)); };
    auto cw = [&](int ii) { return 0.5 * (c(ii, j) + c(wx(g, ii - 1), j)); };
    // f_b = xp_T(ce t) - ce t - cw t + xm_T(cw t)
    fb = ce(im) * t(im) - ce(i) * t(i) - cw(i) * t(i) + cw(ip) * t(ip);
    auto ce_b = [&](int ii) { return t(ii) * (f(wx(g, ii + 1), j) - f(ii, j)); };
    auto cw_b = [&](int ii) { return -t(ii) * (f(ii, j) - f(wx(g, ii - 1), j)); };
    cb = 0.5 * (ce_b(i) + ce_b(im)) + 0.5 * (cw_b(i) + cw_b(ip));
}
template <typename FC, typename FF, typename FL>
__device__ void dyyT(FC c, FF f, FL lam, const Grid& g, int i, int j, double& cb, double& fb) {
    // rows r = 1..ny-1 carry t_r = lam_r / hy^2; cn_r = (c_r + c_{r+1})/2, cs_r = (c_r + c_{r-1})/2
    const double hy2 = g.hy * g.hy;
    auto in = [&](int r) { return r >= 1 && r <= g.ny - 1; };
    auto t = [&](int r) { return lam(i, r) / hy2; };
    auto cn = [&](int r) { return 0.5 * (c(i, r) + c(i, r + 1)); };
    auto cs = [&](int r) { return 0.5 * (c(i, r) + c(i, r - 1)); };
    fb = 0.0;
    if (in(j - 1)) fb += cn(j - 1) * t(j - 1);
    if (in(j)) fb -= (cn(j) + cs(j)) * t(j);
    if (in(j + 1)) fb += cs(j + 1) * t(j + 1);
    auto cn_b = [&](int r) { return t(r) * (f(i, r + 1) - f(i, r)); };
    auto cs_b = [&](int r) { return -t(r) * (f(i, r) - f(i, r - 1)); };
    cb = 0.0;
    if (in(j)) cb += 0.5 * (cn_b(j) + cs_b(j));
    if (in(j - 1)) cb += 0.5 * cn_b(j - 1);
    if (in(j + 1)) cb += 0.5 * cs_b(j + 1);
}

__device__ __forceinline__ double fpp(const PhysDev& P, double ph) {
    if (P.energy == 1) return 2.0 * P.gamma2 * (1.0 - 6.0 * ph + 6.0 * ph * ph);
    return 1.0 / (P.n_poly * ph) + 1.0 / (1.0 - ph) - 2.0 * P.chi;
}
#define ADJ_LOOP                                                           \
    const int i = blockIdx.x * TILE_X + threadIdx.x;                       \
    for (int r = 0; r < TILE_Y / 8; ++r) {                                 \
        const int j = blockIdx.y * TILE_Y + threadIdx.y + 8 * r;           \
        if (i >= g.nx || j > g.ny) continue;                               \
        const size_t e = (size_t)j * g.nx + i;

#define ADJ_END }

}  // namespace

// 1. correction: p_bar = Dx^T(u_bar_int / rho) + Dy^T(v_bar_int / rho)
__global__ void k_adj_correct(Grid g, double inv_rho, const double* __restrict__ ub,
                              const double* __restrict__ vb, double* __restrict__ pb) {
    auto pu = [&](int ii, int jj) { return interior(g, jj) ? at(ub, g, ii, jj) * inv_rho : 0.0; };
    auto pv = [&](int ii, int jj) { return interior(g, jj) ? at(vb, g, ii, jj) * inv_rho : 0.0; };
    ADJ_LOOP
    pb[e] = dxcT(pu, g, i, j) + dycT(pv, g, i, j);
    ADJ_END
}

// q = p_bar / w  (the pressure map is W-self-adjoint: S^T = W S W^-1)
__global__ void k_adj_div_w(Grid g, const double* __restrict__ pb, double* __restrict__ q) {
    ADJ_LOOP
    q[e] = pb[e] / wgt_row(g, j);
    ADJ_END
}

// 3. d_bar = w x; u_bar += rho Dx^T d_bar; v_bar += rho DyOdd^T d_bar
__global__ void k_adj_div(Grid g, double rho, const double* __restrict__ x,
                          double* __restrict__ utb, double* __restrict__ vtb) {
    auto db = [&](int ii, int jj) { return wgt_row(g, jj) * at(x, g, ii, jj); };
    ADJ_LOOP
    utb[e] += rho * dxcT(db, g, i, j);
    vtb[e] += rho * dyoddT(db, g, i, j);
    ADJ_END
}

// zero the wall rows (the predictor's wall rows are constants)
__global__ void k_adj_zero_walls(Grid g, double* __restrict__ f) {
    ADJ_LOOP
    if (!interior(g, j)) f[e] = 0.0;
    ADJ_END
}

// 5a. momentum adjoint, pass A: nodal gx_bar, gy_bar, ex_bar, ey_bar
__global__ void k_adj_mom_a(Grid g, PhysDev P, AdjFields A, const double* __restrict__ bub,
                            const double* __restrict__ bvb) {
    const double* phn = A.phi_new;
    const double* phc = A.phi;
    auto ph = [&](int ii, int jj) { return 0.5 * (at(phn, g, ii, jj) + at(phc, g, ii, jj)); };
    auto us = [&](int ii, int jj) { return 1.5 * at(A.u, g, ii, jj) - 0.5 * at(A.u_prev, g, ii, jj); };
    auto vs = [&](int ii, int jj) { return 1.5 * at(A.v, g, ii, jj) - 0.5 * at(A.v_prev, g, ii, jj); };
    auto lbu = [&](int ii, int jj) { return interior(g, jj) ? at(bub, g, ii, jj) : 0.0; };
    auto lbv = [&](int ii, int jj) { return interior(g, jj) ? at(bvb, g, ii, jj) : 0.0; };
    const double gam = P.gamma_cap;
    ADJ_LOOP
    const double t1 = -gam * dxcT(lbu, g, i, j), t2 = -gam * dycT(lbu, g, i, j);
    const double t3 = -gam * dxcT(lbv, g, i, j), t4 = -gam * dycT(lbv, g, i, j);
    const double gxv = (ph(wx(g, i + 1), j) - ph(wx(g, i - 1), j)) / (2.0 * g.hx);
    const double gyv = interior(g, j) ? (ph(i, j + 1) - ph(i, j - 1)) / (2.0 * g.hy) : 0.0;
    A.gxb[e] = 2.0 * gxv * t1 + gyv * t2 + gyv * t3;
    A.gyb[e] = gxv * t2 + gxv * t3 + 2.0 * gyv * t4;
    const double bu = lbu(i, j), bv = lbv(i, j);
    const double usx = (us(wx(g, i + 1), j) - us(wx(g, i - 1), j)) / (2.0 * g.hx);
    const double usy = interior(g, j) ? (us(i, j + 1) - us(i, j - 1)) / (2.0 * g.hy) : 0.0;
    const double vsx = (vs(wx(g, i + 1), j) - vs(wx(g, i - 1), j)) / (2.0 * g.hx);
    const double vsy = interior(g, j) ? (vs(i, j + 1) - vs(i, j - 1)) / (2.0 * g.hy) : 0.0;
    A.exb[e] = bu * usx + bv * usy;
    A.eyb[e] = bu * vsx + bv * vsy;
    ADJ_END
}

// 5b. momentum adjoint, pass B: ph_bar, us_bar, vs_bar; u^n, v^n bars
__global__ void k_adj_mom_b(Grid g, PhysDev P, AdjFields A, const double* __restrict__ bub,
                            const double* __restrict__ bvb, double* __restrict__ Un,
                            double* __restrict__ Vn) {
    const double* phn = A.phi_new;
    const double* phc = A.phi;
    auto ph = [&](int ii, int jj) { return 0.5 * (at(phn, g, ii, jj) + at(phc, g, ii, jj)); };
    auto ep = [&](int ii, int jj) {
        const double p = ph(ii, jj);
        return p * P.eta_b + (1.0 - p) * P.eta_w - P.eta_bar;
    };
    auto us = [&](int ii, int jj) { return 1.5 * at(A.u, g, ii, jj) - 0.5 * at(A.u_prev, g, ii, jj); };
    auto vs = [&](int ii, int jj) { return 1.5 * at(A.v, g, ii, jj) - 0.5 * at(A.v_prev, g, ii, jj); };
    auto lbu = [&](int ii, int jj) { return interior(g, jj) ? at(bub, g, ii, jj) : 0.0; };
    auto lbv = [&](int ii, int jj) { return interior(g, jj) ? at(bvb, g, ii, jj) : 0.0; };
    auto ex = [&](int ii, int jj) { return (ep(wx(g, ii + 1), jj) - ep(wx(g, ii - 1), jj)) / (2.0 * g.hx); };
    auto ey = [&](int ii, int jj) {
        return interior(g, jj) ? (ep(ii, jj + 1) - ep(ii, jj - 1)) / (2.0 * g.hy) : 0.0;
    };
    auto fgx = [&](int ii, int jj) { return at(A.gxb, g, ii, jj); };
    auto fgy = [&](int ii, int jj) { return at(A.gyb, g, ii, jj); };
    auto fexb = [&](int ii, int jj) { return at(A.exb, g, ii, jj); };
    auto feyb = [&](int ii, int jj) { return at(A.eyb, g, ii, jj); };
    const double rho = P.rho, nu = P.nu;
    ADJ_LOOP
    const double bu = lbu(i, j), bv = lbv(i, j);
    const double cu = -rho * bu, cv = -rho * bv;
    auto us_cu = [&](int ii, int jj) { return us(ii, jj) * -rho * lbu(ii, jj); };
    auto vs_cu = [&](int ii, int jj) { return vs(ii, jj) * -rho * lbu(ii, jj); };
    auto us_cv = [&](int ii, int jj) { return us(ii, jj) * -rho * lbv(ii, jj); };
    auto vs_cv = [&](int ii, int jj) { return vs(ii, jj) * -rho * lbv(ii, jj); };
    auto ex_bu = [&](int ii, int jj) { return ex(ii, jj) * lbu(ii, jj); };
    auto ex_bv = [&](int ii, int jj) { return ex(ii, jj) * lbv(ii, jj); };
    auto ey_bu = [&](int ii, int jj) { return ey(ii, jj) * lbu(ii, jj); };
    auto ey_bv = [&](int ii, int jj) { return ey(ii, jj) * lbv(ii, jj); };
    const double usx = (us(wx(g, i + 1), j) - us(wx(g, i - 1), j)) / (2.0 * g.hx);
    const double usy = interior(g, j) ? (us(i, j + 1) - us(i, j - 1)) / (2.0 * g.hy) : 0.0;
    const double vsx = (vs(wx(g, i + 1), j) - vs(wx(g, i - 1), j)) / (2.0 * g.hx);
    const double vsy = interior(g, j) ? (vs(i, j + 1) - vs(i, j - 1)) / (2.0 * g.hy) : 0.0;
    double usb = cu * usx + dxcT(us_cu, g, i, j) + dycT(vs_cu, g, i, j) + cv * vsx;
    double vsb = cu * usy + dxcT(us_cv, g, i, j) + cv * vsy + dycT(vs_cv, g, i, j);
    double epb = 0.0, cb, fb;
    dxxT(ep, us, lbu, g, i, j, cb, fb);
    epb += cb;
    usb += fb;
    dyyT(ep, us, lbu, g, i, j, cb, fb);
    epb += cb;
    usb += fb;
    usb += dxcT(ex_bu, g, i, j);
    vsb += dxcT(ey_bu, g, i, j);
    dxxT(ep, vs, lbv, g, i, j, cb, fb);
    epb += cb;
    vsb += fb;
    dyyT(ep, vs, lbv, g, i, j, cb, fb);
    epb += cb;
    vsb += fb;
    usb += dycT(ex_bv, g, i, j);
    vsb += dycT(ey_bv, g, i, j);
    epb += dxcT(fexb, g, i, j) + dycT(feyb, g, i, j);
    A.phb[e] = dxcT(fgx, g, i, j) + dycT(fgy, g, i, j) + (P.eta_b - P.eta_w) * epb;
    A.usb[e] = usb;
    A.vsb[e] = vsb;
    // rho u/dt - nu lap_int(u): transpose on the interior-row bars
    auto lapintT = [&](auto lam) {
        double v = 0.0;
        if (interior(g, j))
            v += (2.0 * lam(i, j) - lam(wx(g, i - 1), j) - lam(wx(g, i + 1), j)) / (g.hx * g.hx) +
                 2.0 * lam(i, j) / (g.hy * g.hy);
        if (interior(g, j + 1)) v -= lam(i, j + 1) / (g.hy * g.hy);
        if (interior(g, j - 1)) v -= lam(i, j - 1) / (g.hy * g.hy);
        return v;
    };
    Un[e] += rho * P.idt * bu - nu * lapintT(lbu);
    Vn[e] += rho * P.idt * bv - nu * lapintT(lbv);
    ADJ_END
}

// 7a. T = phi_bar^{n+1} + ph_bar / 2 (kept in Pn1); Pn += ph_bar / 2; sum(T)
__global__ void k_adj_mass_a(Grid g, double* __restrict__ Pn1, double* __restrict__ Pn,
                             const double* __restrict__ phb, SolveDev sd) {
    __shared__ double sh[32];
    double acc = 0.0;
    ADJ_LOOP
    const double h = 0.5 * phb[e];
    Pn1[e] += h;
    Pn[e] += h;
    acc += Pn1[e];
    ADJ_END
    publish_partial(sd.red, 0, block_sum(acc, sh));
    if (!last_block(sd.red)) return;
    const double t = final_sum(sd.red, 0, sh);
    if (flat_tid() == 0) {
        sd.scal[S_TMP0] = t;
        reset_counter(sd.red);
    }
}

// 7b. phit_bar = T - w s, s = sum(T) / sum(w); accumulate m0_bar += s; rhs
// of the W-adjoint CH solve: phit_bar / w
__global__ void k_adj_mass_b(Grid g, const double* __restrict__ Pn1, double* __restrict__ rhs,
                             const double* __restrict__ scal, double inv_sumw,
                             double* __restrict__ acc3) {
    const double s = scal[S_TMP0] * inv_sumw;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) acc3[2] += s;
    ADJ_LOOP
    const double w = wgt_row(g, j);
    rhs[e] = (Pn1[e] - w * s) / w;
    ADJ_END
}

// x *= w (the trapezoid weight of each row)
__global__ void k_adj_mul_w(Grid g, double* __restrict__ x) {
    ADJ_LOOP
    x[e] *= wgt_row(g, j);
    ADJ_END
}

// the mass-correction constant of a step: c = (m0 - <phit, 1>_W) / sum(w)
__global__ void k_adj_save_c(const double* __restrict__ scal, double m0, double inv_sumw,
                             double* __restrict__ c) {
    *c = (m0 - scal[S_MASS]) * inv_sumw;
}

// 9a. w_bar = -W G_a (b_bar / w); psit = kappa L phit + S phit (phit = phi_new - c)
__global__ void k_adj_ch1(Grid g, PhysDev P, AdjFields A, const double* __restrict__ bb,
                          const double* __restrict__ a, const double* __restrict__ mass_c) {
    auto fa = [&](int ii, int jj) { return at(a, g, ii, jj); };
    auto fbw = [&](int ii, int jj) { return at(bb, g, ii, jj) / wgt_row(g, jj); };
    auto phn = [&](int ii, int jj) { return at(A.phi_new, g, ii, jj); };
    const double c = *mass_c;
    ADJ_LOOP
    A.wb[e] = -wgt_row(g, j) * ga_at(fa, fbw, g, i, j);
    A.psit[e] = P.kappa * lap_at(phn, g, i, j) + P.S * (phn(i, j) - c);
    ADJ_END
}

// 9b. a_bar, phi*_bar, the bars of phi^n, phi^{n-1}, u, v levels; chi_bar, M_bar
__global__ void k_adj_ch2(Grid g, PhysDev P, AdjFields A, const double* __restrict__ bb,
                          const double* __restrict__ a, double* __restrict__ Pn,
                          double* __restrict__ Pm, double* __restrict__ Un,
                          double* __restrict__ Um, double* __restrict__ Vn,
                          double* __restrict__ Vm, SolveDev sd, double* __restrict__ acc3) {
    __shared__ double sh[32];
    auto fb = [&](int ii, int jj) { return at(bb, g, ii, jj); };
    auto fpsit = [&](int ii, int jj) { return at(A.psit, g, ii, jj); };
    auto fwf = [&](int ii, int jj) { return at(A.wf, g, ii, jj); };
    auto fwbw = [&](int ii, int jj) { return at(A.wb, g, ii, jj) / wgt_row(g, jj); };
    double chi_acc = 0.0, mob_acc = 0.0;
    ADJ_LOOP
    const double ab = -0.5 * gacoefT(fpsit, fb, g, i, j) - gacoefT(fwf, fb, g, i, j);
    const double fxb = -dxcT(fb, g, i, j);
    const double fyb = -dyoddT(fb, g, i, j);
    const double ps = 1.5 * A.phi[e] - 0.5 * A.phi_prev[e];
    const double us = 1.5 * A.u[e] - 0.5 * A.u_prev[e];
    const double vs = 1.5 * A.v[e] - 0.5 * A.v_prev[e];
    const double wbv = A.wb[e];
    const double psb = us * fxb + vs * fyb + (fpp(P, ps) - P.S) * wbv + P.mobility * ab;
    const double lapT = wgt_row(g, j) * lap_at(fwbw, g, i, j);
    const double phib = bb[e] * P.idt + 0.5 * (P.kappa * lapT + P.S * wbv);
    const double usb = A.usb[e] + ps * fxb;
    const double vsb = A.vsb[e] + ps * fyb;
    Pn[e] += phib + 1.5 * psb;
    Pm[e] += -0.5 * psb;
    Un[e] += 1.5 * usb;
    Um[e] += -0.5 * usb;
    Vn[e] += 1.5 * vsb;
    Vm[e] += -0.5 * vsb;
    chi_acc += (P.energy == 1 ? 0.0 : (1.0 - 2.0 * ps)) * wbv;
    mob_acc += ps * ab;
    ADJ_END
    publish_partial(sd.red, 0, block_sum(chi_acc, sh));
    publish_partial(sd.red, 1, block_sum(mob_acc, sh));
    if (!last_block(sd.red)) return;
    const double tc = final_sum(sd.red, 0, sh);
    const double tm = final_sum(sd.red, 1, sh);
    if (flat_tid() == 0) {
        acc3[0] += tc;
        acc3[1] += tm;
        reset_counter(sd.red);
    }
}

// phi0_bar = P0 + P_{-1} + w m0_bar
__global__ void k_adj_final(Grid g, const double* __restrict__ P0, const double* __restrict__ Pm1,
                            const double* __restrict__ acc3, double* __restrict__ out) {
    const double m0b = acc3[2];
    ADJ_LOOP
    out[e] = P0[e] + Pm1[e] + wgt_row(g, j) * m0b;
    ADJ_END
}

// ---------------------------------------------------------------- launch
static dim3 tg(const Grid& g) { return tile_grid(g.nx, g.ny); }
static const dim3 TB(32, 8);

void launch_adj_correct(const Grid& g, double inv_rho, const double* ub, const double* vb,
                        double* pb, cudaStream_t s) {
    note_launch(); launch_k(k_adj_correct, tg(g), TB, 0, s, g, inv_rho, ub, vb, pb);
}
void launch_adj_div_w(const Grid& g, const double* pb, double* q, cudaStream_t s) {
    note_launch(); launch_k(k_adj_div_w, tg(g), TB, 0, s, g, pb, q);
}
void launch_adj_div(const Grid& g, double rho, const double* x, double* utb, double* vtb,
                    cudaStream_t s) {
    note_launch(); launch_k(k_adj_div, tg(g), TB, 0, s, g, rho, x, utb, vtb);
}
void launch_adj_zero_walls(const Grid& g, double* f, cudaStream_t s) {
    note_launch(); launch_k(k_adj_zero_walls, tg(g), TB, 0, s, g, f);
}
void launch_adj_mom(const Grid& g, const PhysDev& P, const AdjFields& A, const double* bub,
                    const double* bvb, double* Un, double* Vn, cudaStream_t s) {
    note_launch(); launch_k(k_adj_mom_a, tg(g), TB, 0, s, g, P, A, bub, bvb);
    note_launch(); launch_k(k_adj_mom_b, tg(g), TB, 0, s, g, P, A, bub, bvb, Un, Vn);
}
void launch_adj_mass(const Grid& g, double* Pn1, double* Pn, const double* phb, SolveDev sd,
                     double* rhs, double inv_sumw, double* acc3, cudaStream_t s) {
    note_launch(); launch_k(k_adj_mass_a, tg(g), TB, 0, s, g, Pn1, Pn, phb, sd);
    note_launch(); launch_k(k_adj_mass_b, tg(g), TB, 0, s, g, Pn1, rhs, sd.scal, inv_sumw, acc3);
}
void launch_adj_mul_w(const Grid& g, double* x, cudaStream_t s) {
    note_launch(); launch_k(k_adj_mul_w, tg(g), TB, 0, s, g, x);
}
void launch_adj_save_c(const double* scal, double m0, double inv_sumw, double* c, cudaStream_t s) {
    note_launch(); launch_k(k_adj_save_c, 1, 1, 0, s, scal, m0, inv_sumw, c);
}
void launch_adj_ch(const Grid& g, const PhysDev& P, const AdjFields& A, const double* bb,
                   const double* a, const double* mass_c, double* Pn, double* Pm, double* Un,
                   double* Um, double* Vn, double* Vm, SolveDev sd, double* acc3, cudaStream_t s) {
    note_launch(); launch_k(k_adj_ch1, tg(g), TB, 0, s, g, P, A, bb, a, mass_c);
    note_launch(); launch_k(k_adj_ch2, tg(g), TB, 0, s, g, P, A, bb, a, Pn, Pm, Un, Um, Vn, Vm, sd, acc3);
}
void launch_adj_final(const Grid& g, const double* P0, const double* Pm1, const double* acc3,
                      double* out, cudaStream_t s) {
    note_launch(); launch_k(k_adj_final, tg(g), TB, 0, s, g, P0, Pm1, acc3, out);
}

}  // namespace cahn
