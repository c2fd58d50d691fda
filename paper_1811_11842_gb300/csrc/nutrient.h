// Nutrient transport and network production (Eq. 2.5-2.7).  See nutrient.cu.
#pragma once
#include "internal.h"

namespace cahn {

struct NutDev {
    double diff_s, consume_a, mu, kc, eps_g, c_bulk;
    double dt, idt;
    int dtop;            // 1: c = c_bulk on the top wall; 0: zero flux on both walls
};

// The step's nutrient system from phi^{n+1} (phi_new), phi^n (phi) and the
// extrapolation levels: a = D_s phi_s^{n+1/2} / 4, dg, dinv = 1 / diag(K)
// and, when b is not null, the right-hand side b and the initial guess x0
// (c^n; c_bulk on a Dirichlet top wall).  The *32 outputs (may be null)
// receive FP32 copies of a, dg and dinv.  For the frozen-coefficient
// operator of single solves pass phi_new = phi and b = null.  With status
// not null, CTL_DOMAIN is or-ed into *status where the solvent fraction
// 1 - phi^{n+1} is not positive or the diffusion coefficient
// D_s (1 - phi^{n+1/2}) is negative: K is then no longer positive definite.
void launch_nut_prep(const Grid& g, const NutDev& N, const double* phi_new, const double* phi,
                     const double* phi_prev, const double* c, const double* c_prev,
                     const double* u, const double* u_prev, const double* v,
                     const double* v_prev, double* a, double* dg, double* dinv, double* b,
                     double* x0, float* a32, float* dg32, float* dinv32, int* status,
                     cudaStream_t s);
// gr = g_n(phi*, c*) (Eq. 2.5), b += gr
void launch_growth(const Grid& g, const NutDev& N, const double* phi, const double* phi_prev,
                   const double* c, const double* c_prev, double* b, double* gr,
                   cudaStream_t s);
// phi += (target - <phi,1>_W) / <1,1>_W with target = *m + scal[S_TMP1]
// (scal[S_MASS] = <phi,1>_W, scal[S_TMP1] = dt <g_n,1>_W); the target is
// also written to scal[S_TMP0]
void launch_mass_fix_grow(size_t n, double* phi, double* scal, const double* m,
                          double inv_sumw, cudaStream_t s);
// x = b dt on the top wall row (the Dirichlet row of K with N.dtop)
void launch_nut_top(const Grid& g, double* x, const double* b, double dt, cudaStream_t s);

}  // namespace cahn
