// Explicit step kernels (FP64).  See physics.cu.
#pragma once
#include "internal.h"

namespace cahn {

struct PhysDev {
    double kappa, mobility, chi, n_poly, S, gamma2;
    double inv_npoly;    // 1 / n_poly (formed on the host)
    int energy;          // 0 Flory-Huggins, 1 double well
    double idt, rho, nu; // 1/dt, density, eta_bar / 2
    double eta_w, eta_b, eta_bar, gamma_cap, fx, u_wall0, u_wall1;
};

struct MomWs {           // nodal intermediates of the momentum rhs
    double *txx, *txy, *tyy, *ep, *us, *vs;
};

void launch_ch_prep(const Grid& g, const PhysDev& P, const double* phi, const double* phi_prev,
                    double* a, float* a32, double* wr, int* status, const int* gate,
                    cudaStream_t s);
void launch_ch_rhs(const Grid& g, const PhysDev& P, const double* phi, const double* phi_prev,
                   const double* u, const double* u_prev, const double* v, const double* v_prev,
                   const double* a, const double* wr, double* b, int* fold, int* status, cudaStream_t s);
void launch_mass_fix(size_t n, double* phi, const double* scal, double m0, double inv_sumw,
                     cudaStream_t s);
void launch_mom_prep(const Grid& g, const PhysDev& P, const double* phi_new, const double* phi,
                     const double* u, const double* u_prev, const double* v, const double* v_prev,
                     const MomWs& W, cudaStream_t s);
void launch_mom_rhs(const Grid& g, const PhysDev& P, const double* u, const double* v,
                    const MomWs& W, double* bu, double* bv, cudaStream_t s);
void launch_div(const Grid& g, double rho, const double* u, const double* v, double* d,
                cudaStream_t s);
void launch_correct(const Grid& g, double inv_rho, const double* p, double* u, double* v,
                    cudaStream_t s);

}  // namespace cahn
