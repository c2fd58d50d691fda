// Kernels of the discrete adjoint of one time step (FP64).  See adjoint.cu.
#pragma once
#include "physics.h"

namespace cahn {

// Inputs (three time levels of the step n -> n+1 being reversed) and
// nodal work arrays of the reverse step; all [ny+1][nx].
struct AdjFields {
    const double *phi_new, *phi, *phi_prev;   // phi^{n+1}, phi^n, phi^{n-1}
    const double *u, *u_prev, *v, *v_prev;    // u^n, u^{n-1}, v^n, v^{n-1}
    const double* wf;                         // 1/2 (kappa L_h + S) phi^n + F'(phi*) - S phi*
    double *gxb, *gyb, *exb, *eyb;            // bars of grad phi^{n+1/2}, grad eta'
    double *phb, *usb, *vsb;                  // bars of phi^{n+1/2}, u*, v* (momentum part)
    double *wb, *psit;                        // bar of wf; (kappa L_h + S) phit
};

// p_bar = Dx^T(u_bar / rho) + Dy^T(v_bar / rho) on interior rows (Eq. 4.5 reversed)
void launch_adj_correct(const Grid& g, double inv_rho, const double* ub, const double* vb,
                        double* pb, cudaStream_t s);
// q = p_bar / w
void launch_adj_div_w(const Grid& g, const double* pb, double* q, cudaStream_t s);
// d_bar = w x;  utb += rho Dx^T d_bar;  vtb += rho Dy_odd^T d_bar  (Eq. 4.4 rhs reversed)
void launch_adj_div(const Grid& g, double rho, const double* x, double* utb, double* vtb,
                    cudaStream_t s);
void launch_adj_zero_walls(const Grid& g, double* f, cudaStream_t s);
// Reverse of the momentum rhs (Eq. 4.1-4.3) for the interior-row bars bub,
// bvb: fills A.phb, A.usb, A.vsb and adds the u^n, v^n bars into Un, Vn.
void launch_adj_mom(const Grid& g, const PhysDev& P, const AdjFields& A, const double* bub,
                    const double* bvb, double* Un, double* Vn, cudaStream_t s);
// Reverse of the mass correction: Pn1 (bar of phi^{n+1}) += phb/2, Pn += phb/2,
// rhs = (Pn1 - w s) / w with s = sum(Pn1) / sum(w); acc3[2] (bar of m0) += s.
void launch_adj_mass(const Grid& g, double* Pn1, double* Pn, const double* phb, SolveDev sd,
                     double* rhs, double inv_sumw, double* acc3, cudaStream_t s);
void launch_adj_mul_w(const Grid& g, double* x, cudaStream_t s);
void launch_adj_save_c(const double* scal, double m0, double inv_sumw, double* c, cudaStream_t s);
// Reverse of the phase-field rhs and coefficient (Eq. 2.4) for the bar bb
// of b: adds into the bars of phi^n, phi^{n-1}, u^n, u^{n-1}, v^n, v^{n-1};
// acc3[0] += dJ/dchi, acc3[1] += dJ/dM of this step.
void launch_adj_ch(const Grid& g, const PhysDev& P, const AdjFields& A, const double* bb,
                   const double* a, const double* mass_c, double* Pn, double* Pm, double* Un,
                   double* Um, double* Vn, double* Vm, SolveDev sd, double* acc3, cudaStream_t s);
// out = P0 + Pm1 + w acc3[2]  (phi^{-1} = phi^0 and m0 = <phi^0, 1>_W)
void launch_adj_final(const Grid& g, const double* P0, const double* Pm1, const double* acc3,
                      double* out, cudaStream_t s);

}  // namespace cahn
