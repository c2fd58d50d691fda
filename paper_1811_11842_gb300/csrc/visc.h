// Fully implicit variable-viscosity momentum: the whole stress of Eq. 4.1,
// div(2 eta(phi) D(v)), by Crank-Nicolson, u and v coupled.  See visc.cu.
#pragma once
#include "physics.h"

namespace cahn {

// bu, bv = rho v^n/dt - rho (v*.grad) v* + 1/2 div(2 eta D(v^n)) - Gamma
// div(grad phi grad phi) + f on interior rows (rho/dt times the wall values
// on the walls), from the nodal intermediates of launch_mom_prep with
// eta_bar = 0 (W.ep = eta at phi^{n+1/2}).
void launch_mom_rhs_impl(const Grid& g, const PhysDev& P, const double* u, const double* v,
                         const MomWs& W, double* bu, double* bv, cudaStream_t s);

// The operator OP_VISC acts on stacked vectors [u; v] (u rows 0..ny, then v
// rows 0..ny) of the grid op.g = {nx, 2 ny + 1}:
//   rho/dt v - 1/2 div(2 eta D(v)) on interior rows, rho/dt v on wall rows,
// eta = op.a (T*, nx (ny+1) values), c0 = op.c0, 1/hx^2 = op.gx,
// 1/hy^2 = op.gy, 1/(4 hx hy) = op.kx.  Epilogues as launch_op (no
// smoother steps).
template <typename T>
void launch_visc(const Op& op, Epi epi, const T* x, const T* b, T* y, SolveDev sd,
                 const int* gate, double rtol, cudaStream_t s);
// dinv = 1 / diag of OP_VISC (stacked)
template <typename T>
void launch_visc_dinv(const Op& op, T* dinv, cudaStream_t s);

}  // namespace cahn
