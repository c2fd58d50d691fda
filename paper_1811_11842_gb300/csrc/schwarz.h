// Domain-decomposition preconditioner (CAHN_PC_SCHWARZ).  See schwarz.cu.
#pragma once
#include "internal.h"

namespace cahn {

constexpr int SW_CX = 32, SW_CY = 16;   // subdomain tile
constexpr int SW_STEPS = 12;            // local Chebyshev-Jacobi steps
constexpr double SW_ALPHA = 64.0;       // local interval [lam / SW_ALPHA, lam]

// z = M r: one launch, one block per subdomain (op: the fine operator with
// its coefficient fields; dinv: 1/diag (read for the coefficient kinds);
// coef: the SW_STEPS-step table on [lam/SW_ALPHA, lam]; dz: rows held at 0).
template <typename T>
void launch_schwarz(const Op& op, const T* r, T* z, const T* dinv, const double* coef, int dz,
                    const int* gate, cudaStream_t s);

}  // namespace cahn
