// Temporally blocked multigrid passes (FP32 5-point and 13-point
// hierarchies).  See mg_fused.cu.
#pragma once
#include "internal.h"

namespace cahn {

enum FusedMode { FUSED_DOWN = 0, FUSED_UP = 1, FUSED_COARSE = 2 };

// Dynamic shared memory a pass may use (four staged arrays).
constexpr size_t FUSED_SMEM_MAX = 100 * 1024;
// Chebyshev steps of the passes: the smoother's degree (FUSED_DOWN,
// FUSED_UP) and the coarsest level's steps (FUSED_COARSE); hierarchies with
// other counts keep the separate launches.
constexpr int FUSED_DEG_MIN = 3, FUSED_DEG_MAX = 5;
constexpr int FUSED_COARSE_STEPS = 6;
constexpr int FUSED_COARSE_STEPS13 = 3;   // the phase-field hierarchy's coarsest level
// the coarsest-level step counts a fused pass takes for operator `kind`
inline bool fused_coarse_steps(int kind, int steps) {
    return steps == FUSED_COARSE_STEPS || (kind == OP_CH13 && steps == FUSED_COARSE_STEPS13);
}
constexpr int FUSED_MAXK = 8;
// the 13-point passes stage six arrays with a halo of two nodes per step
constexpr size_t FUSED13_SMEM_MAX = 160 * 1024;

// 13-point operator constants rounded to T on the host (as k_ch13v's)
template <typename T>
struct C13 {
    T kx, ky, S, gxq, gyq, idt;
};

// One pass on one level.  ca: the level's smoother operands (D^-1 values,
// the rows held at zero, the step table; FUSED_UP also x_c, its grid and the
// coarsening); steps: Chebyshev steps k = 0 .. steps-1; halo: deg + 1
// (FUSED_DOWN), deg (FUSED_UP), steps - 1 (FUSED_COARSE).  b: the level's
// right-hand side; xin: the down pass's x (FUSED_UP); xout: the new x (must
// not alias b or xin); bc, gc, semi: the coarse right-hand side, its grid and
// the coarsening (FUSED_DOWN).  kc, c1, c2: the operator's constants and the
// step table rounded to T on the host (no FP64 in the kernel).
template <typename T>
struct FusedPass {
    Op op;
    ChebArgs<T> ca;
    Lap5C<T> kc;
    T c1[FUSED_MAXK], c2[FUSED_MAXK];   // 5-point levels (13-point: read from ca.coef)
    C13<T> k13;
    Grid gc;
    int semi, steps, halo;
    const T* b;
    const T* xin;
    T* xout;
    T* bc;
};

// opt the passes of operator `kind` at smoother degree `degree` (and the
// coarsest level's) in to their dynamic shared memory; called at set-up,
// before any launch or stream capture
template <typename T>
void fused_prepare(int kind, int degree);
template <typename T>
void launch_fused(int mode, const FusedPass<T>& fp, const int* gate, cudaStream_t s);

}  // namespace cahn
