// Krylov vector kernels: CG updates, Jacobi scaling, GMRES(m) Arnoldi steps
// (classical Gram-Schmidt as one multi-dot pass and one multi-axpy pass),
// Givens rotations and the restart update.  Every reduction is W-weighted
// (trapezoid weights), accumulated in FP64 whatever the vector type, and
// finished deterministically by the last block, which writes the scalars
// the next kernel reads.  Every kernel returns at once while its gate flag
// is set, so iterations can be queued ahead of the convergence test.
#include "internal.h"

namespace cahn {

__device__ __forceinline__ size_t gtid() {
    return (size_t)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ size_t gstride() { return (size_t)gridDim.x * blockDim.x; }

// ------------------------------------------------------------------ misc
template <typename T>
__global__ void k_copy(const T* __restrict__ x, T* __restrict__ y, size_t n,
                       const int* __restrict__ gate) {
    if (gate && *gate) return;
    for (size_t e = gtid(); e < n; e += gstride()) y[e] = x[e];
}
template <typename Ts, typename Td>
__global__ void k_convert(const Ts* __restrict__ x, Td* __restrict__ y, size_t n) {
    for (size_t e = gtid(); e < n; e += gstride()) y[e] = (Td)x[e];
}
__global__ void k_fill(double* y, double v, size_t n) {
    for (size_t e = gtid(); e < n; e += gstride()) y[e] = v;
}
template <typename T>
__global__ void k_zero(T* y, size_t n, const int* __restrict__ gate) {
    if (gate && *gate) return;
    for (size_t e = gtid(); e < n; e += gstride()) y[e] = (T)0;
}

__global__ void k_ctl_init(Ctl* c, int maxit, const int* __restrict__ gate) {
    if (gate && *gate) {   // enclosing loop finished: this solve is skipped
        c->it = 0;
        c->done = 1;
        c->cycle_end = 1;
        c->idle = 1;
        return;
    }
    c->done = 0;
    c->it = 0;
    c->status = 0;
    c->cycle_end = 1;
    c->k = 0;
    c->maxit = maxit;
    c->cycles = 0;
    c->idle = 1;
}

// <x, y>_W into scal[slot]; or, with `sub_mean`, x -= <x,1>_W / <1,1>_W
// handled by two kernels (reduction then subtraction).
template <typename T>
__global__ void k_wdot(Grid g, const T* __restrict__ x, const T* __restrict__ y,
                       SolveDev sd, int slot, double scale, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride())
        acc.add(wgt_t<T>(e, g), x[e], y ? y[e] : (T)1);
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    double t = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        sd.scal[slot] = t * scale;
        reset_counter(sd.red);
    }
}

template <typename T>
__global__ void k_sub_scalar(T* __restrict__ x, size_t n, const double* __restrict__ s,
                             const int* __restrict__ gate) {
    if (gate && *gate) return;
    T vv[1];
    block_scalars<T, 1>(s, {0}, vv);
    const T v = vv[0];
    for (size_t e = gtid(); e < n; e += gstride()) x[e] -= v;
}

// Dirichlet rows of the velocity predictor: x = b / c0 on the two wall
// rows, so the residual vanishes there and every Krylov vector stays in the
// interior subspace, where the operator is W-symmetric.
template <typename T>
__global__ void k_dirichlet_walls(Grid g, T* __restrict__ x, const T* __restrict__ b,
                                  double inv_c0) {
    const size_t nx = g.nx, top = (size_t)g.ny * g.nx;
    for (size_t e = gtid(); e < 2 * nx; e += gstride()) {
        const size_t k = e < nx ? e : top + (e - nx);
        x[k] = (T)((double)b[k] * inv_c0);
    }
}

// ------------------------------------------------------------------ CG
// x += alpha p ; r -= alpha q ; RR = <r,r>_W ; convergence test.
template <typename T>
__global__ void k_cg_update(Grid g, T* __restrict__ x, T* __restrict__ r,
                            const T* __restrict__ p, const T* __restrict__ q, SolveDev sd,
                            const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    T sv[1];
    block_scalars<T, 1>(sd.scal, {S_ALPHA}, sv);
    const T alpha = sv[0];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        x[e] += alpha * p[e];
        T rv = r[e] - alpha * q[e];
        r[e] = rv;
        acc.add(wgt_t<T>(e, g), rv, rv);
    }
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    double t = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        Ctl* c = sd.ctl;
        sd.scal[S_RR] = t;
        c->it += 1;
        c->total += 1;
        if (!isfinite(t)) {
            c->status |= CTL_NAN;
            c->done = 1;
        } else if (t <= sd.scal[S_TOL2]) {
            c->done = 1;
        } else if (c->it >= c->maxit) {
            c->status |= CTL_NOT_CONVERGED;
            c->done = 1;
        }
        sd.scal[S_RES0] = sqrt(t);
        reset_counter(sd.red);
    }
}

// z = dinv r (if dinv) ; RZnew = <r,z>_W ; BETA = RZnew / RZ ; RZ = RZnew.
template <typename T>
__global__ void k_cg_rz(Grid g, const T* __restrict__ r, const T* __restrict__ dinv,
                        T* __restrict__ z, SolveDev sd, int first,
                        const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        T zv;
        if (dinv) {
            zv = dinv[e] * r[e];
            z[e] = zv;
        } else {
            zv = z[e];
        }
        acc.add(wgt_t<T>(e, g), r[e], zv);
    }
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    double t = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        sd.scal[S_BETA] = first ? 0.0 : (sd.scal[S_RZ] != 0.0 ? t / sd.scal[S_RZ] : 0.0);
        sd.scal[S_RZ] = t;
        if (!isfinite(t)) {
            sd.ctl->status |= CTL_NAN;
            sd.ctl->done = 1;
        }
        reset_counter(sd.red);
    }
}

// The update of the Chronopoulos-Gear CG iteration (after w = A z and the
// scalars of EPI_CGCG): p = z + BETA p, s = w + BETA s (p = z, s = w in the
// first iteration), x += ALPHA p, r -= ALPHA s; RR = <r,r>_W and the
// convergence test of k_cg_update.
template <typename T>
__global__ void k_cgcg_update(Grid g, T* __restrict__ x, T* __restrict__ r, T* __restrict__ p,
                              T* __restrict__ sv, const T* __restrict__ z,
                              const T* __restrict__ w, SolveDev sd, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    T ab[2];
    block_scalars<T, 2>(sd.scal, {S_ALPHA, S_BETA}, ab);
    const T alpha = ab[0], beta = ab[1];
    const bool first = sd.ctl->it == 0;
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        const T pe = first ? z[e] : fma(beta, p[e], z[e]);
        const T se = first ? w[e] : fma(beta, sv[e], w[e]);
        p[e] = pe;
        sv[e] = se;
        x[e] = fma(alpha, pe, x[e]);
        const T rv = fma(-alpha, se, r[e]);
        r[e] = rv;
        acc.add(wgt_t<T>(e, g), rv, rv);
    }
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    double t = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        Ctl* c = sd.ctl;
        sd.scal[S_RR] = t;
        c->it += 1;
        c->total += 1;
        if (!isfinite(t)) {
            c->status |= CTL_NAN;
            c->done = 1;
        } else if (t <= sd.scal[S_TOL2]) {
            c->done = 1;
        } else if (c->it >= c->maxit) {
            c->status |= CTL_NOT_CONVERGED;
            c->done = 1;
        }
        sd.scal[S_RES0] = sqrt(t);
        reset_counter(sd.red);
    }
}

// p = z + BETA p
template <typename T>
__global__ void k_cg_p(size_t n, const T* __restrict__ z, T* __restrict__ p, SolveDev sd,
                       const int* __restrict__ gate) {
    if (gate && *gate) return;
    T bv[1];
    block_scalars<T, 1>(sd.scal, {S_BETA}, bv);
    const T beta = bv[0];
    for (size_t e = gtid(); e < n; e += gstride()) p[e] = z[e] + beta * p[e];
}

// y = dinv x
template <typename T>
__global__ void k_scale_by(size_t n, const T* __restrict__ dinv, const T* __restrict__ x,
                           T* __restrict__ y, const int* __restrict__ gate) {
    if (gate && *gate) return;
    for (size_t e = gtid(); e < n; e += gstride()) y[e] = dinv[e] * x[e];
}

// y = 1 / d
template <typename T>
__global__ void k_invert(size_t n, T* __restrict__ d) {
    for (size_t e = gtid(); e < n; e += gstride()) d[e] = (T)1 / d[e];
}

// x += y  (y scaled by dinv when given)
template <typename T>
__global__ void k_add(size_t n, T* __restrict__ x, const T* __restrict__ y,
                      const T* __restrict__ dinv, const int* __restrict__ gate) {
    if (gate && *gate) return;
    for (size_t e = gtid(); e < n; e += gstride()) x[e] += dinv ? dinv[e] * y[e] : y[e];
}

// x = 0 when ||b|| = 0 (the solution of A x = 0)
template <typename T>
__global__ void k_zero_if_b0(size_t n, T* __restrict__ x, const double* __restrict__ scal) {
    if (scal[S_BN] != 0.0) return;
    for (size_t e = gtid(); e < n; e += gstride()) x[e] = (T)0;
}

// Loop condition of a graph WHILE node: continue while *stop == 0; counts
// its executions.
__global__ void k_set_cond(cudaGraphConditionalHandle h, const int* __restrict__ stop,
                           unsigned* __restrict__ counter) {
    cudaGraphSetConditional(h, *stop ? 0u : 1u);
    if (counter) *counter += 1u;
}

// ------------------------------------------------------------------ refinement
// Stopping test of one refinement sweep, after r = b - A x (EPI_RESID, which
// already stopped the loop if ||r|| <= rtol ||b||) and ||x||^2 in S_TMP2:
// stop at the FP64 rounding floor 16 eps (anorm ||x|| + ||b||), after three
// sweeps in a row without a 10% reduction, or at the sweep cap.

// ------------------------------------------------------------------ refinement transfers
// r32 = r64 / ||r64||_W  (||r|| = scal[S_RES0], from the fused residual)
__global__ void k_ir_down(size_t n, const double* __restrict__ r, float* __restrict__ r32,
                          const double* __restrict__ scal, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sinv;   // one FP64 division per block, not per thread
    if (threadIdx.x == 0) {
        const double s = scal[S_RES0];
        sinv = s > 0.0 ? 1.0 / s : 0.0;
    }
    __syncthreads();
    const double inv = sinv;
    for (size_t e = gtid(); e < n; e += gstride()) r32[e] = (float)(r[e] * inv);
}
// x64 += ||r64|| d32
__global__ void k_ir_up(size_t n, double* __restrict__ x, const float* __restrict__ d32,
                        const double* __restrict__ scal, const int* __restrict__ gate) {
    if (gate && *gate) return;
    const double s = scal[S_RES0];
    for (size_t e = gtid(); e < n; e += gstride()) x[e] += s * (double)d32[e];
}

// ------------------------------------------------------------------ GMRES
// Start of a restart cycle (after r = b - A x with EPI_RESID): V0 = r / beta,
// g = (beta, 0, ...), k = 0.  Stops the solve at the iteration cap.
template <typename T>
__global__ void k_gm_start(Grid g, const T* __restrict__ r, T* __restrict__ V0,
                           T* __restrict__ vk, SolveDev sd, GmDev gm) {
    Ctl* c = sd.ctl;
    const bool capped = c->it >= c->maxit;
    if (c->done || capped) {
        if (capped && !c->done && blockIdx.x == 0 && threadIdx.x == 0) {
            c->status |= CTL_NOT_CONVERGED;
            c->done = 1;
        }
        return;
    }
    const double beta = sqrt(sd.scal[S_RR]);
    const T inv = (T)(1.0 / beta);
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        const T v = r[e] * inv;
        V0[e] = v;
        vk[e] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        gm.g[0] = beta;
        c->k = 0;
        c->cycle_end = 0;
        c->idle = 0;
        c->cycles += 1;
    }
}

// h_i = <w, V_i>_W for i = 0..k  (column k of the Hessenberg matrix).
// Basis vectors are taken 8 at a time: each thread keeps 8 partial sums in
// registers, w is read once per chunk, and one 8-wide block reduction per
// chunk publishes the partials.
constexpr int MD_CHUNK = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_gm_multidot(Grid g, const T* __restrict__ w,
                                                     const T* __restrict__ V, size_t ldv,
                                                     SolveDev sd, GmDev gm,
                                                     const T* __restrict__ z,
                                                     T* __restrict__ Zb) {
    Ctl* c = sd.ctl;
    if (c->cycle_end) return;
    __shared__ double sh[MD_CHUNK][8];   // [value][warp] (FP32: float2 pairs)
    __shared__ double shs[32];
    const int k = c->k;
    const size_t n = g.n();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i0 = 0; i0 <= k; i0 += MD_CHUNK) {
        const int cnt = (k + 1 - i0) < MD_CHUNK ? (k + 1 - i0) : MD_CHUNK;
        WSum<T> part[MD_CHUNK];
        // flexible GMRES: column k of the preconditioned basis is this
        // iteration's z (copied in the first chunk's pass)
        T* __restrict__ zk = (Zb && i0 == 0) ? Zb + (size_t)k * ldv : nullptr;
        for (size_t e = gtid(); e < n; e += gstride()) {
            if (zk) zk[e] = z[e];
            const T wt = wgt_t<T>(e, g), we = w[e];
#pragma unroll
            for (int q = 0; q < MD_CHUNK; ++q)
                if (q < cnt) part[q].add(wt, we, V[(size_t)(i0 + q) * ldv + e]);
        }
        if constexpr (sizeof(T) == 4) {
            // double-float pairs through the warp and block stages (common.cuh)
            float2* shp = reinterpret_cast<float2*>(&sh[0][0]);
#pragma unroll
            for (int q = 0; q < MD_CHUNK; ++q) {
                float ps = part[q].s, pc = part[q].c;
                warp_sum_pair(ps, pc);
                if (lane == 0) shp[q * 8 + wid] = make_float2(ps, pc);
            }
            __syncthreads();
            if (threadIdx.x < cnt) {
                float ps = 0.0f, pc = 0.0f;
                for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
                    const float2 v = shp[threadIdx.x * 8 + wi];
                    pair_add(ps, pc, v.x, v.y);
                }
                publish_pair(sd.red, i0 + threadIdx.x, blockIdx.x, ps, pc);
            }
        } else {
            double acc[MD_CHUNK];
#pragma unroll
            for (int q = 0; q < MD_CHUNK; ++q) acc[q] = warp_sum(part[q].get());
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < MD_CHUNK; ++q) sh[q][wid] = acc[q];
            }
            __syncthreads();
            if (threadIdx.x < cnt) {
                double s = 0.0;
                for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += sh[threadIdx.x][wi];
                sd.red.partials[(size_t)(i0 + threadIdx.x) * sd.red.stride + blockIdx.x] = s;
            }
        }
        __syncthreads();
    }
    if (!last_block(sd.red)) return;
    for (int i = 0; i <= k; ++i) {
        double t = final_wsum<T>(sd.red, i, shs);
        if (threadIdx.x == 0) gm.H[(size_t)k * gm.ldh + i] = t;
    }
    if (threadIdx.x == 0) reset_counter(sd.red);
}

// Givens rotation of column k, residual estimate, end-of-cycle test.
// (run by one thread: the last block of k_gm_multiaxpy, once H[k+1][k] is known)
__device__ __forceinline__ void gm_givens(SolveDev sd, GmDev gm, int m) {
    Ctl* c = sd.ctl;
    const int k = c->k;
    double* h = gm.H + (size_t)k * gm.ldh;
    for (int i = 0; i < k; ++i) {
        double t = gm.cs[i] * h[i] + gm.sn[i] * h[i + 1];
        h[i + 1] = -gm.sn[i] * h[i] + gm.cs[i] * h[i + 1];
        h[i] = t;
    }
    const double hk1 = h[k + 1];
    const double den = hypot(h[k], hk1);
    double cs = 1.0, sn = 0.0;
    if (den != 0.0) {
        cs = h[k] / den;
        sn = hk1 / den;
    }
    gm.cs[k] = cs;
    gm.sn[k] = sn;
    h[k] = den;
    h[k + 1] = 0.0;
    gm.g[k + 1] = -sn * gm.g[k];
    gm.g[k] = cs * gm.g[k];
    const double res = fabs(gm.g[k + 1]);
    c->it += 1;
    c->total += 1;
    c->k = k + 1;
    sd.scal[S_TMP1] = (hk1 != 0.0) ? 1.0 / hk1 : 0.0;
    sd.scal[S_RES0] = res;
    if (!isfinite(res) || !isfinite(den)) {
        c->status |= CTL_NAN;
        c->done = 1;
        c->cycle_end = 1;
    } else if (res * res <= sd.scal[S_TOL2] || k + 1 >= m || c->it >= c->maxit || hk1 == 0.0 ||
               den == 0.0) {
        c->cycle_end = 1;
    }
}

// w -= sum_i h_i V_i ; H[k+1][k] = ||w||_W
template <typename T>
__global__ void k_gm_multiaxpy(Grid g, T* __restrict__ w, const T* __restrict__ V, size_t ldv,
                               SolveDev sd, GmDev gm, int m) {
    Ctl* c = sd.ctl;
    if (c->cycle_end) return;
    __shared__ double sh[32];
    __shared__ T sh_h[MAX_MULTI];
    const int k = c->k;
    for (int i = threadIdx.x; i <= k; i += blockDim.x) sh_h[i] = (T)gm.H[(size_t)k * gm.ldh + i];
    __syncthreads();
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        T wv = w[e];
        for (int i = 0; i <= k; ++i) wv -= sh_h[i] * V[(size_t)i * ldv + e];
        w[e] = wv;
        acc.add(wgt_t<T>(e, g), wv, wv);
    }
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    double t = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        gm.H[(size_t)k * gm.ldh + k + 1] = sqrt(t);
        reset_counter(sd.red);
        gm_givens(sd, gm, m);   // the rotation of column k, in this kernel's last block
    }
}


// V_{k} = w / H[k][k-1]  (k already advanced); vk is a copy of V_k at a
// fixed address for the preconditioner.
template <typename T>
__global__ void k_gm_scale(size_t n, const T* __restrict__ w, T* __restrict__ V, size_t ldv,
                           T* __restrict__ vk, SolveDev sd) {
    Ctl* c = sd.ctl;
    if (c->cycle_end) return;
    T iv[1];
    block_scalars<T, 1>(sd.scal, {S_TMP1}, iv);
    const T inv = iv[0];
    T* __restrict__ v = V + (size_t)c->k * ldv;
    for (size_t e = gtid(); e < n; e += gstride()) {
        const T t = w[e] * inv;
        v[e] = t;
        vk[e] = t;
    }
}

// y = R^{-1} g (upper triangular, k x k) -- one thread.
__global__ void k_gm_trisolve(SolveDev sd, GmDev gm) {
    Ctl* c = sd.ctl;
    if (c->idle || (c->status & CTL_NAN)) return;
    const int k = c->k;
    for (int i = k - 1; i >= 0; --i) {
        double s = gm.g[i];
        for (int j = i + 1; j < k; ++j) s -= gm.H[(size_t)j * gm.ldh + i] * gm.y[j];
        const double d = gm.H[(size_t)i * gm.ldh + i];
        gm.y[i] = d != 0.0 ? s / d : 0.0;
    }
}

// u = sum_{i<k} y_i V_i   (then x += M u by the preconditioner path), or,
// with `dinv` (Jacobi), x += dinv * sum y_i V_i directly.  Marks the cycle
// finished.
template <typename T>
__global__ void k_gm_combine(Grid g, const T* __restrict__ V, size_t ldv, T* __restrict__ out,
                             const T* __restrict__ dinv, int add, SolveDev sd, GmDev gm) {
    Ctl* c = sd.ctl;
    if (c->idle || (c->status & CTL_NAN)) return;
    __shared__ T sy[MAX_MULTI];
    const int k = c->k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) sy[i] = (T)gm.y[i];
    __syncthreads();
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        T s = 0;
        for (int i = 0; i < k; ++i) s += sy[i] * V[(size_t)i * ldv + e];
        if (dinv)
            out[e] += dinv[e] * s;
        else if (add)
            out[e] += s;
        else
            out[e] = s;
    }
}

__global__ void k_gm_finish(Ctl* c) {
    if (c->idle) return;
    c->idle = 1;
    c->k = 0;
}

// ------------------------------------------------------------------ launch
template <typename T>
void launch_copy(const T* x, T* y, size_t n, cudaStream_t s, const int* gate) {
    note_launch(); launch_k(k_copy<T>, vec_blocks(n), RED_THREADS, 0, s, x, y, n, gate);
}
template <typename Ts, typename Td>
void launch_convert(const Ts* x, Td* y, size_t n, cudaStream_t s) {
    note_launch(); launch_k(k_convert<Ts, Td>, vec_blocks(n), RED_THREADS, 0, s, x, y, n);
}
void launch_fill(double* y, double v, size_t n, cudaStream_t s) {
    note_launch(); launch_k(k_fill, vec_blocks(n), RED_THREADS, 0, s, y, v, n);
}
template <typename T>
void launch_zero(T* y, size_t n, const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_zero<T>, vec_blocks(n), RED_THREADS, 0, s, y, n, gate);
}
void launch_ctl_init(Ctl* c, int maxit, cudaStream_t s, const int* gate) {
    note_launch(); launch_k(k_ctl_init, 1, 1, 0, s, c, maxit, gate);
}
template <typename T>
void launch_zero_if_b0(size_t n, T* x, const double* scal, cudaStream_t s) {
    note_launch(); launch_k(k_zero_if_b0<T>, vec_blocks(n), RED_THREADS, 0, s, n, x, scal);
}
void launch_set_cond(cudaGraphConditionalHandle h, const int* stop, unsigned* counter,
                     cudaStream_t s) {
    note_launch(); launch_k(k_set_cond, 1, 1, 0, s, h, stop, counter);
}
template <typename T>
void launch_dirichlet_walls(const Grid& g, T* x, const T* b, double inv_c0, cudaStream_t s) {
    note_launch(); launch_k(k_dirichlet_walls<T>, vec_blocks(2 * (size_t)g.nx), RED_THREADS, 0, s, g, x, b, inv_c0);
}

template <typename T>
void launch_wdot(const Grid& g, const T* x, const T* y, SolveDev sd, int slot, double scale,
                 const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_wdot<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, x, y, sd, slot, scale, gate);
}
template <typename T>
void launch_sub_scalar(T* x, size_t n, const double* sc, const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_sub_scalar<T>, vec_blocks(n), RED_THREADS, 0, s, x, n, sc, gate);
}
// Start of a solve from x = 0: x = 0, r = b, with the bookkeeping of the
// residual epilogue (||b||_W, ||r||_W = ||b||_W, tolerance; done when b = 0)
// and no operator application.
template <typename T>
__global__ void k_start_zero(Grid g, const T* __restrict__ b, T* __restrict__ x,
                             T* __restrict__ r, SolveDev sd, double rtol,
                             const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        const T bv = b[e];
        x[e] = (T)0;
        r[e] = bv;
        acc.add(wgt_t<T>(e, g), bv, bv);
    }
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    const double t0 = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        double* sc = sd.scal;
        sc[S_BN] = sqrt(t0);
        sc[S_RR] = t0;
        sc[S_RES0] = sqrt(t0);
        sc[S_TOL2] = rtol * rtol * t0;
        if (!isfinite(t0)) {
            sd.ctl->status |= CTL_NAN;
            sd.ctl->done = 1;
        } else if (t0 == 0.0) {
            sd.ctl->done = 1;
        }
        reset_counter(sd.red);
    }
}

// ------------------------------------------------------------- BiCGStab
// Right-preconditioned BiCGStab in the W inner product, scalars on the
// device (slots: RHO = rho of the previous iteration, TMP0 = rho, BETA,
// ALPHA, OMEGA).  Every kernel returns at once while *gate != 0.

// after r = b - A x: rhat = r, p = v = 0; rho_old = alpha = omega = 1
template <typename T>
__global__ void k_bicg_init(size_t n, const T* __restrict__ r, T* __restrict__ rhat,
                            T* __restrict__ p, T* __restrict__ v, double* __restrict__ scal,
                            const int* __restrict__ gate) {
    if (gate && *gate) return;
    for (size_t e = gtid(); e < n; e += gstride()) {
        rhat[e] = r[e];
        p[e] = (T)0;
        v[e] = (T)0;
    }
    if (gtid() == 0) {
        scal[S_RHO] = 1.0;
        scal[S_ALPHA] = 1.0;
        scal[S_OMEGA] = 1.0;
    }
}

// rho = <rhat, r>_W; beta = (rho / rho_old)(alpha / omega); rho_old = rho.
// rho = 0 (breakdown) ends the solve as not converged.
template <typename T>
__global__ void k_bicg_rho(Grid g, const T* __restrict__ rhat, const T* __restrict__ r,
                           SolveDev sd, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) acc.add(wgt_t<T>(e, g), rhat[e], r[e]);
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    const double rho = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        double* sc = sd.scal;
        Ctl* c = sd.ctl;
        if (!isfinite(rho)) {
            c->status |= CTL_NAN;
            c->done = 1;
        } else if (rho == 0.0) {
            c->status |= CTL_NOT_CONVERGED;
            c->done = 1;
        }
        sc[S_BETA] = (sc[S_RHO] != 0.0 && sc[S_OMEGA] != 0.0)
                         ? (rho / sc[S_RHO]) * (sc[S_ALPHA] / sc[S_OMEGA]) : 0.0;
        sc[S_TMP0] = rho;
        sc[S_RHO] = rho;
        reset_counter(sd.red);
    }
}

// p = r + beta (p - omega v)
template <typename T>
__global__ void k_bicg_p(size_t n, const T* __restrict__ r, T* __restrict__ p,
                         const T* __restrict__ v, const double* __restrict__ scal,
                         const int* __restrict__ gate) {
    if (gate && *gate) return;
    const T beta = (T)scal[S_BETA], omega = (T)scal[S_OMEGA];
    for (size_t e = gtid(); e < n; e += gstride()) p[e] = fma(beta, fma(-omega, v[e], p[e]), r[e]);
}

// alpha = rho / <rhat, v>_W
template <typename T>
__global__ void k_bicg_alpha(Grid g, const T* __restrict__ rhat, const T* __restrict__ v,
                             SolveDev sd, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) acc.add(wgt_t<T>(e, g), rhat[e], v[e]);
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    const double sig = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        double* sc = sd.scal;
        if (!isfinite(sig) || sig == 0.0) {
            sd.ctl->status |= isfinite(sig) ? CTL_NOT_CONVERGED : CTL_NAN;
            sd.ctl->done = 1;
            sc[S_ALPHA] = 0.0;
        } else {
            sc[S_ALPHA] = sc[S_TMP0] / sig;
        }
        reset_counter(sd.red);
    }
}

// s = r - alpha v
template <typename T>
__global__ void k_bicg_s(size_t n, const T* __restrict__ r, const T* __restrict__ v,
                         T* __restrict__ s, const double* __restrict__ scal,
                         const int* __restrict__ gate) {
    if (gate && *gate) return;
    const T alpha = (T)scal[S_ALPHA];
    for (size_t e = gtid(); e < n; e += gstride()) s[e] = fma(-alpha, v[e], r[e]);
}

// omega = <t, s>_W / <t, t>_W (0 when t = 0)
template <typename T>
__global__ void k_bicg_omega(Grid g, const T* __restrict__ t, const T* __restrict__ s,
                             SolveDev sd, const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    WSum<T> ts, tt;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        const T w = wgt_t<T>(e, g);
        ts.add(w, t[e], s[e]);
        tt.add(w, t[e], t[e]);
    }
    publish_wsum<T>(sd.red, 0, ts, sh);
    publish_wsum<T>(sd.red, 1, tt, sh);
    if (!last_block(sd.red)) return;
    const double a = final_wsum<T>(sd.red, 0, sh);
    const double b = final_wsum<T>(sd.red, 1, sh);
    if (threadIdx.x == 0) {
        sd.scal[S_OMEGA] = (b > 0.0 && isfinite(a) && isfinite(b)) ? a / b : 0.0;
        reset_counter(sd.red);
    }
}

// x += alpha phat + omega shat; r = s - omega t; ||r||_W, convergence
template <typename T>
__global__ void k_bicg_x(Grid g, T* __restrict__ x, T* __restrict__ r,
                         const T* __restrict__ phat, const T* __restrict__ shat,
                         const T* __restrict__ s, const T* __restrict__ t, SolveDev sd,
                         const int* __restrict__ gate) {
    if (gate && *gate) return;
    __shared__ double sh[32];
    const T alpha = (T)sd.scal[S_ALPHA], omega = (T)sd.scal[S_OMEGA];
    WSum<T> acc;
    const size_t n = g.n();
    for (size_t e = gtid(); e < n; e += gstride()) {
        x[e] = fma(omega, shat[e], fma(alpha, phat[e], x[e]));
        const T rv = fma(-omega, t[e], s[e]);
        r[e] = rv;
        acc.add(wgt_t<T>(e, g), rv, rv);
    }
    publish_wsum<T>(sd.red, 0, acc, sh);
    if (!last_block(sd.red)) return;
    const double rr = final_wsum<T>(sd.red, 0, sh);
    if (threadIdx.x == 0) {
        Ctl* c = sd.ctl;
        double* sc = sd.scal;
        sc[S_RR] = rr;
        sc[S_RES0] = sqrt(rr);
        c->it += 1;
        c->total += 1;
        if (!isfinite(rr)) {
            c->status |= CTL_NAN;
            c->done = 1;
        } else if (rr <= sc[S_TOL2]) {
            c->done = 1;
        } else if (sc[S_OMEGA] == 0.0 || c->it >= c->maxit) {
            c->status |= CTL_NOT_CONVERGED;
            c->done = 1;
        }
        reset_counter(sd.red);
    }
}

template <typename T>
void launch_cg_update(const Grid& g, T* x, T* r, const T* p, const T* q, SolveDev sd,
                      const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_cg_update<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, x, r, p, q, sd, gate);
}
template <typename T>
void launch_cgcg_update(const Grid& g, T* x, T* r, T* p, T* sv, const T* z, const T* w,
                        SolveDev sd, const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_cgcg_update<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, x, r, p, sv, z, w, sd, gate);
}
template <typename T>
void launch_cg_rz(const Grid& g, const T* r, const T* dinv, T* z, SolveDev sd, int first,
                  const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_cg_rz<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, r, dinv, z, sd, first, gate);
}
template <typename T>
void launch_cg_p(size_t n, const T* z, T* p, SolveDev sd, const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_cg_p<T>, vec_blocks(n), RED_THREADS, 0, s, n, z, p, sd, gate);
}
template <typename T>
void launch_scale_by(size_t n, const T* dinv, const T* x, T* y, const int* gate,
                     cudaStream_t s) {
    note_launch(); launch_k(k_scale_by<T>, vec_blocks(n), RED_THREADS, 0, s, n, dinv, x, y, gate);
}
template <typename T>
void launch_invert(size_t n, T* d, cudaStream_t s) {
    note_launch(); launch_k(k_invert<T>, vec_blocks(n), RED_THREADS, 0, s, n, d);
}
template <typename T>
void launch_add(size_t n, T* x, const T* y, const T* dinv, const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_add<T>, vec_blocks(n), RED_THREADS, 0, s, n, x, y, dinv, gate);
}
template <typename T>
void launch_gm_start(const Grid& g, const T* r, T* V0, T* vk, SolveDev sd, GmDev gm,
                     cudaStream_t s) {
    note_launch(); launch_k(k_gm_start<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, r, V0, vk, sd, gm);
}
template <typename T>
void launch_gm_arnoldi(const Grid& g, T* w, T* V, size_t ldv, T* vk, SolveDev sd, GmDev gm,
                       int m, cudaStream_t s, const T* z, T* Z) {
    const int nb = vec_blocks(g.n());
    note_launch(); launch_k(k_gm_multidot<T>, nb, RED_THREADS, 0, s, g, w, V, ldv, sd, gm, z, Z);
    note_launch(); launch_k(k_gm_multiaxpy<T>, nb, RED_THREADS, 0, s, g, w, V, ldv, sd, gm, m);
    note_launch(); launch_k(k_gm_scale<T>, nb, RED_THREADS, 0, s, g.n(), w, V, ldv, vk, sd);
}
template <typename T>
void launch_gm_update(const Grid& g, const T* V, size_t ldv, T* out, const T* dinv, SolveDev sd,
                      GmDev gm, cudaStream_t s, int add) {
    note_launch(); launch_k(k_gm_trisolve, 1, 1, 0, s, sd, gm);
    note_launch(); launch_k(k_gm_combine<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, V, ldv, out, dinv, add, sd, gm);
}
void launch_gm_finish(Ctl* c, cudaStream_t s) { note_launch(); launch_k(k_gm_finish, 1, 1, 0, s, c); }
void launch_ir_down(size_t n, const double* r, float* r32, const double* scal, const int* gate,
                    cudaStream_t s) {
    note_launch(); launch_k(k_ir_down, vec_blocks(n), RED_THREADS, 0, s, n, r, r32, scal, gate);
}
void launch_ir_up(size_t n, double* x, const float* d32, const double* scal, const int* gate,
                  cudaStream_t s) {
    note_launch(); launch_k(k_ir_up, vec_blocks(n), RED_THREADS, 0, s, n, x, d32, scal, gate);
}

template <typename T>
void launch_start_zero(const Grid& g, const T* b, T* x, T* r, SolveDev sd, double rtol,
                       const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_start_zero<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, b, x, r, sd, rtol, gate);
}
template <typename T>
void launch_bicg_init(size_t n, const T* r, T* rhat, T* p, T* v, double* scal, const int* gate,
                      cudaStream_t s) {
    note_launch(); launch_k(k_bicg_init<T>, vec_blocks(n), RED_THREADS, 0, s, n, r, rhat, p, v, scal, gate);
}
template <typename T>
void launch_bicg_rho(const Grid& g, const T* rhat, const T* r, SolveDev sd, const int* gate,
                     cudaStream_t s) {
    note_launch(); launch_k(k_bicg_rho<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, rhat, r, sd, gate);
}
template <typename T>
void launch_bicg_p(size_t n, const T* r, T* p, const T* v, const double* scal, const int* gate,
                   cudaStream_t s) {
    note_launch(); launch_k(k_bicg_p<T>, vec_blocks(n), RED_THREADS, 0, s, n, r, p, v, scal, gate);
}
template <typename T>
void launch_bicg_alpha(const Grid& g, const T* rhat, const T* v, SolveDev sd, const int* gate,
                       cudaStream_t s) {
    note_launch(); launch_k(k_bicg_alpha<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, rhat, v, sd, gate);
}
template <typename T>
void launch_bicg_s(size_t n, const T* r, const T* v, T* sv, const double* scal, const int* gate,
                   cudaStream_t s) {
    note_launch(); launch_k(k_bicg_s<T>, vec_blocks(n), RED_THREADS, 0, s, n, r, v, sv, scal, gate);
}
template <typename T>
void launch_bicg_omega(const Grid& g, const T* t, const T* sv, SolveDev sd, const int* gate,
                       cudaStream_t s) {
    note_launch(); launch_k(k_bicg_omega<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, t, sv, sd, gate);
}
template <typename T>
void launch_bicg_x(const Grid& g, T* x, T* r, const T* phat, const T* shat, const T* sv,
                   const T* t, SolveDev sd, const int* gate, cudaStream_t s) {
    note_launch(); launch_k(k_bicg_x<T>, vec_blocks(g.n()), RED_THREADS, 0, s, g, x, r, phat, shat, sv, t, sd, gate);
}

#define CAHN_INST(T)                                                                          \
    template void launch_dirichlet_walls<T>(const Grid&, T*, const T*, double, cudaStream_t); \
    template void launch_zero_if_b0<T>(size_t, T*, const double*, cudaStream_t);                \
    template void launch_copy<T>(const T*, T*, size_t, cudaStream_t, const int*);             \
    template void launch_zero<T>(T*, size_t, const int*, cudaStream_t);                       \
    template void launch_wdot<T>(const Grid&, const T*, const T*, SolveDev, int, double,      \
                                 const int*, cudaStream_t);                                   \
    template void launch_sub_scalar<T>(T*, size_t, const double*, const int*, cudaStream_t);  \
    template void launch_cg_update<T>(const Grid&, T*, T*, const T*, const T*, SolveDev,      \
                                      const int*, cudaStream_t);                              \
    template void launch_cgcg_update<T>(const Grid&, T*, T*, T*, T*, const T*, const T*,      \
                                        SolveDev, const int*, cudaStream_t);                  \
    template void launch_cg_rz<T>(const Grid&, const T*, const T*, T*, SolveDev, int,         \
                                  const int*, cudaStream_t);                                  \
    template void launch_cg_p<T>(size_t, const T*, T*, SolveDev, const int*, cudaStream_t);   \
    template void launch_scale_by<T>(size_t, const T*, const T*, T*, const int*,              \
                                     cudaStream_t);                                           \
    template void launch_invert<T>(size_t, T*, cudaStream_t);                                 \
    template void launch_add<T>(size_t, T*, const T*, const T*, const int*, cudaStream_t);    \
    template void launch_gm_start<T>(const Grid&, const T*, T*, T*, SolveDev, GmDev,          \
                                     cudaStream_t);                                           \
    template void launch_gm_arnoldi<T>(const Grid&, T*, T*, size_t, T*, SolveDev, GmDev, int, \
                                       cudaStream_t, const T*, T*);                           \
    template void launch_gm_update<T>(const Grid&, const T*, size_t, T*, const T*, SolveDev,  \
                                      GmDev, cudaStream_t, int);                              \
    template void launch_start_zero<T>(const Grid&, const T*, T*, T*, SolveDev, double,       \
                                       const int*, cudaStream_t);                             \
    template void launch_bicg_init<T>(size_t, const T*, T*, T*, T*, double*, const int*,      \
                                      cudaStream_t);                                          \
    template void launch_bicg_rho<T>(const Grid&, const T*, const T*, SolveDev, const int*,   \
                                     cudaStream_t);                                           \
    template void launch_bicg_p<T>(size_t, const T*, T*, const T*, const double*, const int*, \
                                   cudaStream_t);                                             \
    template void launch_bicg_alpha<T>(const Grid&, const T*, const T*, SolveDev, const int*, \
                                       cudaStream_t);                                         \
    template void launch_bicg_s<T>(size_t, const T*, const T*, T*, const double*, const int*, \
                                   cudaStream_t);                                             \
    template void launch_bicg_omega<T>(const Grid&, const T*, const T*, SolveDev, const int*, \
                                       cudaStream_t);                                         \
    template void launch_bicg_x<T>(const Grid&, T*, T*, const T*, const T*, const T*,         \
                                   const T*, SolveDev, const int*, cudaStream_t);
CAHN_INST(double)
CAHN_INST(float)
template void launch_convert<double, float>(const double*, float*, size_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, size_t, cudaStream_t);

}  // namespace cahn
