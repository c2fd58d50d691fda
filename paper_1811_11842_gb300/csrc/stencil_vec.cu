// Vectorised fine-grid tiles of the stencil operators (OP_LAP5_NEUMANN,
// OP_LAP5_DIRICHLET, OP_NUT5, OP_CH13), FP32 and FP64.
//
// A block of 32 x 4 threads computes a 128-column output tile of TYV rows
// (FP32: 16, or 8 where the autotuner picks short tiles for a launch without
// reductions; FP64: 8): each thread owns four consecutive columns of TYV / 4
// consecutive rows.  The tile and its halo (two rows for the 13-point
// operator, one for the 5-point ones; four columns each side, so that every
// staged group of four columns starts on a 16-byte boundary) are staged in
// shared memory one row per warp, each lane copying 16 bytes with cp.async
// (no registers, all copies in flight at once); where the load forms x on
// the fly (the smoother's zero-guess and prolongation steps) the values pass
// through registers, all loads issued before the first store.  Constants
// of the operator come rounded to T from the host.
// Rows beyond the walls are reflected evenly (Eq. 4.7) and columns wrap
// periodically, one float4 group at a time, so a grid qualifies when nx is
// a multiple of 4 and at least 128 and every vector it touches is 16-byte
// aligned (vec_eligible); other grids take the general tiles of stencil.cu.
//
// Within a row, the x-neighbours of a thread's four nodes come from the
// lanes beside it by warp shuffles; lanes 0 and 31 read the halo column from
// shared memory instead.  The 13-point operator forms psi = kappa L_h x + S x
// on the tile and a one-node ring (the ring columns by 36 threads apart),
// then G_a psi with each face's coefficient sum and psi difference formed
// once and reused by the two nodes it separates; marching down its rows, a
// thread carries the south face of the next row over from the north face of
// the row before.  Every node is evaluated with the operations, operand
// values and rounding of the general tiles (the reused face sum a_c + a_e of
// one node is the sum a_w + a_c of the next, and IEEE addition commutes), so
// the two kernel families give bit-identical values at every node; only the
// order of the W-weighted reductions differs (fixed per grid: the choice
// depends on the grid and the buffers' alignment only).
#include <cstdlib>

#include "stencil_dev.cuh"

namespace cahn {

constexpr int VTX = 128;        // output columns per block
constexpr int VXW = VTX + 8;    // staged columns: i0 - 4 .. i0 + 131
constexpr int VG4 = VXW / 4;    // groups of four staged columns per row
template <typename T>
struct VRows {
    static constexpr int value = sizeof(T) == 4 ? 16 : 8;
};

template <typename T>
struct Vec4 {
    T v[4];
};

// The operator's constants in the kernel's precision, rounded on the host
// exactly as the general tiles round them on the device.
template <typename T>
struct VConst {
    T kx, ky, S, kcc, gxq, gyq, idt;   // 13-point
    Lap5C<T> l5;                        // 5-point
    T gx, gy;                           // nutrient
};

template <typename T>
VConst<T> vconst(const Op& op) {
    VConst<T> c;
    c.kx = (T)op.kx;
    c.ky = (T)op.ky;
    c.S = (T)op.S;
    c.kcc = (T)(2.0 * op.kx + 2.0 * op.ky + op.S);
    c.gxq = (T)(0.25 * op.gx);
    c.gyq = (T)(0.25 * op.gy);
    c.idt = (T)op.idt;
    c.l5 = lap5_consts<T>(op);
    c.gx = (T)op.gx;
    c.gy = (T)op.gy;
    return c;
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ Vec4<T> ld4(const T* p);
template <>
__device__ __forceinline__ Vec4<float> ld4<float>(const float* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    return Vec4<float>{{q.x, q.y, q.z, q.w}};
}
template <>
__device__ __forceinline__ Vec4<double> ld4<double>(const double* p) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0];
    const double2 q1 = reinterpret_cast<const double2*>(p)[1];
    return Vec4<double>{{q0.x, q0.y, q1.x, q1.y}};
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const Vec4<T>& v);
template <>
__device__ __forceinline__ void st4<float>(float* p, const Vec4<float>& v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double* p, const Vec4<double>& v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v.v[0], v.v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v.v[2], v.v[3]);
}

__device__ __forceinline__ int wrap_once(int i, int nx) {
    return i < 0 ? i + nx : (i >= nx ? i - nx : i);
}

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) {
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shfl_dn1(T v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}

// The prolonged coarse-grid correction at the four fine nodes (j, gi .. gi+3),
// gi a multiple of 4: prolong_at node by node.
template <typename T>
__device__ __forceinline__ Vec4<T> prolong4(const ChebArgs<T>& ca, int ny, int gi, int j) {
    Vec4<T> r{{(T)0, (T)0, (T)0, (T)0}};
    if (dz_row(ca.dirichlet_zero, j, ny)) return r;
    const int ncx = ca.gc.nx;
    const int J0 = j >> 1, J1 = (j & 1) ? J0 + 1 : J0;
    auto rowv = [&](int J) {
        const T* row = ca.xc + (size_t)J * ncx;
        Vec4<T> q;
        if (ca.semi) {
#pragma unroll
            for (int k = 0; k < 4; ++k) q.v[k] = row[gi + k];
        } else {
            const int I0 = gi >> 1;
            const T c0 = row[I0], c1 = row[I0 + 1], c2 = row[I0 + 2 < ncx ? I0 + 2 : 0];
            q.v[0] = c0;
            q.v[1] = (T)0.5 * (c0 + c1);
            q.v[2] = c1;
            q.v[3] = (T)0.5 * (c1 + c2);
        }
        return q;
    };
    const Vec4<T> q0 = rowv(J0);
    if (!(j & 1)) return q0;
    const Vec4<T> q1 = rowv(J1);
#pragma unroll
    for (int k = 0; k < 4; ++k) r.v[k] = (T)0.5 * (q0.v[k] + q1.v[k]);
    return r;
}

// load_x at the four nodes (jr, gi .. gi+3); e = jr nx + gi
template <typename T, int XL, int KIND>
__device__ __forceinline__ Vec4<T> load_x4(const T* __restrict__ x, const T* __restrict__ b,
                                           const ChebArgs<T>& ca, T cz, int ny, int gi, int jr,
                                           size_t e) {
    if (XL == XL_ZERO) {
        const Vec4<T> bb = ld4(b + e);
        Vec4<T> r;
        if (KIND != OP_CH13 && ca.const_dinv) {
            const T di = dinv_at<T, KIND>(ca, ny, jr, e);
#pragma unroll
            for (int k = 0; k < 4; ++k) r.v[k] = mul_rn(mul_rn(cz, di), bb.v[k]);
        } else {
            const Vec4<T> di = ld4(ca.dinv + e);
#pragma unroll
            for (int k = 0; k < 4; ++k) r.v[k] = mul_rn(mul_rn(cz, di.v[k]), bb.v[k]);
        }
        return r;
    }
    Vec4<T> v = ld4(x + e);
    if (XL == XL_PROLONG) {
        const Vec4<T> p = prolong4(ca, ny, gi, jr);
#pragma unroll
        for (int k = 0; k < 4; ++k) v.v[k] = v.v[k] + p.v[k];
    }
    return v;
}

// Stage rows j0 + roff .. j0 + roff + NR - 1 (reflected) of x as the kernel
// reads it (LOADX) or of a plain field, columns i0 - 4 .. i0 + 131: warp w
// takes rows w, w + 4, ..., lane L the column groups L and (lanes 0, 1)
// L + 32.  Plain copies go by cp.async (completed by cp_async_wait_all and
// a barrier); formed values pass through registers.
template <typename T, int NR, int XL, int KIND, bool LOADX>
__device__ __forceinline__ void stage_rows(T (*sm)[VXW], const T* __restrict__ f,
                                           const T* __restrict__ b, const ChebArgs<T>& ca, T cz,
                                           int nx, int ny, int i0, int j0, int roff, int lane,
                                           int wp) {
    constexpr int RPW = (NR + 3) / 4;
    const int gA = lane, gB = lane + 32;
    const bool hasB = gB < VG4;
    const int giA = wrap_once(i0 - 4 + 4 * gA, nx), giB = wrap_once(i0 - 4 + 4 * gB, nx);
    constexpr bool ASYNC = !LOADX || XL == XL_PLAIN;
    if constexpr (ASYNC) {
        // four values: one 16-byte copy (FP32) or two (FP64)
        auto cp4 = [](T* dst, const T* src) {
            cp_async16(dst, src);
            if constexpr (sizeof(T) == 8) cp_async16(dst + 2, src + 2);
        };
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            const int row = wp + 4 * r;
            if (row < NR) {
                const size_t base = (size_t)refly(j0 + roff + row, ny) * nx;
                cp4(&sm[row][4 * gA], f + base + giA);
                if (hasB) cp4(&sm[row][4 * gB], f + base + giB);
            }
        }
    } else {
        Vec4<T> vA[RPW], vB[RPW];
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            const int row = wp + 4 * r;
            if (row < NR) {
                const int jr = refly(j0 + roff + row, ny);
                const size_t base = (size_t)jr * nx;
                vA[r] = load_x4<T, XL, KIND>(f, b, ca, cz, ny, giA, jr, base + giA);
                if (hasB) vB[r] = load_x4<T, XL, KIND>(f, b, ca, cz, ny, giB, jr, base + giB);
            }
        }
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
            const int row = wp + 4 * r;
            if (row < NR) {
                st4(&sm[row][4 * gA], vA[r]);
                if (hasB) st4(&sm[row][4 * gB], vB[r]);
            }
        }
    }
}

// Operands of the epilogue of four consecutive nodes (b, the previous
// smoother correction d, D^-1), loaded before the tile barrier so that
// their latency overlaps the staging.
template <typename T>
struct EpiPre {
    Vec4<T> b, d, di;
};

template <typename T, int EPI, int KIND>
__device__ __forceinline__ EpiPre<T> epi_prefetch(const T* __restrict__ b, const ChebArgs<T>& ca,
                                                  size_t e, int ny, int j, T c1) {
    EpiPre<T> p{};
    constexpr bool CH = EPI == EPI_CHEB || EPI == EPI_CHEB_Z;
    if (EPI == EPI_RPLAIN || EPI == EPI_RESID || EPI == EPI_RESIDX || EPI == EPI_CGCG || CH)
        p.b = ld4(b + e);
    if (CH) {
        if (KIND != OP_CH13 && ca.const_dinv) {
            const T d0 = dinv_at<T, KIND>(ca, ny, j, e);
            p.di = Vec4<T>{{d0, d0, d0, d0}};
        } else {
            p.di = ld4(ca.dinv + e);
        }
        if (EPI == EPI_CHEB && c1 != (T)0) p.d = ld4(ca.d + e);
    }
    return p;
}

// The epilogue of four consecutive nodes of one row (epi_node, vectorised).
template <typename T, int EPI>
__device__ __forceinline__ void epi4(const Vec4<T>& ax, const Vec4<T>& xc, const EpiPre<T>& pre,
                                     T* __restrict__ y, size_t e, T w, EpiAcc<T>& acc,
                                     const ChebArgs<T>& ca, T c1, T c2) {
    Vec4<T> out;
    if (EPI == EPI_APPLY) {
        out = ax;
    } else if (EPI == EPI_RPLAIN) {
#pragma unroll
        for (int k = 0; k < 4; ++k) out.v[k] = pre.b.v[k] - ax.v[k];
    } else if (EPI == EPI_RESID || EPI == EPI_RESIDX) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T bv = pre.b.v[k];
            const T r = bv - ax.v[k];
            acc.s0.add(w, bv, bv);
            acc.s1.add(w, r, r);
            if (EPI == EPI_RESIDX) acc.s2.add(w, xc.v[k], xc.v[k]);
            out.v[k] = r;
        }
    } else if (EPI == EPI_DOTXY) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.s0.add(w, xc.v[k], ax.v[k]);
        out = ax;
    } else if (EPI == EPI_CGCG) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc.s0.add(w, pre.b.v[k], xc.v[k]);
            acc.s1.add(w, xc.v[k], ax.v[k]);
        }
        out = ax;
    } else if (EPI == EPI_NORM) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.s0.add(w, ax.v[k], ax.v[k]);
        out = ax;
    } else {   // EPI_CHEB, EPI_CHEB_Z
        Vec4<T> dn;
        if (EPI == EPI_CHEB_Z) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dn.v[k] = fma(mul_rn(c2, pre.di.v[k]), pre.b.v[k] - ax.v[k], mul_rn(c1, xc.v[k]));
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dn.v[k] = fma(mul_rn(c2, pre.di.v[k]), pre.b.v[k] - ax.v[k],
                              c1 != (T)0 ? mul_rn(c1, pre.d.v[k]) : (T)0);
        }
        st4(ca.d + e, dn);
#pragma unroll
        for (int k = 0; k < 4; ++k) out.v[k] = xc.v[k] + dn.v[k];
    }
    st4(y + e, out);
}

// ------------------------------------------------------------- 5-point
template <typename T, int KIND, int EPI, int XL, int TYV>
__global__ void __launch_bounds__(128) k_lap5v(Op op, VConst<T> vc, const T* __restrict__ x,
                                               const T* __restrict__ b, T* __restrict__ y,
                                               SolveDev sd, const int* __restrict__ gate,
                                               double rtol, ChebArgs<T> ca) {
    if (gate && *gate) return;
    constexpr int RW = TYV / 4, PH = TYV + 2;
    constexpr bool CH = EPI == EPI_CHEB || EPI == EPI_CHEB_Z;
    constexpr bool NUT = KIND == OP_NUT5;
    __shared__ __align__(16) T sx[PH][VXW];
    __shared__ __align__(16) T sa[NUT ? PH : 1][VXW];
    T c1 = 0, c2 = 0, cz = 0;
    if (CH) cheb_consts(ca, c1, c2);
    if (XL == XL_ZERO) cz = (T)ca.coef[1];
    const int nx = op.g.nx, ny = op.g.ny;
    const int i0 = blockIdx.x * VTX, j0 = blockIdx.y * TYV;
    const int lane = threadIdx.x, wp = threadIdx.y;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const T* __restrict__ dg = static_cast<const T*>(op.dg);
    stage_rows<T, PH, XL, KIND, true>(sx, x, b, ca, cz, nx, ny, i0, j0, -1, lane, wp);
    if constexpr (NUT)
        stage_rows<T, PH, XL, KIND, false>(sa, a, b, ca, cz, nx, ny, i0, j0, -1, lane, wp);
    const int c0 = 4 + 4 * lane, i = i0 + 4 * lane;
    EpiPre<T> pre[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        const int j = j0 + wp * RW + k;
        if (i < nx && j <= ny) pre[k] = epi_prefetch<T, EPI, KIND>(b, ca, (size_t)j * nx + i, ny, j, c1);
    }
    cp_async_wait_all();
    __syncthreads();
    const Lap5C<T> kc = vc.l5;
    const T gx = vc.gx, gy = vc.gy;
    EpiAcc<T> acc;
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        const int o = wp * RW + k, j = j0 + o;
        const Vec4<T> xs = ld4(&sx[o][c0]), xc = ld4(&sx[o + 1][c0]), xn = ld4(&sx[o + 2][c0]);
        T xw = shfl_up1(xc.v[3]), xe = shfl_dn1(xc.v[0]);
        if (lane == 0) xw = sx[o + 1][3];
        if (lane == 31) xe = sx[o + 1][c0 + 4];
        Vec4<T> as{}, ac{}, an{};
        T aw = 0, ae = 0;
        if constexpr (NUT) {
            as = ld4(&sa[o][c0]);
            ac = ld4(&sa[o + 1][c0]);
            an = ld4(&sa[o + 2][c0]);
            aw = shfl_up1(ac.v[3]);
            ae = shfl_dn1(ac.v[0]);
            if (lane == 0) aw = sa[o + 1][3];
            if (lane == 31) ae = sa[o + 1][c0 + 4];
        }
        if (i >= nx || j > ny) continue;
        const size_t e = (size_t)j * nx + i;
        const bool wall = j == 0 || j == ny;
        Vec4<T> ax;
        if (KIND == OP_LAP5_DIRICHLET && wall) {
            if (CH && ca.dirichlet_zero) {
                st4(y + e, Vec4<T>{{(T)0, (T)0, (T)0, (T)0}});
                continue;
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) ax.v[m] = mul_rn(kc.c0, xc.v[m]);
        } else if (NUT && op.nut_dtop && j == ny) {
            if (CH && dz_row(ca.dirichlet_zero, j, ny)) {
                st4(y + e, Vec4<T>{{(T)0, (T)0, (T)0, (T)0}});
                continue;
            }
            const Vec4<T> dd = ld4(dg + e);
#pragma unroll
            for (int m = 0; m < 4; ++m) ax.v[m] = mul_rn(dd.v[m], xc.v[m]);
        } else if (NUT) {
            const Vec4<T> dd = ld4(dg + e);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const T xcm = xc.v[m];
                const T xwm = m == 0 ? xw : xc.v[m - 1], xem = m == 3 ? xe : xc.v[m + 1];
                const T awm = m == 0 ? aw : ac.v[m - 1], aem = m == 3 ? ae : ac.v[m + 1];
                const T acm = ac.v[m];
                const T ce = acm + aem, cw = acm + awm;
                const T cn = acm + an.v[m], cs = acm + as.v[m];
                const T sxv = fma(ce, xcm - xem, mul_rn(cw, xcm - xwm));
                const T syv = fma(cn, xcm - xn.v[m], mul_rn(cs, xcm - xs.v[m]));
                ax.v[m] = fma(gx, sxv, fma(gy, syv, mul_rn(dd.v[m], xcm)));
            }
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const T xwm = m == 0 ? xw : xc.v[m - 1], xem = m == 3 ? xe : xc.v[m + 1];
                ax.v[m] = lap5_ax(kc, xc.v[m], xwm, xem, xs.v[m], xn.v[m]);
            }
        }
        epi4<T, EPI>(ax, xc, pre[k], y, e, wall ? (T)0.5 : (T)1, acc, ca, c1, c2);
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

// ------------------------------------------------------------- 13-point
template <typename T, int EPI, int XL, int TYV>
__global__ void __launch_bounds__(128) k_ch13v(Op op, VConst<T> vc, const T* __restrict__ x,
                                               const T* __restrict__ b, T* __restrict__ y,
                                               SolveDev sd, const int* __restrict__ gate,
                                               double rtol, ChebArgs<T> ca) {
    if (gate && *gate) return;
    constexpr int RW = TYV / 4, XH = TYV + 4, PH = TYV + 2;
    constexpr bool CH = EPI == EPI_CHEB || EPI == EPI_CHEB_Z;
    __shared__ __align__(16) T sx[XH][VXW];   // x, rows j0 - 2 .. j0 + TYV + 1
    __shared__ __align__(16) T sa[PH][VXW];   // a, rows j0 - 1 .. j0 + TYV
    __shared__ __align__(16) T sp[PH][VXW];   // psi, rows j0 - 1 .. j0 + TYV
    T c1 = 0, c2 = 0, cz = 0;
    if (CH) cheb_consts(ca, c1, c2);
    if (XL == XL_ZERO) cz = (T)ca.coef[1];
    const int nx = op.g.nx, ny = op.g.ny;
    const int i0 = blockIdx.x * VTX, j0 = blockIdx.y * TYV;
    const int lane = threadIdx.x, wp = threadIdx.y, t = lane + 32 * wp;
    const T* __restrict__ a = static_cast<const T*>(op.a);
    stage_rows<T, PH, XL, OP_CH13, false>(sa, a, b, ca, cz, nx, ny, i0, j0, -1, lane, wp);
    stage_rows<T, XH, XL, OP_CH13, true>(sx, x, b, ca, cz, nx, ny, i0, j0, -2, lane, wp);
    EpiPre<T> pre[RW];
    {
        const int ip = i0 + 4 * lane;
#pragma unroll
        for (int k = 0; k < RW; ++k) {
            const int j = j0 + wp * RW + k;
            if (ip < nx && j <= ny)
                pre[k] = epi_prefetch<T, EPI, OP_CH13>(b, ca, (size_t)j * nx + ip, ny, j, c1);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // psi = kappa L_h x + S x on rows j0 - 1 .. j0 + TYV, columns i0 - 1 .. i0 + 128
    const T kx = vc.kx, ky = vc.ky, S = vc.S;
    const T kcc = vc.kcc;
    auto psi_val = [&](T c, T v0, T v2, T h0, T h2) {
        if (sizeof(T) == 4)
            return fma(ky, (c - v0) + (c - v2), fma(kx, (c - h0) + (c - h2), mul_rn(S, c)));
        return fma(-ky, v0 + v2, fma(-kx, h0 + h2, mul_rn(kcc, c)));
    };
    const int c0 = 4 + 4 * lane;
    {
        const int pr0 = (wp * PH) / 4, pr1 = ((wp + 1) * PH) / 4;
        Vec4<T> up = ld4(&sx[pr0][c0]), cen = ld4(&sx[pr0 + 1][c0]);
        for (int pr = pr0; pr < pr1; ++pr) {
            const Vec4<T> dn = ld4(&sx[pr + 2][c0]);
            T left = shfl_up1(cen.v[3]), right = shfl_dn1(cen.v[0]);
            if (lane == 0) left = sx[pr + 1][3];
            if (lane == 31) right = sx[pr + 1][c0 + 4];
            Vec4<T> ps;
            if (sizeof(T) == 4) {
                // west differences x_m - x_{m-1}; (c - h0) + (c - h2) = E_m - E_{m+1}
                T E[5];
                E[0] = cen.v[0] - left;
#pragma unroll
                for (int m = 1; m < 4; ++m) E[m] = cen.v[m] - cen.v[m - 1];
                E[4] = right - cen.v[3];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const T c = cen.v[m];
                    ps.v[m] = fma(ky, (c - up.v[m]) + (c - dn.v[m]),
                                  fma(kx, E[m] - E[m + 1], mul_rn(S, c)));
                }
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const T h0 = m == 0 ? left : cen.v[m - 1], h2 = m == 3 ? right : cen.v[m + 1];
                    ps.v[m] = psi_val(cen.v[m], up.v[m], dn.v[m], h0, h2);
                }
            }
            st4(&sp[pr][c0], ps);
            up = cen;
            cen = dn;
        }
        if (t < 2 * PH) {   // the ring columns i0 - 1 and i0 + 128
            const int pr = t < PH ? t : t - PH, cc = t < PH ? 3 : 4 + VTX;
            sp[pr][cc] = psi_val(sx[pr + 1][cc], sx[pr][cc], sx[pr + 2][cc], sx[pr + 1][cc - 1],
                                 sx[pr + 1][cc + 1]);
        }
    }
    __syncthreads();
    // y = idt x + 1/2 G_a psi (face means of a: the factor 1/4 in gxq, gyq)
    const T gxq = vc.gxq, gyq = vc.gyq;
    const T idt = vc.idt;
    EpiAcc<T> acc;
    const int i = i0 + 4 * lane;
    const int ob = wp * RW;   // first output row of this thread (tile-relative)
    // psi and a of rows ob (south of the first row) and ob + 1 (its centre)
    Vec4<T> pC = ld4(&sp[ob + 1][c0]), aC = ld4(&sa[ob + 1][c0]);
    T sS[4], dS[4];   // south face of the current row: a_c + a_s, p_c - p_s
    {
        const Vec4<T> pS = ld4(&sp[ob][c0]), aS = ld4(&sa[ob][c0]);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            sS[m] = aC.v[m] + aS.v[m];
            dS[m] = pC.v[m] - pS.v[m];
        }
    }
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        const int o = ob + k, j = j0 + o;
        const Vec4<T> pN = ld4(&sp[o + 2][c0]), aN = ld4(&sa[o + 2][c0]);
        T pw = shfl_up1(pC.v[3]), pe = shfl_dn1(pC.v[0]);
        T aw = shfl_up1(aC.v[3]), ae = shfl_dn1(aC.v[0]);
        if (lane == 0) {
            pw = sp[o + 1][3];
            aw = sa[o + 1][3];
        }
        if (lane == 31) {
            pe = sp[o + 1][c0 + 4];
            ae = sa[o + 1][c0 + 4];
        }
        // face f lies between nodes f - 1 and f (node -1: pw/aw, node 4: pe/ae)
        T sF[5], dF[5];
        sF[0] = aC.v[0] + aw;
        dF[0] = pC.v[0] - pw;
#pragma unroll
        for (int f = 1; f < 4; ++f) {
            sF[f] = aC.v[f - 1] + aC.v[f];
            dF[f] = pC.v[f] - pC.v[f - 1];
        }
        sF[4] = aC.v[3] + ae;
        dF[4] = pe - pC.v[3];
        const Vec4<T> xc = ld4(&sx[o + 2][c0]);
        Vec4<T> ax;
        T sN[4], dN[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            sN[m] = aC.v[m] + aN.v[m];
            dN[m] = pN.v[m] - pC.v[m];
            const T fx = fma(sF[m + 1], dF[m + 1], -mul_rn(sF[m], dF[m]));
            const T fy = fma(sN[m], dN[m], -mul_rn(sS[m], dS[m]));
            ax.v[m] = fma(-gyq, fy, fma(-gxq, fx, mul_rn(idt, xc.v[m])));
        }
        if (i < nx && j <= ny) {
            const size_t e = (size_t)j * nx + i;
            epi4<T, EPI>(ax, xc, pre[k], y, e, (j == 0 || j == ny) ? (T)0.5 : (T)1, acc, ca, c1,
                         c2);
        }
        pC = pN;
        aC = aN;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            sS[m] = sN[m];
            dS[m] = dN[m];
        }
    }
    epi_finish<T, EPI>(acc, sd, rtol);
}

// ------------------------------------------------------------- dispatch
namespace {
// CAHN_VEC=0 in the environment keeps every grid on the general tiles
// (read at each launch, so a test can compare the two families in one process)
bool vec_disabled() {
    const char* e = std::getenv("CAHN_VEC");
    return e && e[0] == '0';
}
inline bool al16(const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }
}  // namespace

dim3 vec_grid(const Grid& g, int rows) {
    return dim3((unsigned)((g.nx + VTX - 1) / VTX), (unsigned)((g.ny + 1 + rows - 1) / rows));
}

template <typename T>
bool vec_eligible(const Op& op, int epi, const void* x, const void* b, const void* y,
                  const ChebArgs<T>& ca, const SolveDev& sd) {
    if (vec_disabled()) return false;
    if (op.kind != OP_LAP5_NEUMANN && op.kind != OP_LAP5_DIRICHLET && op.kind != OP_NUT5 &&
        op.kind != OP_CH13)
        return false;
    if (op.g.nx < VTX || op.g.nx % 4 != 0) return false;
    if (!al16(x) || !al16(b) || !al16(y) || !al16(op.a) || !al16(op.dg) || !al16(ca.dinv) ||
        !al16(ca.d))
        return false;
    const bool reduces = epi == EPI_RESID || epi == EPI_RESIDX || epi == EPI_DOTXY ||
                         epi == EPI_NORM || epi == EPI_CGCG;
    if (reduces) {
        const dim3 gr = vec_grid(op.g, VRows<T>::value);
        if ((long)gr.x * gr.y > (long)sd.red.stride) return false;
    }
    return true;
}

template <typename T, int EPI, int XL, int TYV>
static void launch_vec_ty(const Op& op, const T* x, const T* b, T* y, SolveDev sd,
                          const int* gate, double rtol, cudaStream_t s, const ChebArgs<T>& ca) {
    const dim3 grid = vec_grid(op.g, TYV), blk(32, 4);
    const VConst<T> vc = vconst<T>(op);
    note_launch();
    switch (op.kind) {
        case OP_LAP5_NEUMANN:
            launch_k(k_lap5v<T, OP_LAP5_NEUMANN, EPI, XL, TYV>, grid, blk, 0, s, op, vc, x, b, y, sd, gate, rtol, ca);
            break;
        case OP_LAP5_DIRICHLET:
            launch_k(k_lap5v<T, OP_LAP5_DIRICHLET, EPI, XL, TYV>, grid, blk, 0, s, op, vc, x, b, y, sd, gate, rtol, ca);
            break;
        case OP_NUT5:
            launch_k(k_lap5v<T, OP_NUT5, EPI, XL, TYV>, grid, blk, 0, s, op, vc, x, b, y, sd, gate, rtol, ca);
            break;
        default:
            launch_k(k_ch13v<T, EPI, XL, TYV>, grid, blk, 0, s, op, vc, x, b, y, sd, gate, rtol, ca);
            break;
    }
}

// Launches with reductions keep the default tile (their summation order is
// fixed per grid); the others follow the operator's tuned tile height
// (op.ty = 8 takes the 8-row FP32 tile: twice the blocks on small grids).
template <typename T, int EPI, int XL>
void launch_vec(const Op& op, const T* x, const T* b, T* y, SolveDev sd, const int* gate,
                double rtol, cudaStream_t s, const ChebArgs<T>& ca) {
    constexpr bool RED = EPI == EPI_RESID || EPI == EPI_RESIDX || EPI == EPI_DOTXY ||
                         EPI == EPI_NORM || EPI == EPI_CGCG;
    if constexpr (sizeof(T) == 4 && !RED) {
        if (op.ty == 8) {
            launch_vec_ty<T, EPI, XL, 8>(op, x, b, y, sd, gate, rtol, s, ca);
            return;
        }
    }
    launch_vec_ty<T, EPI, XL, VRows<T>::value>(op, x, b, y, sd, gate, rtol, s, ca);
}

#define CAHN_VEC_INST(T)                                                                     \
    template bool vec_eligible<T>(const Op&, int, const void*, const void*, const void*,      \
                                  const ChebArgs<T>&, const SolveDev&);                       \
    template void launch_vec<T, EPI_APPLY, XL_PLAIN>(const Op&, const T*, const T*, T*,       \
                                                     SolveDev, const int*, double,            \
                                                     cudaStream_t, const ChebArgs<T>&);       \
    template void launch_vec<T, EPI_RESID, XL_PLAIN>(const Op&, const T*, const T*, T*,       \
                                                     SolveDev, const int*, double,            \
                                                     cudaStream_t, const ChebArgs<T>&);       \
    template void launch_vec<T, EPI_RESIDX, XL_PLAIN>(const Op&, const T*, const T*, T*,      \
                                                      SolveDev, const int*, double,           \
                                                      cudaStream_t, const ChebArgs<T>&);      \
    template void launch_vec<T, EPI_DOTXY, XL_PLAIN>(const Op&, const T*, const T*, T*,       \
                                                     SolveDev, const int*, double,            \
                                                     cudaStream_t, const ChebArgs<T>&);       \
    template void launch_vec<T, EPI_CGCG, XL_PLAIN>(const Op&, const T*, const T*, T*,        \
                                                    SolveDev, const int*, double,             \
                                                    cudaStream_t, const ChebArgs<T>&);        \
    template void launch_vec<T, EPI_NORM, XL_PLAIN>(const Op&, const T*, const T*, T*,        \
                                                    SolveDev, const int*, double,             \
                                                    cudaStream_t, const ChebArgs<T>&);        \
    template void launch_vec<T, EPI_RPLAIN, XL_PLAIN>(const Op&, const T*, const T*, T*,      \
                                                      SolveDev, const int*, double,           \
                                                      cudaStream_t, const ChebArgs<T>&);      \
    template void launch_vec<T, EPI_CHEB, XL_PLAIN>(const Op&, const T*, const T*, T*,        \
                                                    SolveDev, const int*, double,             \
                                                    cudaStream_t, const ChebArgs<T>&);        \
    template void launch_vec<T, EPI_CHEB, XL_PROLONG>(const Op&, const T*, const T*, T*,      \
                                                      SolveDev, const int*, double,           \
                                                      cudaStream_t, const ChebArgs<T>&);      \
    template void launch_vec<T, EPI_CHEB_Z, XL_ZERO>(const Op&, const T*, const T*, T*,       \
                                                     SolveDev, const int*, double,            \
                                                     cudaStream_t, const ChebArgs<T>&);
CAHN_VEC_INST(float)
CAHN_VEC_INST(double)

}  // namespace cahn
