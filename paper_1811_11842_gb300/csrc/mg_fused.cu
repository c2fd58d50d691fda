// Temporally blocked multigrid passes for the FP32 hierarchies of the
// 5-point operators (L_h with zero flux, H with Dirichlet walls) and of the
// 13-point phase-field operator.  Each block stages its tile of the level
// and a halo of H nodes in shared memory once, then runs several
// Chebyshev-Jacobi steps on it, the valid region shrinking by the stencil's
// reach per step (not at a wall, where the neighbour rows are rows of the
// tile), so that one launch does what the separate launches do level by
// level:
//   FUSED_DOWN:   steps 0 .. deg-1 from x = 0 (step 0, x = c D^-1 b, formed
//                 at staging), the residual b - A x on the tile and a
//                 one-node ring, and its restriction R (b - A x) to the
//                 coarse nodes of the tile; writes x and the coarse
//                 right-hand side.
//   FUSED_UP:     x + P x_c formed at staging, then steps 0 .. deg-1;
//                 writes x.
//   FUSED_COARSE: steps 0 .. k-1 from x = 0 on the coarsest level.
// Every node is evaluated with the operations of the separate launches
// (lap5_ax; psi and the face sums and differences of G_a as k_ch13 /
// k_ch13v; the step formulas of epi_node; prolong_at; restrict_at), so the
// V-cycle's result is bit for bit theirs; only the redundant halo nodes are
// extra work.
//
// Layout and work split.  A staged row is W = 128, 64 or 32 nodes (the tile
// is W - 2H wide, so the halo rides in the same row), stored with four pad
// columns on each side.  A thread computes four consecutive nodes of a row
// at once, in packed FP32 pairs: float4 shared-memory loads of the row and
// its neighbour rows, the x-neighbours of the four from the lanes beside it
// by warp shuffles; so a warp covers a 128-node row, two 64-node rows or four
// 32-node rows per instruction.  A step computes every group of four that
// meets its valid region: the few nodes of an edge group outside the region
// get values that nothing valid reads, which is cheaper than masking.
#include "mg_fused.h"
#include "stencil_dev.cuh"

namespace cahn {

// 4-byte asynchronous copy global -> shared (every copy of a block in flight
// at once; completed by cp_async_wait4 and a barrier)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait4() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// warps per block: the 5-point passes 8, the 13-point passes 16 (measured:
// the 13-point pass, held to two blocks per SM by its shared memory, hides
// its shared-memory latency better with more warps; the 5-point pass runs
// four blocks of 8)
constexpr int FUSED_WARPS5 = 8, FUSED_WARPS13 = 16;

struct F4 {
    float v[4];
};
__device__ __forceinline__ F4 lds4(const float* p) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void sts4(float* p, const F4& a) {
    *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// Four-node arithmetic in packed FP32 pairs (PTX add/sub/mul/fma.rn.f32x2):
// each lane rounds as the scalar instruction does, so the nodes get the bits
// of the scalar evaluation in half the arithmetic instructions.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(unsigned long long r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
#define CAHN_PAIR_OP2(NAME, OP)                                                          \
    __device__ __forceinline__ F4 NAME(const F4& a, const F4& b) {                      \
        unsigned long long lo, hi;                                                      \
        asm(OP " %0, %1, %2;" : "=l"(lo) : "l"(pk2(a.v[0], a.v[1])), "l"(pk2(b.v[0], b.v[1]))); \
        asm(OP " %0, %1, %2;" : "=l"(hi) : "l"(pk2(a.v[2], a.v[3])), "l"(pk2(b.v[2], b.v[3]))); \
        F4 r;                                                                           \
        up2(lo, r.v[0], r.v[1]);                                                        \
        up2(hi, r.v[2], r.v[3]);                                                        \
        return r;                                                                       \
    }
CAHN_PAIR_OP2(add4, "add.rn.f32x2")
CAHN_PAIR_OP2(sub4, "sub.rn.f32x2")
CAHN_PAIR_OP2(mul4, "mul.rn.f32x2")
#undef CAHN_PAIR_OP2
__device__ __forceinline__ F4 fma4(const F4& a, const F4& b, const F4& c) {
    unsigned long long lo, hi;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(lo)
        : "l"(pk2(a.v[0], a.v[1])), "l"(pk2(b.v[0], b.v[1])), "l"(pk2(c.v[0], c.v[1])));
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(hi)
        : "l"(pk2(a.v[2], a.v[3])), "l"(pk2(b.v[2], b.v[3])), "l"(pk2(c.v[2], c.v[3])));
    F4 r;
    up2(lo, r.v[0], r.v[1]);
    up2(hi, r.v[2], r.v[3]);
    return r;
}
__device__ __forceinline__ F4 bc4(float a) { return F4{{a, a, a, a}}; }
// the x-neighbours of four consecutive nodes: west (left, x0, x1, x2), east (x1, x2, x3, right)
__device__ __forceinline__ F4 west4(const F4& x, float left) { return F4{{left, x.v[0], x.v[1], x.v[2]}}; }
__device__ __forceinline__ F4 east4(const F4& x, float right) { return F4{{x.v[1], x.v[2], x.v[3], right}}; }
// The x-neighbours of a thread's four nodes, from the lanes beside it: the
// lane before holds the column left of the group, the lane after the column
// right of it (lane = g + G ro, group g of row ro).  For group 0 and group
// G-1 the value comes from another row or from the lane itself; it feeds
// only the frame's outermost columns, which no valid region reaches (every
// pass has a halo of at least one node).  All 32 lanes must call these.
__device__ __forceinline__ float left_of(const F4& x) {
    return __shfl_up_sync(0xffffffffu, x.v[3], 1);
}
__device__ __forceinline__ float right_of(const F4& x) {
    return __shfl_down_sync(0xffffffffu, x.v[0], 1);
}

// Rows lo..hi of the frame over the block's warps, R rows per warp
// instruction (one per lane group ro).  Every lane of a warp runs the same
// iterations, as the shuffles need; a lane whose row is past hi works on row
// hi and must not store (ok = false).
template <int NW, int R, typename Body>
__device__ __forceinline__ void for_rows(int lo, int hi, int wp, int ro, Body&& body) {
    for (int base = lo + wp * R; base <= hi; base += NW * R) {
        const int ly = base + ro;
        body(ly <= hi ? ly : hi, ly <= hi);
    }
}

// lap5_ax (FP32) of four nodes
__device__ __forceinline__ F4 lap5_ax4(const Lap5C<float>& k, const F4& c, const F4& w, const F4& e,
                                       const F4& s, const F4& n) {
    return fma4(bc4(k.cy), add4(sub4(c, s), sub4(c, n)),
                fma4(bc4(k.cx), add4(sub4(c, w), sub4(c, e)), mul4(bc4(k.c0), c)));
}

// Staged frame of a block: W nodes per row (the tile TX = W - 2H wide and a
// halo of H on each side), TY + 2H rows, row stride W + 8 (four pad columns
// each side; node lx of a row at offset 4 + lx).
template <int W, int TY, int H>
struct Frame {
    static constexpr int TX = W - 2 * H;
    static constexpr int SY = TY + 2 * H;
    static constexpr int RS = W + 8;
    static constexpr int SN = SY * RS;
    static constexpr int G = W / 4;      // groups of four per row
    static constexpr int R = 32 / G;     // rows per warp instruction
};

template <int MODE, int STEPS, int REACH>
struct FusedShape {
    static constexpr int K0 = MODE == FUSED_UP ? 0 : 1;   // first stencil step
    static constexpr int NST = STEPS - K0;                // stencil steps
    // FUSED_DOWN: the residual on the tile and a one-node ring needs x on the
    // tile + REACH + 1
    static constexpr int H = REACH * NST + (MODE == FUSED_DOWN ? REACH + 1 : 0);
};

// Per-block row bounds: staged rows ly in [lo, hi] hold rows j0 - H + ly of
// the level; wall_lo / wall_hi: the first / last staged row is a wall row.
struct RowSpan {
    int lo, hi;
    bool wall_lo, wall_hi;
    __device__ RowSpan(int j0, int ny, int H, int SY) {
        lo = max(0, H - j0);
        hi = min(SY - 1, ny - j0 + H);
        wall_lo = j0 - H + lo == 0;
        wall_hi = j0 - H + hi == ny;
    }
    // rows of the region shrunk by sh (not at a wall)
    __device__ int rlo(int sh) const { return wall_lo ? lo : lo + sh; }
    __device__ int rhi(int sh) const { return wall_hi ? hi : hi - sh; }
};

// The level columns of this lane's staged columns lx = lane + 32 c (the
// frame wraps periodically in x).
template <int W, int H>
struct LaneCols {
    static constexpr int C = W / 32 > 0 ? W / 32 : 1;
    int col[C];
    __device__ LaneCols(int i0, int nx) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            int i = (i0 - H + (int)threadIdx.x + 32 * c) % nx;
            col[c] = i < 0 ? i + nx : i;
        }
    }
};

// Zero the pad columns of nbase arrays from base, then stage narr arrays
// (src[k] -> dst[k]) of the frame by asynchronous copies: warps over rows,
// lanes over columns.
template <int NW, int W, int TY, int H, int N>
__device__ __forceinline__ void stage(float* const (&dst)[N], const float* const (&src)[N],
                                      int narr, float* base, int nbase, const RowSpan& rs,
                                      const LaneCols<W, H>& lc, int j0, int nx) {
    using F = Frame<W, TY, H>;
    const int lane = threadIdx.x, wp = threadIdx.y;
    if (lane < 8) {   // pads: columns 0..3 and W+4..W+7 of every row
        const int pc = lane < 4 ? lane : W + lane;
        for (int ly = wp; ly < F::SY; ly += NW)
            for (int a = 0; a < nbase; ++a) base[a * F::SN + ly * F::RS + pc] = 0.0f;
    }
    for (int ly = rs.lo + wp; ly <= rs.hi; ly += NW) {
        const size_t row = (size_t)(j0 - H + ly) * nx;
        const int o = ly * F::RS + 4 + lane;
#pragma unroll
        for (int c = 0; c < LaneCols<W, H>::C; ++c) {
            if (lane + 32 * c >= W) break;
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k < narr) cp_async4(dst[k] + o + 32 * c, src[k] + row + lc.col[c]);
        }
    }
    cp_async_wait4();
    __syncthreads();
}

// P x_c added to the staged x (FUSED_UP), lanes over columns
template <int NW, int W, int TY, int H>
__device__ __forceinline__ void add_prolong(float* sx, const ChebArgs<float>& ca, const RowSpan& rs,
                                            const LaneCols<W, H>& lc, int j0, int ny) {
    using F = Frame<W, TY, H>;
    const int lane = threadIdx.x;
    for (int ly = rs.lo + (int)threadIdx.y; ly <= rs.hi; ly += NW) {
        const int j = j0 - H + ly;
#pragma unroll
        for (int c = 0; c < LaneCols<W, H>::C; ++c) {
            if (lane + 32 * c >= W) break;
            sx[ly * F::RS + 4 + lane + 32 * c] += prolong_at(ca, ny, lc.col[c], j);
        }
    }
}

// Restriction of the residual held in sd (frame layout) to the coarse nodes
// whose centre 2J (2I) lies in the tile: warps over coarse rows, each lane
// four consecutive coarse nodes, each node summed in restrict_at's order.
template <int NW, int W, int TY, int H>
__device__ __forceinline__ void restrict_tile(const float* sd, const FusedPass<float>& fp, int i0,
                                              int j0, int ny, int dz) {
    using F = Frame<W, TY, H>;
    const Grid gc = fp.gc;
    const int semi = fp.semi;
    const int J0 = j0 / 2, J1 = min((j0 + TY) / 2, gc.ny + 1);
    const int I0 = semi ? i0 : i0 / 2, I1 = min(semi ? i0 + F::TX : (i0 + F::TX) / 2, gc.nx);
    for (int J = J0 + (int)threadIdx.y; J < J1; J += NW) {
        float* brow = fp.bc + (size_t)J * gc.nx;
        if (dz_row(dz, J, gc.ny)) {
            for (int I = I0 + (int)threadIdx.x; I < I1; I += 32) brow[I] = 0.0f;
            continue;
        }
        for (int q = I0 + 4 * (int)threadIdx.x; q < I1; q += 128) {
            float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int j = 2 * J + dy;
                if (j < 0 || j > ny) continue;
                const float wy = (dy == 0 ? 1.0f : 0.5f) * ((j == 0 || j == ny) ? 0.5f : 1.0f);
                const float* r = sd + (j - j0 + H) * F::RS + 4 + H - i0;
                if (semi) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) sum[m] = fma(wy, r[q + m], sum[m]);
                } else {
                    const float* rc = r + 2 * q;
                    float v[9];
#pragma unroll
                    for (int t = 0; t < 9; ++t) v[t] = rc[t - 1];
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        sum[m] = fma(wy, fma(0.5f, v[2 * m] + v[2 * m + 2], v[2 * m + 1]), sum[m]);
                }
            }
            const float scale = (semi ? 0.5f : 0.25f) * ((J == 0 || J == gc.ny) ? 2.0f : 1.0f);
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (q + m < I1) brow[q + m] = sum[m] * scale;
        }
    }
}

// x on the tile (frame -> level array)
template <int NW, int W, int TY, int H>
__device__ __forceinline__ void write_tile(const float* xf, float* xg, const RowSpan& rs, int i0,
                                           int j0, int nx) {
    using F = Frame<W, TY, H>;
    for (int ly = max(H, rs.lo) + (int)threadIdx.y; ly < H + TY && ly <= rs.hi; ly += NW) {
        const size_t row = (size_t)(j0 - H + ly) * nx;
        for (int c = (int)threadIdx.x; c < F::TX; c += 32)
            if (i0 + c < nx) xg[row + i0 + c] = xf[ly * F::RS + 4 + H + c];
    }
}

// ------------------------------------------------------------------ 5-point
template <int KIND, int MODE, int W, int TY, int STEPS>
__global__ void __launch_bounds__(32 * FUSED_WARPS5) k_mg_fused(FusedPass<float> fp, const int* __restrict__ gate) {
    constexpr int NW = FUSED_WARPS5;
    if (gate && *gate) return;
    using S = FusedShape<MODE, STEPS, 1>;
    constexpr int H = S::H, NST = S::NST, K0 = S::K0;
    using F = Frame<W, TY, H>;
    constexpr int RS = F::RS, G = F::G, R = F::R;
    extern __shared__ __align__(16) unsigned char fsm[];
    float* sb = reinterpret_cast<float*>(fsm);   // b
    float* s0 = sb + F::SN;                      // ping-pong iterates
    float* s1 = s0 + F::SN;
    float* sd = s1 + F::SN;                      // direction d (then the residual)
    const int nx = fp.op.g.nx, ny = fp.op.g.ny;
    const int i0 = blockIdx.x * F::TX, j0 = blockIdx.y * TY;
    const int lane = threadIdx.x, wp = threadIdx.y, nw = NW;
    const int g = lane % G, ro = lane / G;       // this thread's group and row offset
    const ChebArgs<float>& ca = fp.ca;
    const Lap5C<float> kc = fp.kc;
    const int dz = ca.dirichlet_zero;
    auto di_of = [&](int j) {
        return (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) ? ca.di_wall : ca.di_int;
    };
    const RowSpan rs(j0, ny, H, F::SY);
    const LaneCols<W, H> lcol(i0, nx);
    {
        float* const dst[2] = {sb, s0};
        const float* const src[2] = {fp.b, fp.xin};
        stage<NW, W, TY, H, 2>(dst, src, MODE == FUSED_UP ? 2 : 1, sb, 4, rs, lcol, j0, nx);
    }
    // the first iterate: x_1 = c D^-1 b, or x + P x_c
    if (MODE == FUSED_UP) {
        add_prolong<NW, W, TY, H>(s0, ca, rs, lcol, j0, ny);
    } else {
        const float cz = fp.c2[0];
        for (int ly = rs.lo + wp * R + ro; ly <= rs.hi; ly += nw * R) {
            const float czdi = mul_rn(cz, di_of(j0 - H + ly));
            const int o = ly * RS + 4 + 4 * g;
            sts4(s0 + o, mul4(bc4(czdi), lds4(sb + o)));
        }
    }
    __syncthreads();
    // neighbour rows of ly (row j)
    auto nb_rows = [&](int ly, int j, int& lys, int& lyn) {
        if (KIND == OP_LAP5_NEUMANN) {
            lys = j > 0 ? ly - 1 : ly + 1;
            lyn = j < ny ? ly + 1 : ly - 1;
        } else {
            lys = ly - 1;
            lyn = ly + 1;
        }
    };
    // A x at the group at column col of row ly (level row j); the
    // x-neighbours by shuffles, so every lane of the warp calls it
    auto ax4 = [&](const float* x, int ly, int j, int col, bool wall, F4& xc) {
        const int o = ly * RS + col;
        xc = lds4(x + o);
        const float left = left_of(xc), right = right_of(xc);
        if (wall) return mul4(bc4(kc.c0), xc);
        int lys, lyn;
        nb_rows(ly, j, lys, lyn);
        const F4 xs = lds4(x + lys * RS + col), xn = lds4(x + lyn * RS + col);
        return lap5_ax4(kc, xc, west4(xc, left), east4(xc, right), xs, xn);
    };
    const int col = 4 + 4 * g;
    // ---- the stencil steps k = K0 .. STEPS-1 (s0 -> s1 -> s0 ...)
#pragma unroll
    for (int s = 1; s <= NST; ++s) {
        const int k = K0 + s - 1;
        const bool zero = MODE != FUSED_UP && k == 1;   // d = x_1 (the step after the zero guess)
        const float* in = (s % 2 == 1) ? s0 : s1;
        float* out = (s % 2 == 1) ? s1 : s0;
        const float c1 = fp.c1[k], c2 = fp.c2[k];
        const bool cg = g >= s / 4 && g <= (W - s - 1) / 4;   // the group meets the region
        for_rows<NW, R>(rs.rlo(s), rs.rhi(s), wp, ro, [&](int ly, bool ok) {
            const int j = j0 - H + ly;
            const bool wall = KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny);
            const int o = ly * RS + col;
            const bool st = ok && cg;
            F4 xc;
            const F4 ax = ax4(in, ly, j, col, wall, xc);
            if (wall && dz) {
                if (st) sts4(out + o, F4{{0.0f, 0.0f, 0.0f, 0.0f}});
                return;
            }
            const F4 r = sub4(lds4(sb + o), ax);
            const F4 c2di = bc4(mul_rn(c2, di_of(j)));
            F4 dn;
            if (zero)
                dn = fma4(c2di, r, mul4(bc4(c1), xc));
            else if (c1 != 0.0f)
                dn = fma4(c2di, r, mul4(bc4(c1), lds4(sd + o)));
            else   // c1 = 0 at k = 0 (no direction yet)
                dn = fma4(c2di, r, bc4(0.0f));
            if (st) {
                sts4(sd + o, dn);
                sts4(out + o, add4(xc, dn));
            }
        });
        __syncthreads();
    }
    const float* xf = (NST % 2 == 1) ? s1 : s0;   // the last step's iterate
    write_tile<NW, W, TY, H>(xf, fp.xout, rs, i0, j0, nx);
    if constexpr (MODE == FUSED_DOWN) {
        // residual b - A x on the tile and a one-node ring
        const bool cg = g >= (H - 1) / 4 && g <= (H + F::TX) / 4;
        for_rows<NW, R>(max(H - 1, rs.lo), min(H + TY, rs.hi), wp, ro, [&](int ly, bool ok) {
            const int j = j0 - H + ly;
            const bool wall = KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny);
            F4 xc;
            const F4 ax = ax4(xf, ly, j, col, wall, xc);
            if (ok && cg) sts4(sd + ly * RS + col, sub4(lds4(sb + ly * RS + col), ax));
        });
        __syncthreads();
        restrict_tile<NW, W, TY, H>(sd, fp, i0, j0, ny, dz);
    }
}

// ---------------------------------------------------------------- 13-point
// A_phi = I/dt + 1/2 G_a (kappa L_h + S): each stencil application forms
// psi = kappa L_h x + S x on the region and a one-node ring, then A x from
// psi and the staged coefficient a, so the region shrinks by two nodes per
// step.  The iterate is updated in place (A x at a node reads x only at the
// node; its neighbours enter through psi, formed before).  D^-1 is the
// level's array (staged); the step table is read from the device, where the
// spectrum bound is refreshed every time step.
template <int MODE, int W, int TY, int STEPS>
__global__ void __launch_bounds__(32 * FUSED_WARPS13) k_mg_fused13(FusedPass<float> fp, const int* __restrict__ gate) {
    constexpr int NW = FUSED_WARPS13;
    if (gate && *gate) return;
    using S = FusedShape<MODE, STEPS, 2>;
    constexpr int H = S::H, NST = S::NST, K0 = S::K0;
    using F = Frame<W, TY, H>;
    constexpr int RS = F::RS, G = F::G, R = F::R;
    extern __shared__ __align__(16) unsigned char fsm[];
    float* sb = reinterpret_cast<float*>(fsm);   // b
    float* sa = sb + F::SN;                      // coefficient a
    float* sdi = sa + F::SN;                     // D^-1
    float* sx = sdi + F::SN;                     // the iterate (updated in place)
    float* sp = sx + F::SN;                      // psi
    float* sd = sp + F::SN;                      // direction d (then the residual)
    __shared__ float sc1[FUSED_MAXK], sc2[FUSED_MAXK];
    const int nx = fp.op.g.nx, ny = fp.op.g.ny;
    const int i0 = blockIdx.x * F::TX, j0 = blockIdx.y * TY;
    const int lane = threadIdx.x, wp = threadIdx.y, tid = lane + 32 * wp, nw = NW;
    const int g = lane % G, ro = lane / G;
    const ChebArgs<float>& ca = fp.ca;
    const C13<float> k = fp.k13;
    const Lap5C<float> kpsi{k.S, k.kx, k.ky, 0.0f};   // psi's coefficients in lap5_ax's roles
    if (tid < 2 * STEPS) {
        const float v = (float)ca.coef[tid];
        if (tid & 1) sc2[tid >> 1] = v;
        else sc1[tid >> 1] = v;
    }
    const RowSpan rs(j0, ny, H, F::SY);
    const LaneCols<W, H> lcol(i0, nx);
    {
        float* const dst[4] = {sb, sa, sdi, sx};
        const float* const src[4] = {fp.b, static_cast<const float*>(fp.op.a), ca.dinv, fp.xin};
        stage<NW, W, TY, H, 4>(dst, src, MODE == FUSED_UP ? 4 : 3, sb, 6, rs, lcol, j0, nx);
    }
    // the first iterate: x_1 = c D^-1 b, or x + P x_c
    if (MODE == FUSED_UP) {
        add_prolong<NW, W, TY, H>(sx, ca, rs, lcol, j0, ny);
    } else {
        const float cz = sc2[0];
        for (int ly = rs.lo + wp * R + ro; ly <= rs.hi; ly += nw * R) {
            const int o = ly * RS + 4 + 4 * g;
            sts4(sx + o, mul4(mul4(bc4(cz), lds4(sdi + o)), lds4(sb + o)));
        }
    }
    __syncthreads();
    // neighbour rows (zero flux: reflected at the walls)
    auto nb_rows = [&](int ly, int& lys, int& lyn) {
        const int j = j0 - H + ly;
        lys = j > 0 ? ly - 1 : ly + 1;
        lyn = j < ny ? ly + 1 : ly - 1;
    };
    const int col = 4 + 4 * g;
    // psi on the groups meeting the region shrunk by sh
    auto form_psi = [&](int sh) {
        const bool cg = g >= sh / 4 && g <= (W - sh - 1) / 4;
        for_rows<NW, R>(rs.rlo(sh), rs.rhi(sh), wp, ro, [&](int ly, bool ok) {
            int lys, lyn;
            nb_rows(ly, lys, lyn);
            const int o = ly * RS + col;
            const F4 xc = lds4(sx + o), xs = lds4(sx + lys * RS + col), xn = lds4(sx + lyn * RS + col);
            const float left = left_of(xc), right = right_of(xc);
            // psi = S x + kx (2 x - x_w - x_e) + ky (2 x - x_s - x_n), in lap5_ax's order
            const F4 ps = lap5_ax4(kpsi, xc, west4(xc, left), east4(xc, right), xs, xn);
            if (ok && cg) sts4(sp + o, ps);
        });
    };
    // A x at the group at column col of row ly from psi, a and x (the
    // x-neighbours by shuffles: every lane of the warp calls it)
    auto ax4 = [&](int ly, const F4& xc) {
        int lys, lyn;
        nb_rows(ly, lys, lyn);
        const int o = ly * RS + col;
        const F4 pc = lds4(sp + o), ac = lds4(sa + o);
        const F4 pS = lds4(sp + lys * RS + col), pN = lds4(sp + lyn * RS + col);
        const F4 aS = lds4(sa + lys * RS + col), aN = lds4(sa + lyn * RS + col);
        const float pw = left_of(pc), pe = right_of(pc), aw = left_of(ac), ae = right_of(ac);
        // fx = (a + a_E)(p_E - p) - (a + a_W)(p - p_W), the product subtracted
        // rounded alone (negated by -0 - y, exact), fy alike
        const F4 mz = bc4(-0.0f);
        const F4 fx = fma4(add4(ac, east4(ac, ae)), sub4(east4(pc, pe), pc),
                           sub4(mz, mul4(add4(ac, west4(ac, aw)), sub4(pc, west4(pc, pw)))));
        const F4 fy = fma4(add4(ac, aN), sub4(pN, pc), sub4(mz, mul4(add4(ac, aS), sub4(pc, pS))));
        return fma4(bc4(-k.gyq), fy, fma4(bc4(-k.gxq), fx, mul4(bc4(k.idt), xc)));
    };
#pragma unroll
    for (int s = 1; s <= NST; ++s) {
        const int kk = K0 + s - 1;
        const bool zero = MODE != FUSED_UP && kk == 1;
        form_psi(2 * s - 1);
        __syncthreads();
        const float c1 = sc1[kk], c2 = sc2[kk];
        const int sh = 2 * s;
        const bool cg = g >= sh / 4 && g <= (W - sh - 1) / 4;
        for_rows<NW, R>(rs.rlo(sh), rs.rhi(sh), wp, ro, [&](int ly, bool ok) {
            const int o = ly * RS + col;
            const F4 xc = lds4(sx + o);
            const F4 r = sub4(lds4(sb + o), ax4(ly, xc));
            const F4 c2di = mul4(bc4(c2), lds4(sdi + o));
            F4 dn;
            if (zero)
                dn = fma4(c2di, r, mul4(bc4(c1), xc));
            else if (c1 != 0.0f)
                dn = fma4(c2di, r, mul4(bc4(c1), lds4(sd + o)));
            else   // c1 = 0 at k = 0 (no direction yet)
                dn = fma4(c2di, r, bc4(0.0f));
            if (ok && cg) {   // in place: A x at a node reads x only there
                sts4(sd + o, dn);
                sts4(sx + o, add4(xc, dn));
            }
        });
        __syncthreads();
    }
    write_tile<NW, W, TY, H>(sx, fp.xout, rs, i0, j0, nx);
    if constexpr (MODE == FUSED_DOWN) {
        // residual b - A x on the tile and a one-node ring
        form_psi(2 * NST + 1);
        __syncthreads();
        const int sh = 2 * NST + 2;   // = H - 1
        const bool cg = g >= sh / 4 && g <= (W - sh - 1) / 4;
        for_rows<NW, R>(rs.rlo(sh), rs.rhi(sh), wp, ro, [&](int ly, bool ok) {
            const int o = ly * RS + col;
            const F4 rr = sub4(lds4(sb + o), ax4(ly, lds4(sx + o)));
            if (ok && cg) sts4(sd + o, rr);
        });
        __syncthreads();
        restrict_tile<NW, W, TY, H>(sd, fp, i0, j0, ny, 0);
    }
}

// ------------------------------------------------------------------ launch
// Staged row widths and tile heights a pass may take.
constexpr int FT_W[3] = {128, 64, 32}, FT_Y[3] = {16, 16, 8};

template <int W, int TY, int H, int NARR>
constexpr size_t frame_bytes() {
    return (size_t)NARR * Frame<W, TY, H>::SN * sizeof(float);
}

// Tile of a level: the widest whose grid still gives every SM a block (the
// narrower tiles recompute more halo nodes per output node); tiles whose
// halo leaves fewer than two columns are not used.
static int fused_tile(const Grid& g, int H) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CAHN_CUDA_TRY(cudaGetDevice(&dev));
        CAHN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    int t = 0;
    for (; t < 2; ++t) {
        const int tx = FT_W[t] - 2 * H;
        const long blocks = (long)((g.nx + tx - 1) / tx) * ((g.ny + 1 + FT_Y[t] - 1) / FT_Y[t]);
        if (blocks >= sms || FT_W[t + 1] - 2 * H < 2) return t;
    }
    return t;
}

template <int KIND, int MODE, int STEPS, int T>
static void launch_tile5(const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    constexpr int W = FT_W[T], TY = FT_Y[T], H = FusedShape<MODE, STEPS, 1>::H;
    if constexpr (W - 2 * H >= 2) {
        constexpr size_t smem = frame_bytes<W, TY, H, 4>();
        static_assert(smem <= FUSED_SMEM_MAX, "fused pass shared memory");
        auto k = k_mg_fused<KIND, MODE, W, TY, STEPS>;
        if (prep) {
            CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            return;
        }
        constexpr int TX = W - 2 * H;
        const dim3 grid((unsigned)((fp.op.g.nx + TX - 1) / TX), (unsigned)((fp.op.g.ny + 1 + TY - 1) / TY)),
            blk(32, FUSED_WARPS5);
        note_launch();
        launch_k(k, grid, blk, smem, s, fp, gate);
    } else {
        if (!prep) throw ArgError("fused multigrid pass: halo wider than the tile");
    }
}

template <int MODE, int STEPS, int T>
static void launch_tile13(const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    constexpr int W = FT_W[T], TY = FT_Y[T], H = FusedShape<MODE, STEPS, 2>::H;
    if constexpr (W - 2 * H >= 2) {
        constexpr size_t smem = frame_bytes<W, TY, H, 6>();
        static_assert(smem <= FUSED13_SMEM_MAX, "fused pass shared memory");
        auto k = k_mg_fused13<MODE, W, TY, STEPS>;
        if (prep) {
            CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            return;
        }
        constexpr int TX = W - 2 * H;
        const dim3 grid((unsigned)((fp.op.g.nx + TX - 1) / TX), (unsigned)((fp.op.g.ny + 1 + TY - 1) / TY)),
            blk(32, FUSED_WARPS13);
        note_launch();
        launch_k(k, grid, blk, smem, s, fp, gate);
    } else {
        if (!prep) throw ArgError("fused multigrid pass: halo wider than the tile");
    }
}

// one pass on the level's tile (prep: only opt the kernels of every tile in
// to their shared memory, no launch)
template <int KIND, int MODE, int STEPS>
static void launch5(const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    if (prep) {
        launch_tile5<KIND, MODE, STEPS, 0>(fp, gate, s, true);
        launch_tile5<KIND, MODE, STEPS, 1>(fp, gate, s, true);
        launch_tile5<KIND, MODE, STEPS, 2>(fp, gate, s, true);
        return;
    }
    switch (fused_tile(fp.op.g, FusedShape<MODE, STEPS, 1>::H)) {
        case 0: launch_tile5<KIND, MODE, STEPS, 0>(fp, gate, s, false); break;
        case 1: launch_tile5<KIND, MODE, STEPS, 1>(fp, gate, s, false); break;
        default: launch_tile5<KIND, MODE, STEPS, 2>(fp, gate, s, false); break;
    }
}

template <int MODE, int STEPS>
static void launch13(const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    if (prep) {
        launch_tile13<MODE, STEPS, 0>(fp, gate, s, true);
        launch_tile13<MODE, STEPS, 1>(fp, gate, s, true);
        launch_tile13<MODE, STEPS, 2>(fp, gate, s, true);
        return;
    }
    switch (fused_tile(fp.op.g, FusedShape<MODE, STEPS, 2>::H)) {
        case 0: launch_tile13<MODE, STEPS, 0>(fp, gate, s, false); break;
        case 1: launch_tile13<MODE, STEPS, 1>(fp, gate, s, false); break;
        default: launch_tile13<MODE, STEPS, 2>(fp, gate, s, false); break;
    }
}

// the smoother's degree fp.steps (FUSED_DEG_MIN .. FUSED_DEG_MAX)
template <int KIND, int MODE>
static void launch_deg5(const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    switch (fp.steps) {
        case 3: launch5<KIND, MODE, 3>(fp, gate, s, prep); break;
        case 4: launch5<KIND, MODE, 4>(fp, gate, s, prep); break;
        case 5: launch5<KIND, MODE, 5>(fp, gate, s, prep); break;
        default: throw ArgError("fused multigrid pass: unsupported smoother degree");
    }
}
template <int MODE>
static void launch_deg13(const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    switch (fp.steps) {
        case 3: launch13<MODE, 3>(fp, gate, s, prep); break;
        case 4: launch13<MODE, 4>(fp, gate, s, prep); break;
        case 5: launch13<MODE, 5>(fp, gate, s, prep); break;
        default: throw ArgError("fused multigrid pass: unsupported smoother degree");
    }
}

static void dispatch(int mode, const FusedPass<float>& fp, const int* gate, cudaStream_t s, bool prep) {
    const bool dir = fp.op.kind == OP_LAP5_DIRICHLET;
    if (mode == FUSED_COARSE && !fused_coarse_steps(fp.op.kind, fp.steps))
        throw ArgError("fused multigrid pass: unsupported coarse step count");
    if (fp.op.kind == OP_CH13) {
        switch (mode) {
            case FUSED_DOWN: launch_deg13<FUSED_DOWN>(fp, gate, s, prep); break;
            case FUSED_UP: launch_deg13<FUSED_UP>(fp, gate, s, prep); break;
            default:
                if (fp.steps == FUSED_COARSE_STEPS13) launch13<FUSED_COARSE, FUSED_COARSE_STEPS13>(fp, gate, s, prep);
                else launch13<FUSED_COARSE, FUSED_COARSE_STEPS>(fp, gate, s, prep);
                break;
        }
        return;
    }
    if (fp.op.kind != OP_LAP5_DIRICHLET && fp.op.kind != OP_LAP5_NEUMANN)
        throw ArgError("fused multigrid pass: 5-point and 13-point operators only");
    switch (mode) {
        case FUSED_DOWN:
            if (dir) launch_deg5<OP_LAP5_DIRICHLET, FUSED_DOWN>(fp, gate, s, prep);
            else launch_deg5<OP_LAP5_NEUMANN, FUSED_DOWN>(fp, gate, s, prep);
            break;
        case FUSED_UP:
            if (dir) launch_deg5<OP_LAP5_DIRICHLET, FUSED_UP>(fp, gate, s, prep);
            else launch_deg5<OP_LAP5_NEUMANN, FUSED_UP>(fp, gate, s, prep);
            break;
        default:
            if (dir) launch5<OP_LAP5_DIRICHLET, FUSED_COARSE, FUSED_COARSE_STEPS>(fp, gate, s, prep);
            else launch5<OP_LAP5_NEUMANN, FUSED_COARSE, FUSED_COARSE_STEPS>(fp, gate, s, prep);
            break;
    }
}

template <typename T>
void fused_prepare(int kind, int degree) {
    static_assert(sizeof(T) == 4, "fused passes: FP32 hierarchies");
    FusedPass<float> fp{};
    fp.op.kind = kind;
    fp.steps = degree;
    dispatch(FUSED_DOWN, fp, nullptr, nullptr, true);
    dispatch(FUSED_UP, fp, nullptr, nullptr, true);
    fp.steps = FUSED_COARSE_STEPS;
    dispatch(FUSED_COARSE, fp, nullptr, nullptr, true);
    if (kind == OP_CH13) {
        fp.steps = FUSED_COARSE_STEPS13;
        dispatch(FUSED_COARSE, fp, nullptr, nullptr, true);
    }
}

template <typename T>
void launch_fused(int mode, const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    static_assert(sizeof(T) == 4, "fused passes: FP32 hierarchies");
    dispatch(mode, fp, gate, s, false);
}

template void launch_fused<float>(int, const FusedPass<float>&, const int*, cudaStream_t);
template void fused_prepare<float>(int, int);

}  // namespace cahn
