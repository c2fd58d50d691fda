// Temporally blocked multigrid passes for the FP32 5-point hierarchies
// (L_h with zero flux, H with Dirichlet walls).  Each block stages its tile
// of the level and a halo of H nodes in shared memory once, then runs
// several Chebyshev-Jacobi steps on it, the region shrinking by one node per
// stencil application (not at a wall, where the neighbour rows are rows of
// the tile), so that one launch does what the separate launches do level by
// level:
//   FUSED_DOWN:   steps 0 .. deg-1 from x = 0 (step 0, x = c D^-1 b, formed
//                 in the staging), the residual b - A x on the tile and a
//                 one-node ring, and its restriction R (b - A x) to the
//                 coarse nodes of the tile; writes x and the coarse
//                 right-hand side.  H = deg + 1.
//   FUSED_UP:     x + P x_c formed in the staging, then steps 0 .. deg-1;
//                 writes x.  H = deg.
//   FUSED_COARSE: steps 0 .. k-1 from x = 0 on the coarsest level.
//                 H = k - 1.
// Every node is evaluated with the operations of the separate launches
// (lap5_ax, the step formulas of epi_node, prolong_at, restrict_at), so the
// V-cycle's result is bit for bit theirs; only the redundant halo nodes are
// extra work.  Tile, halo and step count are compile-time, so the loops over
// a row unroll and the per-row constants (D^-1 c2, the neighbour rows) are
// formed once per row.
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

template <int MODE, int STEPS>
struct FusedShape {
    static constexpr int K0 = MODE == FUSED_UP ? 0 : 1;         // first stencil step
    static constexpr int NST = STEPS - K0;                      // stencil steps
    static constexpr int H = NST + (MODE == FUSED_DOWN ? 2 : 0);   // halo
};

template <typename T, int KIND, int MODE, int TX, int TY, int STEPS>
__global__ void __launch_bounds__(256) k_mg_fused(FusedPass<T> fp, const int* __restrict__ gate) {
    if (gate && *gate) return;
    using S = FusedShape<MODE, STEPS>;
    constexpr int H = S::H, NST = S::NST, K0 = S::K0;
    constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SN = SX * SY;
    constexpr int CX = (SX + 31) / 32;   // 32-column chunks of a staged row
    extern __shared__ __align__(16) unsigned char fsm[];
    T* sb = reinterpret_cast<T*>(fsm);   // b on the staged region
    T* s0 = sb + SN;                     // ping-pong iterates
    T* s1 = s0 + SN;
    T* sd = s1 + SN;                     // Chebyshev direction d (then the residual)
    const Op& op = fp.op;
    const int nx = op.g.nx, ny = op.g.ny;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const ChebArgs<T>& ca = fp.ca;
    const Lap5C<T> kc = fp.kc;
    const int dz = ca.dirichlet_zero;
    auto di_of = [&](int j) {
        return (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) ? ca.di_wall : ca.di_int;
    };
    // staged rows: j = j0 - H + ly for ly in [ly_lo, ly_hi] (the rows 0 .. ny)
    const int ly_lo = max(0, H - j0), ly_hi = min(SY - 1, ny - j0 + H);
    const bool wall_lo = j0 - H + ly_lo == 0, wall_hi = j0 - H + ly_hi == ny;
    // ---- staging: b (and x for FUSED_UP) by asynchronous copies, every copy
    // of the block in flight at once; then the first iterate in place
    // (x_1 = c D^-1 b, or x + P x_c)
    for (int ly = ly_lo + ty; ly <= ly_hi; ly += 8) {
        const size_t row = (size_t)(j0 - H + ly) * nx;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            const int lx = tx + 32 * c;
            if (lx >= SX) break;
            int i = (i0 - H + lx) % nx;
            if (i < 0) i += nx;
            cp_async4(sb + ly * SX + lx, fp.b + row + i);
            if (MODE == FUSED_UP) cp_async4(s0 + ly * SX + lx, fp.xin + row + i);
        }
    }
    cp_async_wait4();
    __syncthreads();
    {
        const T cz = fp.c2[0];
        for (int ly = ly_lo + ty; ly <= ly_hi; ly += 8) {
            const int j = j0 - H + ly;
            const T czdi = mul_rn(cz, di_of(j));
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = tx + 32 * c;
                if (lx >= SX) break;
                if (MODE == FUSED_UP) {
                    int i = (i0 - H + lx) % nx;
                    if (i < 0) i += nx;
                    s0[ly * SX + lx] += prolong_at(ca, ny, i, j);
                } else {
                    s0[ly * SX + lx] = mul_rn(czdi, sb[ly * SX + lx]);
                }
            }
        }
    }
    __syncthreads();
    // ---- the stencil steps k = K0 .. STEPS-1 (in s0 -> s1 -> s0 ...)
#pragma unroll
    for (int s = 1; s <= NST; ++s) {
        const int k = K0 + s - 1;
        const bool zero = MODE != FUSED_UP && k == 1;   // d = x_1 (the step after the zero guess)
        const T* in = (s % 2 == 1) ? s0 : s1;
        T* out = (s % 2 == 1) ? s1 : s0;
        const T c1 = fp.c1[k], c2 = fp.c2[k];
        const int rlo = wall_lo ? ly_lo : ly_lo + s, rhi = wall_hi ? ly_hi : ly_hi - s;
        for (int ly = rlo + ty; ly <= rhi; ly += 8) {
            const int j = j0 - H + ly;
            const bool wall = KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny);
            int lys, lyn;
            if (KIND == OP_LAP5_NEUMANN) {
                lys = j > 0 ? ly - 1 : ly + 1;
                lyn = j < ny ? ly + 1 : ly - 1;
            } else {
                lys = ly - 1;
                lyn = ly + 1;
            }
            const T* ic = in + ly * SX;
            const T* is = in + lys * SX;
            const T* in_ = in + lyn * SX;
            const T* bc = sb + ly * SX;
            T* dc = sd + ly * SX;
            T* oc = out + ly * SX;
            const T c2di = mul_rn(c2, di_of(j));
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = tx + 32 * c;
                if (lx < s || lx >= SX - s) continue;
                const T xc = ic[lx];
                T ax;
                if (wall) {
                    if (dz) {
                        oc[lx] = (T)0;
                        continue;
                    }
                    ax = mul_rn(kc.c0, xc);
                } else {
                    ax = lap5_ax(kc, xc, ic[lx - 1], ic[lx + 1], is[lx], in_[lx]);
                }
                const T r = bc[lx] - ax;
                T dn;
                if (zero)
                    dn = fma(c2di, r, mul_rn(c1, xc));
                else   // c1 = 0 at k = 0 (no direction yet)
                    dn = fma(c2di, r, c1 != (T)0 ? mul_rn(c1, dc[lx]) : (T)0);
                dc[lx] = dn;
                oc[lx] = xc + dn;
            }
        }
        __syncthreads();
    }
    const T* xf = (NST % 2 == 1) ? s1 : s0;   // the last step's iterate
    // ---- x on the tile
    {
        T* xg = fp.xout;
        for (int ly = max(H, ly_lo) + ty; ly < H + TY && ly <= ly_hi; ly += 8) {
            const size_t row = (size_t)(j0 - H + ly) * nx;
#pragma unroll
            for (int c = 0; c < (TX + 31) / 32; ++c) {
                const int lx = H + tx + 32 * c;
                const int i = i0 + tx + 32 * c;
                if (lx < H + TX && i < nx) xg[row + i] = xf[ly * SX + lx];
            }
        }
    }
    if constexpr (MODE == FUSED_DOWN) {
        // residual b - A x on the tile and a one-node ring (k_resid_restrict's res)
        for (int ly = max(H - 1, ly_lo) + ty; ly <= H + TY && ly <= ly_hi; ly += 8) {
            const int j = j0 - H + ly;
            const bool wall = KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny);
            int lys, lyn;
            if (KIND == OP_LAP5_NEUMANN) {
                lys = j > 0 ? ly - 1 : ly + 1;
                lyn = j < ny ? ly + 1 : ly - 1;
            } else {
                lys = ly - 1;
                lyn = ly + 1;
            }
            const T* xc_ = xf + ly * SX;
            const T* xs_ = xf + lys * SX;
            const T* xn_ = xf + lyn * SX;
            const T* bc = sb + ly * SX;
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = H - 1 + tx + 32 * c;
                if (lx > H + TX) continue;
                const T xv = xc_[lx];
                const T ax = wall ? mul_rn(kc.c0, xv)
                                  : lap5_ax(kc, xv, xc_[lx - 1], xc_[lx + 1], xs_[lx], xn_[lx]);
                sd[ly * SX + lx] = bc[lx] - ax;
            }
        }
        __syncthreads();
        // restriction to the coarse nodes whose centre 2J (2I) lies in the tile
        const Grid gc = fp.gc;
        const int semi = fp.semi;
        const int J0 = j0 / 2, J1 = min((j0 + TY) / 2, gc.ny + 1);
        const int I0 = semi ? i0 : i0 / 2, I1 = min(semi ? i0 + TX : (i0 + TX) / 2, gc.nx);
        for (int J = J0 + ty; J < J1; J += 8) {
            for (int I = I0 + tx; I < I1; I += 32) {
                const size_t ec = (size_t)J * gc.nx + I;
                if (dz_row(dz, J, gc.ny)) {
                    fp.bc[ec] = (T)0;
                    continue;
                }
                const int lc = (semi ? I : 2 * I) - i0 + H;
                auto res = [&](int j, int dx) { return sd[(j - j0 + H) * SX + lc + dx]; };
                fp.bc[ec] = restrict_at<T>(res, J, ny, semi, gc.ny);
            }
        }
    }
}

// ---------------------------------------------------------- 13-point
// The same passes for the FP32 phase-field hierarchies (A_phi = I/dt +
// 1/2 G_a (kappa L_h + S)).  Each stencil application forms psi = kappa L_h x
// + S x on the region and a one-node ring, then A x from psi and the staged
// coefficient a: the region shrinks by two nodes per step.  The iterate is
// updated in place (A x at a node reads x only at the node; its neighbours
// enter through psi, formed before).  D^-1 is the level's array (staged);
// the step table is read from the device, where the spectrum bound is
// refreshed every time step.  Every node is evaluated with the operations
// of k_ch13 / k_ch13v (psi in the difference form, the face sums and
// differences of G_a), the step formulas, prolong_at and restrict_at.
template <int MODE, int STEPS>
struct Fused13Shape {
    static constexpr int K0 = MODE == FUSED_UP ? 0 : 1;
    static constexpr int NST = STEPS - K0;
    // FUSED_DOWN: the residual on the tile and a ring needs x on the tile + 3
    static constexpr int H = 2 * NST + (MODE == FUSED_DOWN ? 3 : 0);
};

template <typename T, int MODE, int TX, int TY, int STEPS>
__global__ void __launch_bounds__(256) k_mg_fused13(FusedPass<T> fp, const int* __restrict__ gate) {
    if (gate && *gate) return;
    using S = Fused13Shape<MODE, STEPS>;
    constexpr int H = S::H, NST = S::NST, K0 = S::K0;
    constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SN = SX * SY;
    constexpr int CX = (SX + 31) / 32;
    extern __shared__ __align__(16) unsigned char fsm[];
    T* sb = reinterpret_cast<T*>(fsm);   // b
    T* sa = sb + SN;                     // coefficient a
    T* sdi = sa + SN;                    // D^-1
    T* sx = sdi + SN;                    // the iterate (updated in place)
    T* sp = sx + SN;                     // psi
    T* sd = sp + SN;                     // Chebyshev direction d (then the residual)
    __shared__ T sc1[FUSED_MAXK], sc2[FUSED_MAXK];
    const Op& op = fp.op;
    const int nx = op.g.nx, ny = op.g.ny;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int tid = tx + 32 * ty;
    const ChebArgs<T>& ca = fp.ca;
    const C13<T> k = fp.k13;
    const T* __restrict__ ag = static_cast<const T*>(op.a);
    if (tid < 2 * STEPS) {
        const T v = (T)ca.coef[tid];
        if (tid & 1) sc2[tid >> 1] = v;
        else sc1[tid >> 1] = v;
    }
    const int ly_lo = max(0, H - j0), ly_hi = min(SY - 1, ny - j0 + H);
    const bool wall_lo = j0 - H + ly_lo == 0, wall_hi = j0 - H + ly_hi == ny;
    // ---- staging: b, a, D^-1 (and x for FUSED_UP), every copy in flight
    for (int ly = ly_lo + ty; ly <= ly_hi; ly += 8) {
        const size_t row = (size_t)(j0 - H + ly) * nx;
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            const int lx = tx + 32 * c;
            if (lx >= SX) break;
            int i = (i0 - H + lx) % nx;
            if (i < 0) i += nx;
            const int o = ly * SX + lx;
            cp_async4(sb + o, fp.b + row + i);
            cp_async4(sa + o, ag + row + i);
            cp_async4(sdi + o, ca.dinv + row + i);
            if (MODE == FUSED_UP) cp_async4(sx + o, fp.xin + row + i);
        }
    }
    cp_async_wait4();
    __syncthreads();
    // the first iterate: x_1 = c D^-1 b, or x + P x_c
    {
        const T cz = sc2[0];
        for (int ly = ly_lo + ty; ly <= ly_hi; ly += 8) {
            const int j = j0 - H + ly;
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = tx + 32 * c;
                if (lx >= SX) break;
                const int o = ly * SX + lx;
                if (MODE == FUSED_UP) {
                    int i = (i0 - H + lx) % nx;
                    if (i < 0) i += nx;
                    sx[o] += prolong_at(ca, ny, i, j);
                } else {
                    sx[o] = mul_rn(mul_rn(cz, sdi[o]), sb[o]);
                }
            }
        }
    }
    __syncthreads();
    // neighbour rows (zero flux: reflected at the walls)
    auto rows_of = [&](int ly, int j, int& lys, int& lyn) {
        lys = j > 0 ? ly - 1 : ly + 1;
        lyn = j < ny ? ly + 1 : ly - 1;
    };
    // psi on the region shrunk by sh nodes (not at a wall)
    auto form_psi = [&](int sh) {
        const int rlo = wall_lo ? ly_lo : ly_lo + sh, rhi = wall_hi ? ly_hi : ly_hi - sh;
        for (int ly = rlo + ty; ly <= rhi; ly += 8) {
            int lys, lyn;
            rows_of(ly, j0 - H + ly, lys, lyn);
            const T* xc_ = sx + ly * SX;
            const T* xs_ = sx + lys * SX;
            const T* xn_ = sx + lyn * SX;
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = tx + 32 * c;
                if (lx < sh || lx >= SX - sh) continue;
                const T cv = xc_[lx];
                sp[ly * SX + lx] = fma(k.ky, (cv - xs_[lx]) + (cv - xn_[lx]),
                                       fma(k.kx, (cv - xc_[lx - 1]) + (cv - xc_[lx + 1]),
                                           mul_rn(k.S, cv)));
            }
        }
    };
    // A x at (ly, lx) from psi, a and x
    auto ax_at = [&](int ly, int lx, int lys, int lyn) {
        const int o = ly * SX + lx;
        const T pc = sp[o], ac = sa[o];
        const T fx = fma(ac + sa[o + 1], sp[o + 1] - pc, -mul_rn(ac + sa[o - 1], pc - sp[o - 1]));
        const T fy = fma(ac + sa[lyn * SX + lx], sp[lyn * SX + lx] - pc,
                         -mul_rn(ac + sa[lys * SX + lx], pc - sp[lys * SX + lx]));
        return fma(-k.gyq, fy, fma(-k.gxq, fx, mul_rn(k.idt, sx[o])));
    };
#pragma unroll
    for (int s = 1; s <= NST; ++s) {
        const int kk = K0 + s - 1;
        const bool zero = MODE != FUSED_UP && kk == 1;
        form_psi(2 * s - 1);
        __syncthreads();
        const T c1 = sc1[kk], c2 = sc2[kk];
        const int sh = 2 * s;
        const int rlo = wall_lo ? ly_lo : ly_lo + sh, rhi = wall_hi ? ly_hi : ly_hi - sh;
        for (int ly = rlo + ty; ly <= rhi; ly += 8) {
            int lys, lyn;
            rows_of(ly, j0 - H + ly, lys, lyn);
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = tx + 32 * c;
                if (lx < sh || lx >= SX - sh) continue;
                const int o = ly * SX + lx;
                const T xc = sx[o];
                const T r = sb[o] - ax_at(ly, lx, lys, lyn);
                T dn;
                if (zero)
                    dn = fma(mul_rn(c2, sdi[o]), r, mul_rn(c1, xc));
                else   // c1 = 0 at k = 0 (no direction yet)
                    dn = fma(mul_rn(c2, sdi[o]), r, c1 != (T)0 ? mul_rn(c1, sd[o]) : (T)0);
                sd[o] = dn;
                sx[o] = xc + dn;
            }
        }
        __syncthreads();
    }
    // ---- x on the tile
    {
        T* xg = fp.xout;
        for (int ly = max(H, ly_lo) + ty; ly < H + TY && ly <= ly_hi; ly += 8) {
            const size_t row = (size_t)(j0 - H + ly) * nx;
#pragma unroll
            for (int c = 0; c < (TX + 31) / 32; ++c) {
                const int lx = H + tx + 32 * c;
                const int i = i0 + tx + 32 * c;
                if (lx < H + TX && i < nx) xg[row + i] = sx[ly * SX + lx];
            }
        }
    }
    if constexpr (MODE == FUSED_DOWN) {
        // residual b - A x on the tile and a one-node ring
        form_psi(2 * NST + 1);
        __syncthreads();
        const int sh = 2 * NST + 2;   // = H - 1
        const int rlo = wall_lo ? ly_lo : ly_lo + sh, rhi = wall_hi ? ly_hi : ly_hi - sh;
        for (int ly = rlo + ty; ly <= rhi; ly += 8) {
            int lys, lyn;
            rows_of(ly, j0 - H + ly, lys, lyn);
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int lx = tx + 32 * c;
                if (lx < sh || lx >= SX - sh) continue;
                const int o = ly * SX + lx;
                sd[o] = sb[o] - ax_at(ly, lx, lys, lyn);
            }
        }
        __syncthreads();
        const Grid gc = fp.gc;
        const int semi = fp.semi;
        const int J0 = j0 / 2, J1 = min((j0 + TY) / 2, gc.ny + 1);
        const int I0 = semi ? i0 : i0 / 2, I1 = min(semi ? i0 + TX : (i0 + TX) / 2, gc.nx);
        for (int J = J0 + ty; J < J1; J += 8) {
            for (int I = I0 + tx; I < I1; I += 32) {
                const int lc = (semi ? I : 2 * I) - i0 + H;
                auto res = [&](int j, int dx) { return sd[(j - j0 + H) * SX + lc + dx]; };
                fp.bc[(size_t)J * gc.nx + I] = restrict_at<T>(res, J, ny, semi, gc.ny);
            }
        }
    }
}

// The tile shapes a pass may take (columns x rows).
constexpr int FT_X[3] = {128, 64, 32}, FT_Y[3] = {16, 16, 8};

// Tile of a level: the widest whose grid still gives every SM a block (the
// narrower tiles recompute more halo nodes per output node).
static int fused_tile(const Grid& g) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CAHN_CUDA_TRY(cudaGetDevice(&dev));
        CAHN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    for (int t = 0; t < 3; ++t) {
        const long blocks = (long)((g.nx + FT_X[t] - 1) / FT_X[t]) * ((g.ny + 1 + FT_Y[t] - 1) / FT_Y[t]);
        if (blocks >= sms) return t;
    }
    return 2;
}

template <int MODE, int STEPS>
constexpr size_t smem_of(int t) {
    return 4 * sizeof(float) * (size_t)(FT_X[t] + 2 * FusedShape<MODE, STEPS>::H) *
           (FT_Y[t] + 2 * FusedShape<MODE, STEPS>::H);
}

// every pass and tile in FUSED_SMEM_MAX
static_assert(smem_of<FUSED_DOWN, FUSED_DEG_MAX>(0) <= FUSED_SMEM_MAX, "fused pass shared memory");
static_assert(smem_of<FUSED_UP, FUSED_DEG_MAX>(0) <= FUSED_SMEM_MAX, "fused pass shared memory");
static_assert(smem_of<FUSED_COARSE, FUSED_COARSE_STEPS>(0) <= FUSED_SMEM_MAX, "fused pass shared memory");

template <typename T, int KIND, int MODE, int STEPS>
static void launch_shape(const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    const int t = fused_tile(fp.op.g);
    constexpr int H = FusedShape<MODE, STEPS>::H;
    const size_t smem = 4 * sizeof(T) * (size_t)(FT_X[t] + 2 * H) * (FT_Y[t] + 2 * H);
    const dim3 grid((unsigned)((fp.op.g.nx + FT_X[t] - 1) / FT_X[t]),
                    (unsigned)((fp.op.g.ny + 1 + FT_Y[t] - 1) / FT_Y[t])),
        blk(32, 8);
    note_launch();
    switch (t) {
        case 0: launch_k(k_mg_fused<T, KIND, MODE, 128, 16, STEPS>, grid, blk, smem, s, fp, gate); break;
        case 1: launch_k(k_mg_fused<T, KIND, MODE, 64, 16, STEPS>, grid, blk, smem, s, fp, gate); break;
        default: launch_k(k_mg_fused<T, KIND, MODE, 32, 8, STEPS>, grid, blk, smem, s, fp, gate); break;
    }
}

template <int MODE, int STEPS>
constexpr size_t smem13_of(int t) {
    return 6 * sizeof(float) * (size_t)(FT_X[t] + 2 * Fused13Shape<MODE, STEPS>::H) *
           (FT_Y[t] + 2 * Fused13Shape<MODE, STEPS>::H);
}
static_assert(smem13_of<FUSED_DOWN, FUSED_DEG_MAX>(0) <= FUSED13_SMEM_MAX, "fused pass shared memory");
static_assert(smem13_of<FUSED_UP, FUSED_DEG_MAX>(0) <= FUSED13_SMEM_MAX, "fused pass shared memory");
static_assert(smem13_of<FUSED_COARSE, FUSED_COARSE_STEPS>(0) <= FUSED13_SMEM_MAX,
              "fused pass shared memory");

template <typename T, int MODE, int STEPS>
static void launch_shape13(const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    const int t = fused_tile(fp.op.g);
    constexpr int H = Fused13Shape<MODE, STEPS>::H;
    const size_t smem = 6 * sizeof(T) * (size_t)(FT_X[t] + 2 * H) * (FT_Y[t] + 2 * H);
    const dim3 grid((unsigned)((fp.op.g.nx + FT_X[t] - 1) / FT_X[t]),
                    (unsigned)((fp.op.g.ny + 1 + FT_Y[t] - 1) / FT_Y[t])),
        blk(32, 8);
    note_launch();
    switch (t) {
        case 0: launch_k(k_mg_fused13<T, MODE, 128, 16, STEPS>, grid, blk, smem, s, fp, gate); break;
        case 1: launch_k(k_mg_fused13<T, MODE, 64, 16, STEPS>, grid, blk, smem, s, fp, gate); break;
        default: launch_k(k_mg_fused13<T, MODE, 32, 8, STEPS>, grid, blk, smem, s, fp, gate); break;
    }
}

template <typename T, int DEG>
static void prepare13_deg() {
    auto set = [](auto k) {
        CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FUSED13_SMEM_MAX));
    };
    set(k_mg_fused13<T, FUSED_DOWN, 128, 16, DEG>);
    set(k_mg_fused13<T, FUSED_DOWN, 64, 16, DEG>);
    set(k_mg_fused13<T, FUSED_DOWN, 32, 8, DEG>);
    set(k_mg_fused13<T, FUSED_UP, 128, 16, DEG>);
    set(k_mg_fused13<T, FUSED_UP, 64, 16, DEG>);
    set(k_mg_fused13<T, FUSED_UP, 32, 8, DEG>);
}

template <typename T>
static void prepare13() {
    auto set = [](auto k) {
        CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FUSED13_SMEM_MAX));
    };
    prepare13_deg<T, 3>();
    prepare13_deg<T, 4>();
    prepare13_deg<T, 5>();
    set(k_mg_fused13<T, FUSED_COARSE, 128, 16, FUSED_COARSE_STEPS>);
    set(k_mg_fused13<T, FUSED_COARSE, 64, 16, FUSED_COARSE_STEPS>);
    set(k_mg_fused13<T, FUSED_COARSE, 32, 8, FUSED_COARSE_STEPS>);
}

template <typename T, int KIND, int DEG>
static void prepare_deg() {
    auto set = [](auto k) {
        CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FUSED_SMEM_MAX));
    };
    set(k_mg_fused<T, KIND, FUSED_DOWN, 128, 16, DEG>);
    set(k_mg_fused<T, KIND, FUSED_DOWN, 64, 16, DEG>);
    set(k_mg_fused<T, KIND, FUSED_DOWN, 32, 8, DEG>);
    set(k_mg_fused<T, KIND, FUSED_UP, 128, 16, DEG>);
    set(k_mg_fused<T, KIND, FUSED_UP, 64, 16, DEG>);
    set(k_mg_fused<T, KIND, FUSED_UP, 32, 8, DEG>);
}

template <typename T, int KIND>
static void prepare_kind() {
    auto set = [](auto k) {
        CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FUSED_SMEM_MAX));
    };
    prepare_deg<T, KIND, 3>();
    prepare_deg<T, KIND, 4>();
    prepare_deg<T, KIND, 5>();
    set(k_mg_fused<T, KIND, FUSED_COARSE, 128, 16, FUSED_COARSE_STEPS>);
    set(k_mg_fused<T, KIND, FUSED_COARSE, 64, 16, FUSED_COARSE_STEPS>);
    set(k_mg_fused<T, KIND, FUSED_COARSE, 32, 8, FUSED_COARSE_STEPS>);
}

template <typename T>
void fused_prepare() {
    static bool done = false;
    if (done) return;
    prepare_kind<T, OP_LAP5_DIRICHLET>();
    prepare_kind<T, OP_LAP5_NEUMANN>();
    prepare13<T>();
    done = true;
}

// one pass of `mode` with the smoother's degree fp.steps (FUSED_DEG_MIN ..
// FUSED_DEG_MAX; FUSED_COARSE: FUSED_COARSE_STEPS)
template <typename T, int KIND, int MODE>
static void launch_deg(const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    switch (fp.steps) {
        case 3: launch_shape<T, KIND, MODE, 3>(fp, gate, s); break;
        case 4: launch_shape<T, KIND, MODE, 4>(fp, gate, s); break;
        case 5: launch_shape<T, KIND, MODE, 5>(fp, gate, s); break;
        default: throw ArgError("fused multigrid pass: unsupported smoother degree");
    }
}
template <typename T, int MODE>
static void launch_deg13(const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    switch (fp.steps) {
        case 3: launch_shape13<T, MODE, 3>(fp, gate, s); break;
        case 4: launch_shape13<T, MODE, 4>(fp, gate, s); break;
        case 5: launch_shape13<T, MODE, 5>(fp, gate, s); break;
        default: throw ArgError("fused multigrid pass: unsupported smoother degree");
    }
}

template <typename T>
void launch_fused(int mode, const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    const bool dir = fp.op.kind == OP_LAP5_DIRICHLET;
    if (mode == FUSED_COARSE && fp.steps != FUSED_COARSE_STEPS)
        throw ArgError("fused multigrid pass: unsupported coarse step count");
    if (fp.op.kind == OP_CH13) {
        switch (mode) {
            case FUSED_DOWN: launch_deg13<T, FUSED_DOWN>(fp, gate, s); break;
            case FUSED_UP: launch_deg13<T, FUSED_UP>(fp, gate, s); break;
            default: launch_shape13<T, FUSED_COARSE, FUSED_COARSE_STEPS>(fp, gate, s); break;
        }
        return;
    }
    if (fp.op.kind != OP_LAP5_DIRICHLET && fp.op.kind != OP_LAP5_NEUMANN)
        throw ArgError("fused multigrid pass: 5-point and 13-point operators only");
    switch (mode) {
        case FUSED_DOWN:
            if (dir) launch_deg<T, OP_LAP5_DIRICHLET, FUSED_DOWN>(fp, gate, s);
            else launch_deg<T, OP_LAP5_NEUMANN, FUSED_DOWN>(fp, gate, s);
            break;
        case FUSED_UP:
            if (dir) launch_deg<T, OP_LAP5_DIRICHLET, FUSED_UP>(fp, gate, s);
            else launch_deg<T, OP_LAP5_NEUMANN, FUSED_UP>(fp, gate, s);
            break;
        default:
            if (dir) launch_shape<T, OP_LAP5_DIRICHLET, FUSED_COARSE, FUSED_COARSE_STEPS>(fp, gate, s);
            else launch_shape<T, OP_LAP5_NEUMANN, FUSED_COARSE, FUSED_COARSE_STEPS>(fp, gate, s);
            break;
    }
}

template void launch_fused<float>(int, const FusedPass<float>&, const int*, cudaStream_t);
template void fused_prepare<float>();

}  // namespace cahn
