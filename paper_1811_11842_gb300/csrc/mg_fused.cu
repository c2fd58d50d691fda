// Temporally blocked multigrid passes for the FP32 5-point hierarchies
// (L_h with zero flux, H with Dirichlet walls).  Each block stages its tile
// of the level and a halo of H nodes in shared memory once, then runs
// several Chebyshev-Jacobi steps on it, the region shrinking by one node per
// stencil application (not at a wall, where the neighbour rows are rows of
// the tile), so that one launch does what the separate launches do level by
// level:
//   FUSED_DOWN:   steps 0 .. deg-1 from x = 0 (step 0 formed from b), the
//                 residual b - A x on the tile and a one-node ring, and its
//                 restriction R (b - A x) to the coarse nodes of the tile;
//                 writes x and the coarse right-hand side.  H = deg + 1.
//   FUSED_UP:     x + P x_c formed in the staging, then steps 0 .. deg-1;
//                 writes x.  H = deg.
//   FUSED_COARSE: steps 0 .. k-1 from x = 0 on the coarsest level.
//                 H = k - 1.
// Every node is evaluated with the operations of the separate launches
// (lap5_ax, the step formulas of epi_node, prolong_at, the restriction
// weights of k_resid_restrict), so the V-cycle's result is bit for bit
// theirs; only the redundant halo nodes are extra work.
#include "mg_fused.h"
#include "stencil_dev.cuh"

namespace cahn {

template <typename T, int KIND, int MODE>
__global__ void __launch_bounds__(256) k_mg_fused(FusedPass<T> fp, const int* __restrict__ gate) {
    if (gate && *gate) return;
    extern __shared__ __align__(16) unsigned char fsm[];
    const int H = fp.halo, TX = fp.tx, TY = fp.ty;
    const int SX = TX + 2 * H, SY = TY + 2 * H, SN = SX * SY;
    T* sb = reinterpret_cast<T*>(fsm);   // b on the staged region
    T* sa = sb + SN;                     // ping-pong iterates
    T* sc = sa + SN;
    T* sd = sc + SN;                     // Chebyshev direction d (then the residual)
    const Op& op = fp.op;
    const int nx = op.g.nx, ny = op.g.ny;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const ChebArgs<T>& ca = fp.ca;
    const Lap5C<T> kc = lap5_consts<T>(op);
    const int dz = ca.dirichlet_zero;
    auto di_of = [&](int j) {
        return (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) ? ca.di_wall : ca.di_int;
    };
    // staged rows: j = j0 - H + ly for ly in [ly_lo, ly_hi] (the rows 0 .. ny)
    const int ly_lo = max(0, H - j0), ly_hi = min(SY - 1, ny - j0 + H);
    const bool wall_lo = j0 - H + ly_lo == 0, wall_hi = j0 - H + ly_hi == ny;
    auto gcol = [&](int lx) {
        int i = (i0 - H + lx) % nx;
        return i < 0 ? i + nx : i;
    };
    // ---- staging
    for (int ly = ly_lo + ty; ly <= ly_hi; ly += 8) {
        const int j = j0 - H + ly;
        const size_t row = (size_t)j * nx;
        for (int lx = tx; lx < SX; lx += 32) {
            const int i = gcol(lx);
            const size_t e = row + i;
            sb[ly * SX + lx] = fp.b[e];
            if (MODE == FUSED_UP) sa[ly * SX + lx] = fp.xin[e] + prolong_at(ca, ny, i, j);
        }
    }
    __syncthreads();
    // ---- Chebyshev steps
    const int k0 = MODE == FUSED_UP ? 0 : 1;
    const T cz = (T)ca.coef[1];
    T* in = sa;   // FUSED_UP: x + P x_c
    T* out = MODE == FUSED_UP ? sc : sa;
    for (int k = k0; k < fp.steps; ++k) {
        const int s = k - k0 + 1;   // stencil applications so far
        const bool zero = MODE != FUSED_UP && k == 1;   // step 1 reads x_1 = cz D^-1 b
        const T c1 = (T)ca.coef[2 * k], c2 = (T)ca.coef[2 * k + 1];
        auto X = [&](int ly, int lx) -> T {
            const int idx = ly * SX + lx;
            if (zero) return mul_rn(mul_rn(cz, di_of(j0 - H + ly)), sb[idx]);
            return in[idx];
        };
        const int rlo = wall_lo ? ly_lo : ly_lo + s, rhi = wall_hi ? ly_hi : ly_hi - s;
        for (int ly = rlo + ty; ly <= rhi; ly += 8) {
            const int j = j0 - H + ly;
            for (int lx = s + tx; lx < SX - s; lx += 32) {
                const int idx = ly * SX + lx;
                const T xc = X(ly, lx);
                T ax;
                if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) {
                    ax = mul_rn(kc.c0, xc);
                    if (dz) {
                        out[idx] = (T)0;
                        continue;
                    }
                } else {
                    int lys, lyn;
                    if (KIND == OP_LAP5_NEUMANN) {
                        lys = j > 0 ? ly - 1 : ly + 1;
                        lyn = j < ny ? ly + 1 : ly - 1;
                    } else {
                        lys = ly - 1;
                        lyn = ly + 1;
                    }
                    ax = lap5_ax(kc, xc, X(ly, lx - 1), X(ly, lx + 1), X(lys, lx), X(lyn, lx));
                }
                const T r = sb[idx] - ax;
                const T di = di_of(j);
                T dn;
                if (zero)
                    dn = fma(mul_rn(c2, di), r, mul_rn(c1, xc));
                else   // c1 = 0 at k = 0 (no direction yet)
                    dn = fma(mul_rn(c2, di), r, c1 != (T)0 ? mul_rn(c1, sd[idx]) : (T)0);
                sd[idx] = dn;
                out[idx] = xc + dn;
            }
        }
        __syncthreads();
        in = out;
        out = (out == sa) ? sc : sa;
    }
    const T* xf = in;   // the last step's iterate
    // ---- x on the tile
    T* xg = fp.xout;
    for (int ly = max(H, ly_lo) + ty; ly < H + TY && ly <= ly_hi; ly += 8) {
        const size_t row = (size_t)(j0 - H + ly) * nx;
        for (int lx = H + tx; lx < H + TX; lx += 32) {
            const int i = i0 - H + lx;
            if (i < nx) xg[row + i] = xf[ly * SX + lx];
        }
    }
    if constexpr (MODE == FUSED_DOWN) {
        // residual b - A x on the tile and a one-node ring (k_resid_restrict's res)
        for (int ly = max(H - 1, ly_lo) + ty; ly <= H + TY && ly <= ly_hi; ly += 8) {
            const int j = j0 - H + ly;
            for (int lx = H - 1 + tx; lx <= H + TX; lx += 32) {
                const int idx = ly * SX + lx;
                const T xc = xf[idx];
                T res;
                if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) {
                    res = sb[idx] - mul_rn(kc.c0, xc);
                } else {
                    int lys, lyn;
                    if (KIND == OP_LAP5_NEUMANN) {
                        lys = j > 0 ? ly - 1 : ly + 1;
                        lyn = j < ny ? ly + 1 : ly - 1;
                    } else {
                        lys = ly - 1;
                        lyn = ly + 1;
                    }
                    res = sb[idx] - lap5_ax(kc, xc, xf[idx - 1], xf[idx + 1], xf[lys * SX + lx],
                                            xf[lyn * SX + lx]);
                }
                sd[idx] = res;
            }
        }
        __syncthreads();
        // restriction to the coarse nodes whose centre 2J (2I) lies in the tile
        const Grid gc = fp.gc;
        const int semi = fp.semi;
        const double inv_ratio = semi ? 0.5 : 0.25;
        const int J0 = j0 / 2, J1 = min((j0 + TY) / 2, gc.ny + 1);
        const int I0 = semi ? i0 : i0 / 2, I1 = min(semi ? i0 + TX : (i0 + TX) / 2, gc.nx);
        for (int J = J0 + ty; J < J1; J += 8) {
            for (int I = I0 + tx; I < I1; I += 32) {
                const size_t ec = (size_t)J * gc.nx + I;
                if (dz_row(dz, J, gc.ny)) {
                    fp.bc[ec] = (T)0;
                    continue;
                }
                double sum = 0.0;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int j = 2 * J + dy;
                    if (j < 0 || j > ny) continue;
                    const double wy = (dy == 0 ? 1.0 : 0.5) * ((j == 0 || j == ny) ? 0.5 : 1.0);
                    const T* rrow = sd + (j - j0 + H) * SX;
                    if (semi) {
                        sum += wy * (double)rrow[I - i0 + H];
                    } else {
                        const int lc = 2 * I - i0 + H;
                        sum += wy * ((double)rrow[lc] + 0.5 * ((double)rrow[lc - 1] + (double)rrow[lc + 1]));
                    }
                }
                const double wc = (J == 0 || J == gc.ny) ? 0.5 : 1.0;
                fp.bc[ec] = (T)(sum * inv_ratio / wc);
            }
        }
    }
}

// Tile of a level: the widest whose grid still gives every SM a block (the
// narrower tiles recompute more halo nodes per output node).
static void fused_tile(const Grid& g, int& tx, int& ty) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        CAHN_CUDA_TRY(cudaGetDevice(&dev));
        CAHN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    static const int cand[3][2] = {{128, 16}, {64, 16}, {32, 8}};
    for (const auto& c : cand) {
        const long blocks = (long)((g.nx + c[0] - 1) / c[0]) * ((g.ny + 1 + c[1] - 1) / c[1]);
        tx = c[0];
        ty = c[1];
        if (blocks >= sms) return;
    }
}

size_t fused_smem_bytes(int tx, int ty, int halo, size_t elem) {
    return 4 * (size_t)(tx + 2 * halo) * (ty + 2 * halo) * elem;
}

template <typename T>
void fused_prepare() {
    static bool done = false;
    if (done) return;
    auto set = [](auto k) {
        CAHN_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FUSED_SMEM_MAX));
    };
    set(k_mg_fused<T, OP_LAP5_DIRICHLET, FUSED_DOWN>);
    set(k_mg_fused<T, OP_LAP5_DIRICHLET, FUSED_UP>);
    set(k_mg_fused<T, OP_LAP5_DIRICHLET, FUSED_COARSE>);
    set(k_mg_fused<T, OP_LAP5_NEUMANN, FUSED_DOWN>);
    set(k_mg_fused<T, OP_LAP5_NEUMANN, FUSED_UP>);
    set(k_mg_fused<T, OP_LAP5_NEUMANN, FUSED_COARSE>);
    done = true;
}

template <typename T, int KIND, int MODE>
static void launch_one(FusedPass<T> fp, const int* gate, cudaStream_t s) {
    fused_tile(fp.op.g, fp.tx, fp.ty);
    const size_t smem = fused_smem_bytes(fp.tx, fp.ty, fp.halo, sizeof(T));
    if (smem > FUSED_SMEM_MAX) throw ArgError("fused multigrid pass: halo too deep for shared memory");
    const dim3 grid((unsigned)((fp.op.g.nx + fp.tx - 1) / fp.tx),
                    (unsigned)((fp.op.g.ny + 1 + fp.ty - 1) / fp.ty)),
        blk(32, 8);
    note_launch();
    launch_k(k_mg_fused<T, KIND, MODE>, grid, blk, smem, s, fp, gate);
}

template <typename T>
void launch_fused(int mode, const FusedPass<T>& fp, const int* gate, cudaStream_t s) {
    const bool dir = fp.op.kind == OP_LAP5_DIRICHLET;
    if (fp.op.kind != OP_LAP5_DIRICHLET && fp.op.kind != OP_LAP5_NEUMANN)
        throw ArgError("fused multigrid pass: 5-point operators only");
    switch (mode) {
        case FUSED_DOWN:
            if (dir) launch_one<T, OP_LAP5_DIRICHLET, FUSED_DOWN>(fp, gate, s);
            else launch_one<T, OP_LAP5_NEUMANN, FUSED_DOWN>(fp, gate, s);
            break;
        case FUSED_UP:
            if (dir) launch_one<T, OP_LAP5_DIRICHLET, FUSED_UP>(fp, gate, s);
            else launch_one<T, OP_LAP5_NEUMANN, FUSED_UP>(fp, gate, s);
            break;
        default:
            if (dir) launch_one<T, OP_LAP5_DIRICHLET, FUSED_COARSE>(fp, gate, s);
            else launch_one<T, OP_LAP5_NEUMANN, FUSED_COARSE>(fp, gate, s);
            break;
    }
}

template void launch_fused<float>(int, const FusedPass<float>&, const int*, cudaStream_t);
template void fused_prepare<float>();

}  // namespace cahn
