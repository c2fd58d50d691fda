// Domain-decomposition preconditioner (precond = CAHN_PC_SCHWARZ): the
// preconditioners "based on domain decomposition ideas" that the paper
// plans in place of Jacobi (§4.1, §6), as one launch per application.
//
// The grid is split into tiles of SW_CX x SW_CY nodes (the subdomains; the
// last tile in x and y ragged).  Block i extends its tile by OVL nodes on
// every side (periodic in x, clipped at the walls) and solves the local
// problem A_ii z_i = r_i on the extended subdomain, with zero outside it
// (the walls keep their own conditions), approximately: SW_STEPS
// Chebyshev-Jacobi steps from zero over the whole local spectrum
// [lam / SW_ALPHA, lam] (lam the Gershgorin bound of D^-1 A), every vector
// in shared memory.  It writes z on its own tile only:
//   OVL = 2: restricted additive Schwarz (RAS), for the non-symmetric
//            phase-field system under GMRES;
//   OVL = 0: non-overlapping block Jacobi, M = sum_i R_i^T p(D_i^-1 A_ii)
//            D_i^-1 R_i, a fixed polynomial of each diagonal block: self-
//            adjoint and positive definite in the W inner product when A
//            is, so CG keeps its theory (H, L_h, the nutrient K).
// There is no coarse space: a one-level method, so iterations grow with
// the number of subdomains across the grid.
#include "schwarz.h"

namespace cahn {

template <typename T, int KIND, int OVL>
__global__ void __launch_bounds__(256) k_schwarz(Op op, const T* __restrict__ r, T* __restrict__ z,
                                                 const T* __restrict__ dinv,
                                                 const double* __restrict__ coef, int steps, int dz,
                                                 const int* __restrict__ gate) {
    if (gate && *gate) return;
    constexpr int EW = SW_CX + 2 * OVL, EH = SW_CY + 2 * OVL, EN = EW * EH;
    constexpr bool CH = KIND == OP_CH13;
    constexpr bool NUT = KIND == OP_NUT5;
    constexpr int RW = EW + 2, RH = EH + 2;   // with a one-node ring (psi, a)
    __shared__ T sx[EN], sxt[EN], sd[EN], sr[EN], sdi[EN];
    __shared__ T spsi[CH ? RH * RW : 1], sa[(CH || NUT) ? RH * RW : 1], sdg[NUT ? EN : 1];
    __shared__ unsigned char sinside[EN];   // node inside the extended subdomain
    const int nx = op.g.nx, ny = op.g.ny;
    const int i0 = blockIdx.x * SW_CX, j0 = blockIdx.y * SW_CY;
    const int iend = min(i0 + SW_CX, nx), jend = min(j0 + SW_CY, ny + 1);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    // extended subdomain: columns i0 - OVL .. iend + OVL - 1 (periodic), rows
    // max(j0 - OVL, 0) .. min(jend + OVL, ny + 1) - 1; local (lx, ly) ->
    // global (i0 - OVL + lx, j0 - OVL + ly)
    const int ilo = i0 - OVL, ihi = iend + OVL;   // [ilo, ihi)
    const int jlo = max(j0 - OVL, 0), jhi = min(jend + OVL, ny + 1);
    auto gi_of = [&](int lx) { int g = ilo + lx; return g < 0 ? g + nx : (g >= nx ? g - nx : g); };
    // local index of global node (i, j), or -1 when outside the subdomain
    auto loc = [&](int i, int j) -> int {
        if (j < jlo || j >= jhi) return -1;
        int d = i - ilo;
        if (d < 0) d += nx;
        if (d >= nx) d -= nx;
        if (d >= ihi - ilo) return -1;
        return (j - (j0 - OVL)) * EW + d;
    };
    const T* __restrict__ a = static_cast<const T*>(op.a);
    const T* __restrict__ dg = static_cast<const T*>(op.dg);
    for (int t = tid; t < EN; t += nt) {
        const int lx = t % EW, ly = t / EW;
        const int j = j0 - OVL + ly;
        const bool in = j >= jlo && j < jhi && lx < ihi - ilo;
        sinside[t] = in;
        sx[t] = sxt[t] = sd[t] = (T)0;
        if (in) {
            const size_t e = (size_t)j * nx + gi_of(lx);
            sr[t] = r[e];
            if (KIND == OP_LAP5_DIRICHLET) {
                const double dd = (j == 0 || j == ny) ? op.c0 : op.c0 + 2 * op.cx + 2 * op.cy;
                sdi[t] = (T)(1.0 / dd);
            } else if (KIND == OP_LAP5_NEUMANN) {
                sdi[t] = (T)(1.0 / (op.c0 + 2 * op.cx + 2 * op.cy));
            } else {
                sdi[t] = dinv[e];
            }
            if (NUT) sdg[t] = dg[e];
        } else {
            sr[t] = sdi[t] = (T)0;
        }
    }
    if (CH || NUT) {   // a on the subdomain box and a one-node ring (periodic, reflected)
        for (int t = tid; t < RH * RW; t += nt) {
            const int lx = t % RW - 1, ly = t / RW - 1;
            sa[t] = a[(size_t)refly(j0 - OVL + ly, ny) * nx + gi_of(lx)];
        }
    }
    __syncthreads();
    // value of the local iterate v at global node (i, j): zero outside
    auto V = [&](const T* v, int i, int j) -> T {
        const int k = loc(i, j);
        return k < 0 ? (T)0 : v[k];
    };
    auto A_at = [&](const T* v, int t) -> T {   // (A_ii v) at local node t
        const int lx = t % EW, ly = t / EW;
        const int i = gi_of(lx), j = j0 - OVL + ly;
        const int im = i > 0 ? i - 1 : nx - 1, ip = i < nx - 1 ? i + 1 : 0;
        const T c = v[t];
        if (KIND == OP_LAP5_DIRICHLET || KIND == OP_LAP5_NEUMANN) {
            const Lap5C<T> kc = lap5_consts<T>(op);
            if (KIND == OP_LAP5_DIRICHLET && (j == 0 || j == ny)) return mul_rn(kc.c0, c);
            const int js = KIND == OP_LAP5_NEUMANN ? refly(j - 1, ny) : j - 1;
            const int jn = KIND == OP_LAP5_NEUMANN ? refly(j + 1, ny) : j + 1;
            return lap5_ax(kc, c, V(v, im, j), V(v, ip, j), V(v, i, js), V(v, i, jn));
        } else if (NUT) {
            if (op.nut_dtop && j == ny) return mul_rn(sdg[t], c);
            const int js = refly(j - 1, ny), jn = refly(j + 1, ny);
            auto A_ = [&](int dx, int dy) { return sa[(ly + 1 + dy) * RW + lx + 1 + dx]; };
            const T ac = A_(0, 0);
            const T sxv = fma(ac + A_(1, 0), c - V(v, ip, j), mul_rn(ac + A_(-1, 0), c - V(v, im, j)));
            const T syv = fma(ac + A_(0, 1), c - V(v, i, jn), mul_rn(ac + A_(0, -1), c - V(v, i, js)));
            return fma((T)op.gx, sxv, fma((T)op.gy, syv, mul_rn(sdg[t], c)));
        } else {   // 13-point: psi on the subdomain and ring is in spsi
            auto P = [&](int dx, int dy) { return spsi[(ly + 1 + dy) * RW + lx + 1 + dx]; };
            auto A_ = [&](int dx, int dy) { return sa[(ly + 1 + dy) * RW + lx + 1 + dx]; };
            const T pc = P(0, 0), ac = A_(0, 0);
            const T fx = fma(ac + A_(1, 0), P(1, 0) - pc, -mul_rn(ac + A_(-1, 0), pc - P(-1, 0)));
            const T fy = fma(ac + A_(0, 1), P(0, 1) - pc, -mul_rn(ac + A_(0, -1), pc - P(0, -1)));
            return fma(-(T)(0.25 * op.gy), fy, fma(-(T)(0.25 * op.gx), fx, mul_rn((T)op.idt, c)));
        }
    };
    // psi = kappa L_h v + S v of the zero-extended iterate on the subdomain and
    // its ring; the ring rows beyond a wall are the reflections of the rows inside
    auto form_psi = [&](const T* v) {
        for (int t = tid; t < RH * RW; t += nt) {
            const int lx = t % RW - 1, ly = t / RW - 1;
            const int ii = gi_of(lx);
            const int j = refly(j0 - OVL + ly, ny);
            const int im = ii > 0 ? ii - 1 : nx - 1, ip = ii < nx - 1 ? ii + 1 : 0;
            const int js = refly(j - 1, ny), jn = refly(j + 1, ny);
            const T c = V(v, ii, j);
            spsi[t] = fma((T)op.ky, (c - V(v, ii, js)) + (c - V(v, ii, jn)),
                          fma((T)op.kx, (c - V(v, im, j)) + (c - V(v, ip, j)), mul_rn((T)op.S, c)));
        }
        __syncthreads();
    };
    // Chebyshev from zero: d = c2(0) D^-1 r, x = d; then d = c1 d + c2 D^-1 (r - A x)
    T* cur = sx;
    T* nxt = sxt;
    for (int k = 0; k < steps; ++k) {
        const T c1 = (T)coef[2 * k], c2 = (T)coef[2 * k + 1];
        if (CH && k > 0) form_psi(cur);
        for (int t = tid; t < EN; t += nt) {
            if (!sinside[t]) continue;
            const int j = j0 - OVL + t / EW;
            if (dz_row(dz, j, ny)) {
                nxt[t] = (T)0;
                continue;
            }
            T dn;
            if (k == 0) {
                dn = mul_rn(mul_rn(c2, sdi[t]), sr[t]);
                nxt[t] = dn;
            } else {
                const T res = sr[t] - A_at(cur, t);
                dn = fma(mul_rn(c2, sdi[t]), res, mul_rn(c1, sd[t]));
                nxt[t] = cur[t] + dn;
            }
            sd[t] = dn;
        }
        __syncthreads();
        T* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    // restricted write: this tile's own nodes
    for (int t = tid; t < EN; t += nt) {
        const int lx = t % EW, ly = t / EW;
        const int gi = ilo + lx, j = j0 - OVL + ly;
        if (gi < i0 || gi >= iend || j < j0 || j >= jend) continue;
        z[(size_t)j * nx + gi] = cur[t];
    }
}

template <typename T>
void launch_schwarz(const Op& op, const T* r, T* z, const T* dinv, const double* coef, int dz,
                    const int* gate, cudaStream_t s) {
    const dim3 grid((unsigned)((op.g.nx + SW_CX - 1) / SW_CX),
                    (unsigned)((op.g.ny + 1 + SW_CY - 1) / SW_CY)),
        blk(32, 8);
    note_launch();
    switch (op.kind) {
        case OP_LAP5_NEUMANN:
            launch_k(k_schwarz<T, OP_LAP5_NEUMANN, 0>, grid, blk, 0, s, op, r, z, dinv, coef, SW_STEPS, dz, gate);
            break;
        case OP_LAP5_DIRICHLET:
            launch_k(k_schwarz<T, OP_LAP5_DIRICHLET, 0>, grid, blk, 0, s, op, r, z, dinv, coef, SW_STEPS, dz, gate);
            break;
        case OP_NUT5:
            launch_k(k_schwarz<T, OP_NUT5, 0>, grid, blk, 0, s, op, r, z, dinv, coef, SW_STEPS, dz, gate);
            break;
        case OP_CH13:
            launch_k(k_schwarz<T, OP_CH13, 2>, grid, blk, 0, s, op, r, z, dinv, coef, SW_STEPS, dz, gate);
            break;
        default:
            throw ArgError("CAHN_PC_SCHWARZ: no subdomain solve for this operator");
    }
}

template void launch_schwarz<double>(const Op&, const double*, double*, const double*,
                                     const double*, int, const int*, cudaStream_t);
template void launch_schwarz<float>(const Op&, const float*, float*, const float*, const double*,
                                    int, const int*, cudaStream_t);

}  // namespace cahn
