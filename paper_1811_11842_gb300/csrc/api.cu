// C ABI: context life cycle, the time step and single solves.
//
// One step (§4): phase field first (Eq. 2.4 with CN + extrapolation:
// explicit rhs, 13-point solve, mass correction), then the projection
// method with the new phase field: velocity predictor (Eq. 4.3, two
// Dirichlet Helmholtz solves), pressure Poisson (Eq. 4.4, singular,
// projected right-hand side) and velocity correction (Eq. 4.5).  With the
// nutrient on, the phase-field rhs carries the network production (Eq. 2.5),
// the mass target grows with it, and the nutrient system (Eq. 2.6) is solved
// right after the phase field.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cahn.h"
#include "adjoint.h"
#include "mg.h"
#include "nutrient.h"
#include "visc.h"
#include "physics.h"
#include "solver.h"

using namespace cahn;

namespace cahn {
std::atomic<int64_t> g_launches{0};
}

namespace {

thread_local std::string g_init_error;

template <typename T>
T* dalloc(std::vector<void*>& list, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw std::bad_alloc();
    }
    list.push_back(p);
    return static_cast<T*>(p);
}

// Per-system control blocks and scalars of one step, in one device block
// so that graph mode reads every statistic back with a single copy.
struct SysBlock {
    Ctl ctl64[CAHN_NSYS];        // FP64 solve (mixed: refinement sweeps)
    Ctl ctl32[CAHN_NSYS];        // FP32 inner solves (mixed only)
    double scal64[CAHN_NSYS][S_COUNT];
    double scal32[CAHN_NSYS][S_COUNT];
    int status;                  // CTL_DOMAIN from the phase-field rhs
    int nut_status;              // CTL_DOMAIN from the nutrient system (phi^{n+1} >= 1)
};

constexpr int GRAPH_LOOPS = 64;   // loops per captured step graph

struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    GraphCount gc;
    unsigned* h_counters = nullptr;
};

struct Instance {
    cahn_params prm{};
    Grid g{};
    size_t n = 0;
    double *phi_c = nullptr, *u_c = nullptr, *v_c = nullptr, *p_c = nullptr;  // caller's
    double *phi, *phi_prev, *phi_new, *u, *u_prev, *u_new, *v, *v_prev, *v_new, *p, *p_new;
    double *a, *wr, *b, *bu, *bv, *d;
    double *dinv_ch, *dinv_h, *dinv_p;
    MomWs mom{};
    PhysDev P{};
    Op op_ch{}, op_h{}, op_p{};
    KrylovWs<double> kw;
    Multigrid<double> mg_ch, mg_h, mg_p;
    PrecFn<double> pc_ch, pc_h, pc_p;
    bool use_mg = false;
    // mixed precision: FP32 inner solves under FP64 refinement
    bool mixed = false;
    float *a32 = nullptr, *r32 = nullptr, *d32 = nullptr;
    float *dinv32_ch = nullptr, *dinv32_h = nullptr, *dinv32_p = nullptr;
    Op op32_ch{}, op32_h{}, op32_p{};
    KrylovWs<float> kw32;
    Multigrid<float> mg32_ch, mg32_h, mg32_p;
    PrecFn<float> pc32_ch, pc32_h, pc32_p;
    int predict32[CAHN_NSYS] = {4, 4, 4, 8, 16};
    RedWs red{};
    int* d_status = nullptr;   // points into d_sys
    int* d_nut_status = nullptr;   // points into d_sys
    double m0 = 0.0, sumw = 0.0, inv_sumw = 0.0;
    int predict[CAHN_NSYS] = {4, 4, 4, 8, 16};
    bool coef_valid = false;   // a, dinv_ch match the current state
    // graph mode: the step graph forms the next step's phase-field
    // coefficient (a, a32, wr, the hierarchy) from phi^{n+1} and phi^n on a
    // branch of its own, beside the velocity and pressure solves.  Its
    // domain check lands in coef_status, which the next step's graph moves
    // into its own status (k_ch_rhs) before anything reads it.
    int* d_coef_status = nullptr;
    int* d_coef_skip = nullptr;     // != 0: the branch returns at once (the call's last step)
    RedWs red_ch{};                 // the phase-field hierarchy's set-up reductions
    cudaStream_t cbranch = nullptr;
    cudaEvent_t ev_cfork = nullptr, ev_cjoin = nullptr;
    cudaEvent_t ev_ejoin = nullptr;   // a batch's coefficient formed before its graph
    SysBlock* d_sys = nullptr;
    SysBlock* h_sys = nullptr;
    // graph mode: the two predictor solves run as parallel branches of the
    // step graph; the v solve then has workspaces of its own
    bool split_v = false;
    RedWs red_v{};
    KrylovWs<double> kw_v;
    KrylovWs<float> kw32_v;
    Multigrid<double> mg_h_v;
    Multigrid<float> mg32_h_v;
    PrecFn<double> pc_h_v;
    PrecFn<float> pc32_h_v;
    float *r32_v = nullptr, *d32_v = nullptr;
    cudaStream_t vbranch = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // nutrient transport (Eq. 2.6) and network production (Eq. 2.5)
    bool nut = false;             // params.nutrient
    bool nut_ready = false;       // the caller's c is registered
    double* c_c = nullptr;        // caller's
    double *c = nullptr, *c_prev = nullptr, *c_new = nullptr;
    double *ka = nullptr, *kd = nullptr, *dinv_c = nullptr, *bc = nullptr, *gr = nullptr;
    float *ka32 = nullptr, *kd32 = nullptr, *dinv32_c = nullptr;
    double* d_mass = nullptr;     // [1]: the mass target, grown by the production
    NutDev N{};
    Op op_c{}, op32_c{};
    Multigrid<double> mg_c;       // CAHN_PC_MG: V-cycle of the nutrient operator
    Multigrid<float> mg32_c;
    PrecFn<double> pc_c;
    PrecFn<float> pc32_c;
    // fully implicit variable-viscosity momentum (params.momentum): one
    // coupled solve on stacked [u; v] vectors of the grid {nx, 2 ny + 1};
    // eta at phi^{n+1/2} lives in mom.ep
    bool impl_mom = false;
    Grid g_uv{};
    Op op_uv{}, op32_uv{};
    double *buv = nullptr, *xuv = nullptr, *dinv_uv = nullptr;
    float *eta32 = nullptr, *dinv32_uv = nullptr, *r32_uv = nullptr, *d32_uv = nullptr;
    KrylovWs<double> kw_uv;
    KrylovWs<float> kw32_uv;
    // graph mode: one captured step per phase of the 3-buffer rotation
    bool use_graph = false;
    int phase = 0;
    GraphSlot slot[3];
    std::vector<cudaStream_t> cap;
    std::vector<void*> allocs;

    ~Instance() {
        for (GraphSlot& G : slot) {
            if (G.exec) cudaGraphExecDestroy(G.exec);
            if (G.h_counters) cudaFreeHost(G.h_counters);
        }
        for (cudaStream_t c : cap) cudaStreamDestroy(c);
        if (vbranch) cudaStreamDestroy(vbranch);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (cbranch) cudaStreamDestroy(cbranch);
        if (ev_cfork) cudaEventDestroy(ev_cfork);
        if (ev_cjoin) cudaEventDestroy(ev_cjoin);
        if (ev_ejoin) cudaEventDestroy(ev_ejoin);
        if (h_sys) cudaFreeHost(h_sys);
        kw.release();
        kw32.release();
        kw_v.release();
        kw_uv.release();
        kw32_uv.release();
        kw32_v.release();
        mg32_h_v.release();
        mg_h_v.release();
        mg32_c.release();
        mg_c.release();
        mg32_ch.release();
        mg32_h.release();
        mg32_p.release();
        mg_ch.release();
        mg_h.release();
        mg_p.release();
        for (void* q : allocs) cudaFree(q);
    }
};

}  // namespace

struct cahn_ctx {
    std::vector<Instance*> inst;
    cudaStream_t s = nullptr;
    std::string err;
    int64_t launches = 0;
    // batched graph mode: every instance of the context in one graph per
    // buffer phase, one parallel branch per instance
    bool batch_graph = false;
    cudaStream_t bcap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaEvent_t cfork = nullptr;   // the coefficients formed before a batch graph
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t bexec[3] = {nullptr, nullptr, nullptr};
    int bphase = 0;
    void drop_batch_graphs() {
        for (cudaGraphExec_t& e : bexec) {
            if (e) cudaGraphExecDestroy(e);
            e = nullptr;
        }
        bphase = 0;
    }
    ~cahn_ctx() {
        drop_batch_graphs();
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (cfork) cudaEventDestroy(cfork);
        if (bcap) cudaStreamDestroy(bcap);
        for (Instance* I : inst) delete I;
    }
};

namespace {

int fail(cahn_ctx* c, int code, const std::string& msg) {
    if (c)
        c->err = msg;
    else
        g_init_error = msg;
    return code;
}

std::string check_params(const cahn_params& q) {
    if (q.nx < 4 || q.nx % 2) return "nx must be even and >= 4";
    if (q.ny < 4 || q.ny % 2) return "ny must be even and >= 4";
    if ((double)q.nx * (q.ny + 1) > 6.0e7) return "grid too large (nx*(ny+1) > 6e7)";
    if (!(q.lx > 0) || !(q.ly > 0)) return "lx, ly must be > 0";
    if (!(q.eps > 0)) return "eps must be > 0";
    if (!(q.mobility >= 0)) return "mobility must be >= 0";
    if (!(q.dt > 0)) return "dt must be > 0";
    if (!(q.n_poly > 0)) return "n_poly must be > 0";
    if (!(q.stab_s >= 0)) return "stab_s must be >= 0";
    if (!(q.eta_water > 0) || !(q.eta_biofilm > 0)) return "viscosities must be > 0";
    if (!(q.rho_water > 0) || q.rho_water != q.rho_biofilm)
        return "densities must be equal and > 0 (variable density is not supported)";
    if (!(q.gamma_cap >= 0)) return "gamma_cap must be >= 0";
    if (q.flow_mode != CAHN_FLOW_POISEUILLE && q.flow_mode != CAHN_FLOW_SHEAR) return "bad flow_mode";
    if (q.precision != CAHN_FP64 && q.precision != CAHN_MIXED) return "bad precision";
    if (q.krylov != CAHN_GMRES && q.krylov != CAHN_BICGSTAB) return "bad krylov";
    if (q.restart < 1 || q.restart > 64) return "restart must be in 1..64";
    if (q.mg_levels < 1 || q.mg_levels > 16) return "mg_levels must be in 1..16";
    if (q.max_iters < 1) return "max_iters must be >= 1";
    if (!(q.rtol > 0) || !(q.rtol < 1)) return "rtol must be in (0,1)";
    if (q.energy != CAHN_ENERGY_FLORY_HUGGINS && q.energy != CAHN_ENERGY_DOUBLE_WELL) return "bad energy";
    if (q.precond != CAHN_PC_MG && q.precond != CAHN_PC_JACOBI && q.precond != CAHN_PC_SCHWARZ)
        return "bad precond";
    if (q.precond == CAHN_PC_SCHWARZ && (q.nx < 48 || q.ny < 24))
        return "CAHN_PC_SCHWARZ needs nx >= 48 and ny >= 24 (subdomains of 32 x 16 nodes)";
    if (q.nutrient != 0 && q.nutrient != 1) return "nutrient must be 0 or 1";
    if (q.momentum != CAHN_MOM_SPLIT && q.momentum != CAHN_MOM_IMPLICIT) return "bad momentum";
    if (q.nutrient) {
        if (!(q.diff_s >= 0)) return "diff_s must be >= 0";
        if (!(q.growth_mu >= 0) || !(q.growth_eps >= 0)) return "growth_mu, growth_eps must be >= 0";
        if (!(q.growth_kc > 0)) return "growth_kc must be > 0";
        if (!(q.consume_a >= 0)) return "consume_a must be >= 0";
        if (!std::isfinite(q.c_bulk)) return "c_bulk must be finite";
        if (q.nutrient_bc != CAHN_NUT_BC_ZERO_FLUX && q.nutrient_bc != CAHN_NUT_BC_BULK_TOP)
            return "bad nutrient_bc";
    }
    return "";
}

int sm_count() {
    int dev = 0, sms = 0;
    CAHN_CUDA_TRY(cudaGetDevice(&dev));
    CAHN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

// The instances of a batch graph run concurrently, each with at most one
// 5-point V-cycle at a time (u, v and p one after the other): give every
// instance's cooperative V-cycles a share of the device's cooperative
// capacity proportional to its grid, at least one block, so that all of
// them fit at once; if they cannot, the batch keeps the separate launches.
void batch_coop(std::vector<Instance*>& inst) {
    const int cap = Multigrid<float>::coop_capacity();
    double total = 0.0;
    for (Instance* I : inst)
        if (I->mixed && I->use_mg && I->prm.precond == CAHN_PC_MG) total += (double)I->n;
    if (cap <= 0 || total <= 0.0) return;
    std::vector<int> blocks(inst.size(), 0);
    const long nb = (long)inst.size();
    if (nb > cap) return;
    long sum = 0;
    for (size_t k = 0; k < inst.size(); ++k) {
        Instance* I = inst[k];
        if (!(I->mixed && I->use_mg && I->prm.precond == CAHN_PC_MG)) continue;
        // floor((cap - nb) share) + (at most) 1 per instance: the sum stays <= cap
        blocks[k] = std::max(1, (int)std::floor((double)(cap - nb) * (double)I->n / total));
        sum += blocks[k];
    }
    if (sum > cap) return;
    for (size_t k = 0; k < inst.size(); ++k) {
        if (!blocks[k]) continue;
        inst[k]->mg32_h.enable_coop(blocks[k]);
        inst[k]->mg32_p.enable_coop(blocks[k]);
    }
}

// A preconditioner hierarchy: the V-cycle (levels, stop as given) or, with
// CAHN_PC_SCHWARZ, the fine level alone with the domain-decomposition solve.
template <typename T>
void build_pc(Multigrid<T>& m, const Op& op, int levels, size_t stop, RedWs red,
              const cahn_params& q, cudaStream_t s) {
    if (q.precond == CAHN_PC_SCHWARZ) {
        m.build(op, 1, 0, red, s);
        m.enable_schwarz();
    } else {
        m.build(op, levels, stop, red, s);
    }
}

void setup_instance(Instance& I, const cahn_params& q, double* phi, double* u, double* v,
                    double* p, cudaStream_t s, bool batched) {
    I.prm = q;
    I.g = Grid{q.nx, q.ny, q.lx / q.nx, q.ly / q.ny};
    I.n = I.g.n();
    const size_t n = I.n;
    I.phi_c = phi;
    I.u_c = u;
    I.v_c = v;
    I.p_c = p;
    auto F = [&]() { return dalloc<double>(I.allocs, n); };
    I.phi = F(); I.phi_prev = F(); I.phi_new = F();
    I.u = F(); I.u_prev = F(); I.u_new = F();
    I.v = F(); I.v_prev = F(); I.v_new = F();
    I.p = F(); I.p_new = F();
    I.a = F(); I.wr = F(); I.b = F(); I.bu = F(); I.bv = F(); I.d = F();
    I.dinv_ch = F(); I.dinv_h = F(); I.dinv_p = F();
    I.mom.txx = F(); I.mom.txy = F(); I.mom.tyy = F();
    I.mom.ep = F(); I.mom.us = F(); I.mom.vs = F();
    const int stride = std::max(tile_blocks(q.nx, q.ny), VEC_MAX_BLOCKS);
    I.red.stride = stride;
    I.red.partials = dalloc<double>(I.allocs, (size_t)MAX_MULTI * stride);
    I.red.counter = dalloc<unsigned>(I.allocs, 4);
    CAHN_CUDA_TRY(cudaMemset(I.red.counter, 0, 4 * sizeof(unsigned)));
    I.d_sys = dalloc<SysBlock>(I.allocs, 1);
    CAHN_CUDA_TRY(cudaMemset(I.d_sys, 0, sizeof(SysBlock)));
    CAHN_CUDA_TRY(cudaMallocHost(&I.h_sys, sizeof(SysBlock)));
    I.d_status = &I.d_sys->status;
    I.d_nut_status = &I.d_sys->nut_status;
    I.d_coef_status = dalloc<int>(I.allocs, 1);
    CAHN_CUDA_TRY(cudaMemset(I.d_coef_status, 0, sizeof(int)));
    I.d_coef_skip = dalloc<int>(I.allocs, 1);
    CAHN_CUDA_TRY(cudaMemset(I.d_coef_skip, 0, sizeof(int)));
    I.use_graph = q.use_graph != 0;
    // the phase-field hierarchy's set-up reduces into scratch of its own, so
    // that the graph's coefficient branch may run beside the other solves
    I.red_ch.stride = stride;
    I.red_ch.partials = dalloc<double>(I.allocs, (size_t)MAX_MULTI * stride);
    I.red_ch.counter = dalloc<unsigned>(I.allocs, 4);
    CAHN_CUDA_TRY(cudaMemset(I.red_ch.counter, 0, 4 * sizeof(unsigned)));
    if (I.use_graph) {
        CAHN_CUDA_TRY(cudaStreamCreateWithFlags(&I.cbranch, cudaStreamNonBlocking));
        CAHN_CUDA_TRY(cudaEventCreateWithFlags(&I.ev_cfork, cudaEventDisableTiming));
        CAHN_CUDA_TRY(cudaEventCreateWithFlags(&I.ev_cjoin, cudaEventDisableTiming));
        CAHN_CUDA_TRY(cudaEventCreateWithFlags(&I.ev_ejoin, cudaEventDisableTiming));
        for (int k = 0; k < 6; ++k) {
            cudaStream_t c;
            CAHN_CUDA_TRY(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
            I.cap.push_back(c);
        }
        for (GraphSlot& G : I.slot) {
            G.gc.capacity = GRAPH_LOOPS;
            G.gc.body.reserve(GRAPH_LOOPS);
            G.gc.d_counters = dalloc<unsigned>(I.allocs, GRAPH_LOOPS);
            CAHN_CUDA_TRY(cudaMallocHost(&G.h_counters, GRAPH_LOOPS * sizeof(unsigned)));
        }
    }
    I.kw.alloc(I.g, q.restart, true, I.red, q.precond != CAHN_PC_JACOBI && q.precision != CAHN_MIXED);

    // physics constants
    PhysDev& P = I.P;
    P.kappa = q.eps * q.eps;
    P.mobility = q.mobility;
    P.chi = q.chi;
    P.n_poly = q.n_poly;
    P.inv_npoly = 1.0 / q.n_poly;
    P.S = q.stab_s;
    P.gamma2 = q.gamma2;
    P.energy = q.energy;
    P.idt = 1.0 / q.dt;
    P.rho = q.rho_water;
    P.eta_w = q.eta_water;
    P.eta_b = q.eta_biofilm;
    P.eta_bar = std::max(q.eta_water, q.eta_biofilm);
    P.nu = 0.5 * P.eta_bar;
    P.gamma_cap = q.gamma_cap;
    P.fx = q.flow_mode == CAHN_FLOW_POISEUILLE ? 8.0 * q.eta_water * q.u_max / (q.ly * q.ly) : 0.0;
    P.u_wall0 = 0.0;
    P.u_wall1 = q.flow_mode == CAHN_FLOW_SHEAR ? q.u_max : 0.0;

    const double gx = 1.0 / (I.g.hx * I.g.hx), gy = 1.0 / (I.g.hy * I.g.hy);
    Op& oc = I.op_ch;
    oc.g = I.g;
    oc.kind = OP_CH13;
    oc.kx = P.kappa * gx;
    oc.ky = P.kappa * gy;
    oc.S = P.S;
    oc.idt = P.idt;
    oc.gx = gx;
    oc.gy = gy;
    oc.a = I.a;
    Op& oh = I.op_h;
    oh.g = I.g;
    oh.kind = OP_LAP5_DIRICHLET;
    oh.c0 = P.rho * P.idt;
    oh.cx = P.nu * gx;
    oh.cy = P.nu * gy;
    Op& op = I.op_p;
    op.g = I.g;
    op.kind = OP_LAP5_NEUMANN;
    op.c0 = 0.0;
    op.cx = gx;
    op.cy = gy;

    // Jacobi scalings of the constant-coefficient systems
    std::vector<double> h(n);
    for (int j = 0; j <= q.ny; ++j)
        for (int i = 0; i < q.nx; ++i)
            h[(size_t)j * q.nx + i] = (j == 0 || j == q.ny) ? 1.0 / oh.c0
                                                            : 1.0 / (oh.c0 + 2 * oh.cx + 2 * oh.cy);
    CAHN_CUDA_TRY(cudaMemcpy(I.dinv_h, h.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    std::fill(h.begin(), h.end(), 1.0 / (2 * gx + 2 * gy));
    CAHN_CUDA_TRY(cudaMemcpy(I.dinv_p, h.data(), n * sizeof(double), cudaMemcpyHostToDevice));

    // fully implicit momentum: the prep kernel then stores eta itself
    // (eta_bar = 0) for the coupled operator
    I.impl_mom = q.momentum == CAHN_MOM_IMPLICIT;
    if (I.impl_mom) {
        P.eta_bar = 0.0;
        I.g_uv = Grid{q.nx, 2 * q.ny + 1, I.g.hx, I.g.hy};
        I.buv = dalloc<double>(I.allocs, 2 * n);
        I.xuv = dalloc<double>(I.allocs, 2 * n);
        I.dinv_uv = dalloc<double>(I.allocs, 2 * n);
        Op& ov = I.op_uv;
        ov.g = I.g_uv;
        ov.kind = OP_VISC;
        ov.c0 = P.rho * P.idt;
        ov.gx = gx;
        ov.gy = gy;
        ov.kx = 0.25 / (I.g.hx * I.g.hy);
        ov.a = I.mom.ep;
        I.kw_uv.alloc(I.g_uv, 1, false, I.red);
        if (q.precision == CAHN_MIXED) {
            I.eta32 = dalloc<float>(I.allocs, n);
            I.dinv32_uv = dalloc<float>(I.allocs, 2 * n);
            I.r32_uv = dalloc<float>(I.allocs, 2 * n);
            I.d32_uv = dalloc<float>(I.allocs, 2 * n);
            I.op32_uv = ov;
            I.op32_uv.a = I.eta32;
            I.kw32_uv.alloc(I.g_uv, 1, false, I.red);
        }
    }

    // multigrid hierarchies (CH and velocity predictor: up to mg_levels;
    // the singular pressure problem coarsens to a small grid whatever the cap)
    I.use_mg = q.precond == CAHN_PC_MG || q.precond == CAHN_PC_SCHWARZ;   // a hierarchy object
    I.mixed = q.precision == CAHN_MIXED;
    if (I.mixed) {
        auto F32 = [&]() { return dalloc<float>(I.allocs, n); };
        I.a32 = F32();
        I.r32 = F32();
        I.d32 = F32();
        I.dinv32_ch = F32();
        I.dinv32_h = F32();
        I.dinv32_p = F32();
        I.kw32.alloc(I.g, q.restart, true, I.red, q.precond != CAHN_PC_JACOBI);
        I.op32_ch = I.op_ch;
        I.op32_ch.a = I.a32;
        I.op32_h = I.op_h;
        I.op32_p = I.op_p;
        if (I.use_mg) {
            build_pc(I.mg32_ch, I.op32_ch, q.mg_levels, 0, I.red_ch, q, s);
            I.mg32_ch.coarse_iters =
                std::min(I.mg32_ch.coarse_iters, I.mg32_ch.single_block_coarse ? 64 : 3);
            build_pc(I.mg32_h, I.op32_h, q.mg_levels, 0, I.red, q, s);
            build_pc(I.mg32_p, I.op32_p, 16, 512, I.red, q, s);
            // a lone instance runs each 5-point V-cycle as one cooperative
            // launch of one block per SM: the u and v branches may run two at
            // once (a batch sizes its V-cycles in cahn_init)
            if (!batched) {
                const int cap = Multigrid<float>::coop_capacity();
                if (cap >= 2 * sm_count()) {
                    I.mg32_h.enable_coop(sm_count());
                    I.mg32_p.enable_coop(sm_count());
                }
            }
            Instance* self = &I;
            I.pc32_ch = [self](const float* r, float* z, const int* gate, cudaStream_t st) {
                self->mg32_ch.vcycle(r, z, gate, st);
            };
            I.pc32_h = [self](const float* r, float* z, const int* gate, cudaStream_t st) {
                self->mg32_h.vcycle(r, z, gate, st);
            };
            I.pc32_p = [self](const float* r, float* z, const int* gate, cudaStream_t st) {
                self->mg32_p.vcycle(r, z, gate, st);
            };
        }
        launch_convert<double, float>(I.dinv_h, I.dinv32_h, n, s);
        launch_convert<double, float>(I.dinv_p, I.dinv32_p, n, s);
    }
    if (I.use_mg && !I.mixed) {
        build_pc(I.mg_ch, I.op_ch, q.mg_levels, 0, I.red_ch, q, s);
        I.mg_ch.coarse_iters = std::min(I.mg_ch.coarse_iters, I.mg_ch.single_block_coarse ? 64 : 3);
        build_pc(I.mg_h, I.op_h, q.mg_levels, 0, I.red, q, s);
        build_pc(I.mg_p, I.op_p, 16, 512, I.red, q, s);
        Instance* self = &I;
        I.pc_ch = [self](const double* r, double* z, const int* gate, cudaStream_t st) {
            self->mg_ch.vcycle(r, z, gate, st);
        };
        I.pc_h = [self](const double* r, double* z, const int* gate, cudaStream_t st) {
            self->mg_h.vcycle(r, z, gate, st);
        };
        I.pc_p = [self](const double* r, double* z, const int* gate, cudaStream_t st) {
            self->mg_p.vcycle(r, z, gate, st);
        };
    }

    // nutrient: coefficient fields (filled each step), FP32 shadows when mixed
    I.nut = q.nutrient != 0;
    if (I.nut) {
        I.c = F(); I.c_prev = F(); I.c_new = F();
        I.ka = F(); I.kd = F(); I.dinv_c = F(); I.bc = F(); I.gr = F();
        CAHN_CUDA_TRY(cudaMemsetAsync(I.ka, 0, n * 8, s));
        CAHN_CUDA_TRY(cudaMemsetAsync(I.kd, 0, n * 8, s));
        I.d_mass = dalloc<double>(I.allocs, 1);
        NutDev& N = I.N;
        N.diff_s = q.diff_s;
        N.consume_a = q.consume_a;
        N.mu = q.growth_mu;
        N.kc = q.growth_kc;
        N.eps_g = q.growth_eps;
        N.c_bulk = q.c_bulk;
        N.dt = q.dt;
        N.idt = 1.0 / q.dt;
        N.dtop = q.nutrient_bc == CAHN_NUT_BC_BULK_TOP ? 1 : 0;
        Op& on = I.op_c;
        on.g = I.g;
        on.kind = OP_NUT5;
        on.gx = gx;
        on.gy = gy;
        on.a = I.ka;
        on.dg = I.kd;
        on.nut_dtop = I.N.dtop;
        if (I.mixed) {
            I.ka32 = dalloc<float>(I.allocs, n);
            I.kd32 = dalloc<float>(I.allocs, n);
            I.dinv32_c = dalloc<float>(I.allocs, n);
            CAHN_CUDA_TRY(cudaMemsetAsync(I.ka32, 0, n * 4, s));
            CAHN_CUDA_TRY(cudaMemsetAsync(I.kd32, 0, n * 4, s));
            I.op32_c = on;
            I.op32_c.a = I.ka32;
            I.op32_c.dg = I.kd32;
        }
        if (I.use_mg) {
            Instance* self = &I;
            if (I.mixed) {
                build_pc(I.mg32_c, I.op32_c, q.mg_levels, 0, I.red, q, s);
                I.pc32_c = [self](const float* r, float* z, const int* gate, cudaStream_t st) {
                    self->mg32_c.vcycle(r, z, gate, st);
                };
            } else {
                build_pc(I.mg_c, I.op_c, q.mg_levels, 0, I.red, q, s);
                I.pc_c = [self](const double* r, double* z, const int* gate, cudaStream_t st) {
                    self->mg_c.vcycle(r, z, gate, st);
                };
            }
        }
    }

    // tile heights of the fine-grid operators (cached per kind, precision, grid)
    if (I.nut) {
        I.op_c.ty = tune_tile<double>(I.op_c, s);
        if (I.mixed) I.op32_c.ty = tune_tile<float>(I.op32_c, s);
    }
    I.op_ch.ty = tune_tile<double>(I.op_ch, s);
    I.op_h.ty = tune_tile<double>(I.op_h, s);
    I.op_p.ty = tune_tile<double>(I.op_p, s);
    if (I.mixed) {
        I.op32_ch.ty = tune_tile<float>(I.op32_ch, s);
        I.op32_h.ty = tune_tile<float>(I.op32_h, s);
        I.op32_p.ty = tune_tile<float>(I.op32_p, s);
    }

    // graph mode: workspaces of the v predictor solve (its own reduction
    // scratch, Krylov vectors, refinement scratch and hierarchy).  A batch
    // already runs its instances as parallel branches, so only a lone
    // instance splits its step further.
    if (I.use_graph && !batched && !I.impl_mom) {
        I.split_v = true;
        I.red_v.stride = stride;
        I.red_v.partials = dalloc<double>(I.allocs, (size_t)MAX_MULTI * stride);
        I.red_v.counter = dalloc<unsigned>(I.allocs, 4);
        CAHN_CUDA_TRY(cudaMemset(I.red_v.counter, 0, 4 * sizeof(unsigned)));
        I.kw_v.alloc(I.g, q.restart, false, I.red_v);
        Instance* self = &I;
        if (I.mixed) {
            I.kw32_v.alloc(I.g, q.restart, false, I.red_v);
            I.r32_v = dalloc<float>(I.allocs, n);
            I.d32_v = dalloc<float>(I.allocs, n);
            if (I.use_mg) {
                build_pc(I.mg32_h_v, I.op32_h, q.mg_levels, 0, I.red_v, q, s);
                if (Multigrid<float>::coop_capacity() >= 2 * sm_count())
                    I.mg32_h_v.enable_coop(sm_count());
                I.pc32_h_v = [self](const float* r, float* z, const int* gate, cudaStream_t st) {
                    self->mg32_h_v.vcycle(r, z, gate, st);
                };
            }
        } else if (I.use_mg) {
            build_pc(I.mg_h_v, I.op_h, q.mg_levels, 0, I.red_v, q, s);
            I.pc_h_v = [self](const double* r, double* z, const int* gate, cudaStream_t st) {
                self->mg_h_v.vcycle(r, z, gate, st);
            };
        }
        CAHN_CUDA_TRY(cudaStreamCreateWithFlags(&I.vbranch, cudaStreamNonBlocking));
        CAHN_CUDA_TRY(cudaEventCreateWithFlags(&I.ev_fork, cudaEventDisableTiming));
        CAHN_CUDA_TRY(cudaEventCreateWithFlags(&I.ev_join, cudaEventDisableTiming));
    }

    I.sumw = (double)q.nx * (q.ny - 1) + (double)q.nx;   // interior rows + two half rows
    I.inv_sumw = 1.0 / I.sumw;

    // state: q^{-1} = q^0
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi, phi, n * 8, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi_prev, phi, n * 8, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.u, u, n * 8, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.u_prev, u, n * 8, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.v, v, n * 8, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.v_prev, v, n * 8, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.p, p, n * 8, cudaMemcpyDeviceToDevice, s));
    launch_wdot<double>(I.g, I.phi, (const double*)nullptr, I.kw.sd, S_MASS, 1.0, nullptr, s);
    I.kw.read_back(s);
    I.m0 = I.kw.h_scal[S_MASS];
    if (I.nut) CAHN_CUDA_TRY(cudaMemcpy(I.d_mass, &I.m0, sizeof(double), cudaMemcpyHostToDevice));
}

int status_code(int st) {
    if (st & CTL_DOMAIN) return CAHN_ERR_DOMAIN;
    if (st & CTL_NAN) return CAHN_ERR_NAN;
    if (st & CTL_NOT_CONVERGED) return CAHN_ERR_NOT_CONVERGED;
    return CAHN_OK;
}

const char* sys_name(int s) {
    static const char* names[CAHN_NSYS] = {"phi", "u", "v", "p", "c"};
    return (s >= 0 && s < CAHN_NSYS) ? names[s] : "?";
}

void copy_in(Instance& I, cudaStream_t s) {
    const size_t b = I.n * sizeof(double);
    I.coef_valid = false;
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi, I.phi_c, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.u, I.u_c, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.v, I.v_c, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.p, I.p_c, b, cudaMemcpyDeviceToDevice, s));
    if (I.nut_ready) CAHN_CUDA_TRY(cudaMemcpyAsync(I.c, I.c_c, b, cudaMemcpyDeviceToDevice, s));
}
void copy_out(Instance& I, cudaStream_t s) {
    const size_t b = I.n * sizeof(double);
    if (I.nut_ready) CAHN_CUDA_TRY(cudaMemcpyAsync(I.c_c, I.c, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi_c, I.phi, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.u_c, I.u, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.v_c, I.v, b, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.p_c, I.p, b, cudaMemcpyDeviceToDevice, s));
}

// Route the Krylov workspaces' bookkeeping to system `sys`'s blocks.
void use_sys(Instance& I, int sys) {
    I.kw.sd.ctl = &I.d_sys->ctl64[sys];
    I.kw.sd.scal = I.d_sys->scal64[sys];
    if (I.mixed) {
        I.kw32.sd.ctl = &I.d_sys->ctl32[sys];
        I.kw32.sd.scal = I.d_sys->scal32[sys];
    }
}

// Record one solve's result (host mode); returns a CAHN code.
int record(Instance& I, int sys, const SolveResult& r, cahn_stats& st) {
    st.iters[sys] += r.it;
    st.resid[sys] = r.rel_res;
    int code = status_code(r.status);
    if (code != CAHN_OK && st.failed_system < 0) st.failed_system = sys;
    return code;
}
int record_ir(Instance& I, int sys, const IrResult& r, cahn_stats& st) {
    st.outer[sys] += r.outer.it;
    SolveResult s2 = r.outer;
    s2.it = r.inner_it;
    return record(I, sys, s2, st);
}

// FP32 inner tolerance and refinement cap of the mixed form.  A
// multigrid-preconditioned inner solve that has not met its tolerance in
// IR_INNER_MG_CAP iterations hands back to the FP64 refinement.
constexpr double IR_INNER_RTOL = 1e-5;
constexpr int IR_MAX_OUTER = 30;
constexpr int IR_INNER_MG_CAP = 60;
// Upper bound of ||A|| for the refinement's rounding floor: the
// checkerboard eigenvalue of the 5-point operators; for A_phi the bound
// with the largest mobility coefficient a <= M (phi* < 1).
inline double anorm(const Op& op, double mobility) {
    if (op.kind == OP_NUT5) return 0.0;   // see anorm_nut
    if (op.kind != OP_CH13) return op.c0 + 4.0 * op.cx + 4.0 * op.cy;
    const double lam = 4.0 * op.gx + 4.0 * op.gy;
    return op.idt + 0.5 * mobility * lam * ((4.0 * op.kx + 4.0 * op.ky) + op.S);
}
// ||K|| <= 1/dt + A/2 + 2 D_s (1/hx^2 + 1/hy^2) for phi in (0, 1)
inline double anorm_nut(const Instance& I) {
    return I.N.idt + 0.5 * I.N.consume_a + 2.0 * I.N.diff_s * (I.op_c.gx + I.op_c.gy);
}
inline int inner_cap(const Instance& I) {
    return I.use_mg ? std::min(I.prm.max_iters, IR_INNER_MG_CAP) : I.prm.max_iters;
}

// The phase-field coefficient a = M phi*, the explicit part wr and the
// preconditioner's set-up, from phi^n = phi and phi^{n-1} = phi_prev; the
// domain check of phi* into status.  gate (may be null): the heavy
// launches return at once while *gate != 0.
void coefficient(Instance& I, cudaStream_t s, const double* phi, const double* phi_prev,
                 int* status, const int* gate = nullptr) {
    launch_ch_prep(I.g, I.P, phi, phi_prev, I.a, I.mixed ? I.a32 : nullptr, I.wr, status, gate, s);
    if (I.mixed) {
        if (I.use_mg) {
            I.mg32_ch.set_coefficient(I.a32, s, gate);
        } else {
            launch_ch13_diag<float>(I.op32_ch, I.dinv32_ch, s);
            launch_invert<float>(I.n, I.dinv32_ch, s);
        }
    } else if (I.use_mg) {
        I.mg_ch.set_coefficient(I.a, s, gate);
    } else {
        launch_ch13_diag<double>(I.op_ch, I.dinv_ch, s);
        launch_invert<double>(I.n, I.dinv_ch, s);
    }
}
// the coefficient of the current state, formed now
void coefficient(Instance& I, cudaStream_t s) {
    coefficient(I, s, I.phi, I.phi_prev, I.d_status);
    I.coef_valid = true;
}

int domain_status(Instance& I, cudaStream_t s) {
    CAHN_CUDA_TRY(cudaMemcpyAsync(&I.h_sys->status, I.d_status, sizeof(int),
                                  cudaMemcpyDeviceToHost, s));
    CAHN_CUDA_TRY(cudaStreamSynchronize(s));
    return I.h_sys->status;
}

int nut_domain_status(Instance& I, cudaStream_t s) {
    CAHN_CUDA_TRY(cudaMemcpyAsync(&I.h_sys->nut_status, I.d_nut_status, sizeof(int),
                                  cudaMemcpyDeviceToHost, s));
    CAHN_CUDA_TRY(cudaStreamSynchronize(s));
    return I.h_sys->nut_status;
}

int solve_phi(Instance& I, double* x, const double* b, Driver& d, cahn_stats& st) {
    const cahn_params& q = I.prm;
    use_sys(I, CAHN_SYS_PHI);
    const bool bicg = q.krylov == CAHN_BICGSTAB;
    if (I.mixed) {
        InnerSolve inner = [&](const float* rhs, float* sol, Driver& di, const int* skip) {
            auto solve = bicg ? bicgstab_solve<float> : gmres_solve<float>;
            return solve(I.kw32, I.op32_ch, sol, rhs, I.use_mg ? nullptr : I.dinv32_ch,
                         I.use_mg ? &I.pc32_ch : nullptr, IR_INNER_RTOL, inner_cap(I),
                         I.predict32[CAHN_SYS_PHI], di, skip, true);
        };
        IrResult r = ir_solve(I.kw, I.op_ch, x, b, I.r32, I.d32, inner, q.rtol, IR_MAX_OUTER,
                              false, I.inv_sumw, anorm(I.op_ch, I.P.mobility), d);
        return record_ir(I, CAHN_SYS_PHI, r, st);
    }
    auto solve = bicg ? bicgstab_solve<double> : gmres_solve<double>;
    SolveResult r = solve(I.kw, I.op_ch, x, b, I.use_mg ? nullptr : I.dinv_ch,
                          I.use_mg ? &I.pc_ch : nullptr, q.rtol, q.max_iters,
                          I.predict[CAHN_SYS_PHI], d, nullptr, false);
    return record(I, CAHN_SYS_PHI, r, st);
}
int solve_h(Instance& I, int sys, double* x, const double* b, Driver& d, cahn_stats& st) {
    const cahn_params& q = I.prm;
    use_sys(I, sys);
    // the v solve of a graph-mode step runs beside the u solve, on its own
    // workspaces (same arithmetic: only the memory differs)
    const bool alt = sys == CAHN_SYS_V && I.split_v && d.graph;
    KrylovWs<double>& kw = alt ? I.kw_v : I.kw;
    KrylovWs<float>& kw32 = alt ? I.kw32_v : I.kw32;
    float* r32 = alt ? I.r32_v : I.r32;
    float* d32 = alt ? I.d32_v : I.d32;
    const PrecFn<double>* pc = alt ? &I.pc_h_v : &I.pc_h;
    const PrecFn<float>* pc32 = alt ? &I.pc32_h_v : &I.pc32_h;
    if (alt) {
        kw.sd.ctl = &I.d_sys->ctl64[sys];
        kw.sd.scal = I.d_sys->scal64[sys];
        if (I.mixed) {
            kw32.sd.ctl = &I.d_sys->ctl32[sys];
            kw32.sd.scal = I.d_sys->scal32[sys];
        }
    }
    launch_dirichlet_walls<double>(I.g, x, b, 1.0 / I.op_h.c0, d.s);
    if (I.mixed) {
        InnerSolve inner = [&](const float* rhs, float* sol, Driver& di, const int* skip) {
            return cg_solve<float>(kw32, I.op32_h, sol, rhs, I.use_mg ? nullptr : I.dinv32_h,
                                   I.use_mg ? pc32 : nullptr, IR_INNER_RTOL, inner_cap(I),
                                   false, I.inv_sumw, I.predict32[sys], di, skip, true);
        };
        IrResult r = ir_solve(kw, I.op_h, x, b, r32, d32, inner, q.rtol, IR_MAX_OUTER,
                              false, I.inv_sumw, anorm(I.op_h, 0.0), d);
        return record_ir(I, sys, r, st);
    }
    SolveResult r = cg_solve<double>(kw, I.op_h, x, b, I.use_mg ? nullptr : I.dinv_h,
                                     I.use_mg ? pc : nullptr, q.rtol, q.max_iters, false,
                                     I.inv_sumw, I.predict[sys], d);
    return record(I, sys, r, st);
}
// ||A|| bound of the coupled momentum operator (Gershgorin): rho/dt plus
// max(eta) times the absolute row sums of div(2 eta D(.)) / 2
inline double anorm_uv(const Instance& I) {
    const double em = std::max(I.prm.eta_water, I.prm.eta_biofilm);
    return I.op_uv.c0 + em * (4.0 * I.op_uv.gx + 4.0 * I.op_uv.gy + 2.0 * I.op_uv.kx);
}

// The coupled system stops on one norm of [u; v], dominated by the larger
// component (u is about 30x v on the workloads); it runs at rtol / 100 so
// that v, and the pressure it drives, keep the accuracy that the separate
// predictor solves of the split form give them.
constexpr double UV_RTOL_FACTOR = 1e-2;

// The coupled momentum system on stacked [u; v] (coefficient eta in mom.ep,
// its FP32 shadow already converted); statistics in the U slot.  Jacobi:
// the inverse diagonal of both blocks, formed from eta.
int solve_uv(Instance& I, double* x, const double* b, Driver& d, cahn_stats& st) {
    const cahn_params& q = I.prm;
    const double rtol = q.rtol * UV_RTOL_FACTOR;
    const size_t n = I.n;
    I.kw_uv.sd.ctl = &I.d_sys->ctl64[CAHN_SYS_U];
    I.kw_uv.sd.scal = I.d_sys->scal64[CAHN_SYS_U];
    const double inv_c0 = 1.0 / I.op_uv.c0;
    launch_dirichlet_walls<double>(I.g, x, b, inv_c0, d.s);
    launch_dirichlet_walls<double>(I.g, x + n, b + n, inv_c0, d.s);
    if (I.mixed) {
        I.kw32_uv.sd.ctl = &I.d_sys->ctl32[CAHN_SYS_U];
        I.kw32_uv.sd.scal = I.d_sys->scal32[CAHN_SYS_U];
        launch_visc_dinv<float>(I.op32_uv, I.dinv32_uv, d.s);
        InnerSolve inner = [&](const float* rhs, float* sol, Driver& di, const int* skip) {
            return cg_solve<float>(I.kw32_uv, I.op32_uv, sol, rhs, I.dinv32_uv, nullptr,
                                   IR_INNER_RTOL, q.max_iters, false, I.inv_sumw,
                                   I.predict32[CAHN_SYS_U], di, skip, true);
        };
        IrResult r = ir_solve(I.kw_uv, I.op_uv, x, b, I.r32_uv, I.d32_uv, inner, rtol,
                              IR_MAX_OUTER, false, I.inv_sumw, anorm_uv(I), d);
        return record_ir(I, CAHN_SYS_U, r, st);
    }
    launch_visc_dinv<double>(I.op_uv, I.dinv_uv, d.s);
    SolveResult r = cg_solve<double>(I.kw_uv, I.op_uv, x, b, I.dinv_uv, nullptr, rtol,
                                     q.max_iters, false, I.inv_sumw, I.predict[CAHN_SYS_U], d);
    return record(I, CAHN_SYS_U, r, st);
}

// eta at the current phi (single solves and applies of CAHN_SYS_UV)
void uv_coefficient(Instance& I, cudaStream_t s) {
    launch_mom_prep(I.g, I.P, I.phi, I.phi, I.u, I.u_prev, I.v, I.v_prev, I.mom, s);
    if (I.mixed) launch_convert<double, float>(I.mom.ep, I.eta32, I.n, s);
}

int solve_p(Instance& I, double* x, const double* b, Driver& d, cahn_stats& st) {
    const cahn_params& q = I.prm;
    use_sys(I, CAHN_SYS_P);
    if (I.mixed) {
        InnerSolve inner = [&](const float* rhs, float* sol, Driver& di, const int* skip) {
            return cg_solve<float>(I.kw32, I.op32_p, sol, rhs, I.use_mg ? nullptr : I.dinv32_p,
                                   I.use_mg ? &I.pc32_p : nullptr, IR_INNER_RTOL, inner_cap(I),
                                   true, I.inv_sumw, I.predict32[CAHN_SYS_P], di, skip, true);
        };
        IrResult r = ir_solve(I.kw, I.op_p, x, b, I.r32, I.d32, inner, q.rtol, IR_MAX_OUTER,
                              true, I.inv_sumw, anorm(I.op_p, 0.0), d);
        return record_ir(I, CAHN_SYS_P, r, st);
    }
    SolveResult r = cg_solve<double>(I.kw, I.op_p, x, b, I.use_mg ? nullptr : I.dinv_p,
                                     I.use_mg ? &I.pc_p : nullptr, q.rtol, q.max_iters, true,
                                     I.inv_sumw, I.predict[CAHN_SYS_P], d);
    return record(I, CAHN_SYS_P, r, st);
}

// Nutrient system (CAHN_SYS_C): CG preconditioned by the V-cycle or by
// Jacobi, or FP64 refinement around FP32 CG.  x holds the initial guess (with
// the Dirichlet top row when the top wall holds c_bulk).
int solve_c(Instance& I, double* x, const double* b, Driver& d, cahn_stats& st) {
    const cahn_params& q = I.prm;
    use_sys(I, CAHN_SYS_C);
    if (I.mixed) {
        InnerSolve inner = [&](const float* rhs, float* sol, Driver& di, const int* skip) {
            return cg_solve<float>(I.kw32, I.op32_c, sol, rhs, I.use_mg ? nullptr : I.dinv32_c,
                                   I.use_mg ? &I.pc32_c : nullptr, IR_INNER_RTOL, inner_cap(I),
                                   false, I.inv_sumw, I.predict32[CAHN_SYS_C], di, skip, true);
        };
        IrResult r = ir_solve(I.kw, I.op_c, x, b, I.r32, I.d32, inner, q.rtol, IR_MAX_OUTER,
                              false, I.inv_sumw, anorm_nut(I), d);
        return record_ir(I, CAHN_SYS_C, r, st);
    }
    SolveResult r = cg_solve<double>(I.kw, I.op_c, x, b, I.use_mg ? nullptr : I.dinv_c,
                                     I.use_mg ? &I.pc_c : nullptr, q.rtol, q.max_iters, false,
                                     I.inv_sumw, I.predict[CAHN_SYS_C], d);
    return record(I, CAHN_SYS_C, r, st);
}

// Coefficients of the nutrient hierarchy from the fine fields just formed.
void nut_hierarchy(Instance& I, cudaStream_t s) {
    if (!I.use_mg) return;
    if (I.mixed)
        I.mg32_c.set_coefficients(I.ka32, I.kd32, s);
    else
        I.mg_c.set_coefficients(I.ka, I.kd, s);
}

// Frozen-coefficient nutrient operator (phi^{n+1} = phi^n = phi) of single
// solves and applies.
void nut_coefficients(Instance& I, cudaStream_t s) {
    launch_nut_prep(I.g, I.N, I.phi, I.phi, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, I.ka, I.kd, I.dinv_c, nullptr, nullptr, I.ka32, I.kd32, I.dinv32_c,
                    nullptr, s);
    nut_hierarchy(I, s);
}

void rotate(Instance& I) {
    I.coef_valid = false;
    if (I.nut) {
        std::swap(I.c_prev, I.c);
        std::swap(I.c, I.c_new);
    }
    std::swap(I.phi_prev, I.phi);
    std::swap(I.phi, I.phi_new);
    std::swap(I.u_prev, I.u);
    std::swap(I.u, I.u_new);
    std::swap(I.v_prev, I.v);
    std::swap(I.v, I.v_new);
}

// p = p_new unless a solve or the phase-field rhs of this step failed
// (then the step leaves every field at its start value).
__global__ void k_commit_p(size_t n, const double* __restrict__ src, double* __restrict__ dst,
                           const SysBlock* __restrict__ sb) {
    int bad = sb->status | sb->nut_status;
    for (int k = 0; k < CAHN_NSYS; ++k) bad |= sb->ctl64[k].status | (sb->ctl32[k].status & CTL_NAN);
    if (bad) return;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// The mass target of the next step (scal[S_TMP0], written by the grown
// mass correction), unless a solve or the phase-field rhs failed.
__global__ void k_commit_mass(const SysBlock* __restrict__ sb, double* __restrict__ m) {
    int bad = sb->status | sb->nut_status;
    for (int k = 0; k < CAHN_NSYS; ++k) bad |= sb->ctl64[k].status | (sb->ctl32[k].status & CTL_NAN);
    if (!bad && threadIdx.x == 0) m[0] = sb->scal64[CAHN_SYS_PHI][S_TMP0];
}

// One time step: in host mode it runs and checks as it goes; in graph mode
// it is being captured and every decision is taken on the device.
int step_body(Instance& I, Driver& d, cahn_stats& st) {
    const cudaStream_t s = d.s;
    const bool host = !d.graph;
    const size_t n = I.n, nb = n * sizeof(double);
    // 1-2. phase field (graph mode: the coefficient was formed before the
    // launch, or by the previous step's graph)
    if (host) {
        CAHN_CUDA_TRY(cudaMemsetAsync(I.d_status, 0, 2 * sizeof(int), s));   // both statuses
        coefficient(I, s);
    }
    launch_ch_rhs(I.g, I.P, I.phi, I.phi_prev, I.u, I.u_prev, I.v, I.v_prev, I.a, I.wr, I.b,
                  host ? nullptr : I.d_coef_status, I.d_status, s);
    if (I.nut) launch_growth(I.g, I.N, I.phi, I.phi_prev, I.c, I.c_prev, I.b, I.gr, s);
    if (host && (domain_status(I, s) & CTL_DOMAIN)) {
        st.failed_system = CAHN_SYS_PHI;
        return CAHN_ERR_DOMAIN;
    }
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi_new, I.phi, nb, cudaMemcpyDeviceToDevice, s));
    int code = solve_phi(I, I.phi_new, I.b, d, st);
    if (host && code) return code;
    // 3. mass correction (bookkeeping in the phi system's scalars); with the
    // production on, the target grows by dt <g_n, 1>_W
    launch_wdot<double>(I.g, I.phi_new, (const double*)nullptr, I.kw.sd, S_MASS, 1.0, nullptr, s);
    if (I.nut) {
        launch_wdot<double>(I.g, I.gr, (const double*)nullptr, I.kw.sd, S_TMP1, I.prm.dt, nullptr, s);
        launch_mass_fix_grow(n, I.phi_new, I.kw.sd.scal, I.d_mass, I.inv_sumw, s);
    } else {
        launch_mass_fix(n, I.phi_new, I.kw.sd.scal, I.m0, I.inv_sumw, s);
    }
    if (host) {
        I.kw.read_back(s);
        const double target = I.nut ? I.kw.h_scal[S_TMP0] : I.m0;
        st.mass_drift = target != 0.0 ? (I.kw.h_scal[S_MASS] - target) / target : 0.0;
    }
    // graph mode: the next step's coefficient from phi^{n+1} and phi^n, on a
    // branch of its own beside the predictor and pressure solves (joined at
    // the end of the step).  It forks after the momentum rhs, whose FP64
    // work it would otherwise share the FP64 pipe with; nothing after that
    // point reads a, a32, wr or the phase-field hierarchy.
    auto fork_coefficient = [&]() {
        if (host) return;
        CAHN_CUDA_TRY(cudaEventRecord(I.ev_cfork, s));
        CAHN_CUDA_TRY(cudaStreamWaitEvent(I.cbranch, I.ev_cfork, 0));
        coefficient(I, I.cbranch, I.phi_new, I.phi, I.d_coef_status, I.d_coef_skip);
        CAHN_CUDA_TRY(cudaEventRecord(I.ev_cjoin, I.cbranch));
    };
    // nutrient (Eq. 2.6) with the corrected phi^{n+1}
    if (I.nut) {
        launch_nut_prep(I.g, I.N, I.phi_new, I.phi, I.phi_prev, I.c, I.c_prev, I.u, I.u_prev,
                        I.v, I.v_prev, I.ka, I.kd, I.dinv_c, I.bc, I.c_new, I.ka32, I.kd32,
                        I.dinv32_c, I.d_nut_status, s);
        if (host && (nut_domain_status(I, s) & CTL_DOMAIN)) {
            st.failed_system = CAHN_SYS_C;
            return CAHN_ERR_DOMAIN;
        }
        nut_hierarchy(I, s);
        if ((code = solve_c(I, I.c_new, I.bc, d, st)) && host) return code;
    }
    // 4-5. velocity predictor
    launch_mom_prep(I.g, I.P, I.phi_new, I.phi, I.u, I.u_prev, I.v, I.v_prev, I.mom, s);
    if (I.impl_mom) {
        // one coupled solve on [u; v], started from [u^n; v^n]
        launch_mom_rhs_impl(I.g, I.P, I.u, I.v, I.mom, I.buv, I.buv + n, s);
        if (I.mixed) launch_convert<double, float>(I.mom.ep, I.eta32, n, s);
        fork_coefficient();
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.xuv, I.u, nb, cudaMemcpyDeviceToDevice, s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.xuv + n, I.v, nb, cudaMemcpyDeviceToDevice, s));
        code = solve_uv(I, I.xuv, I.buv, d, st);
        if (host && code) return code;
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.u_new, I.xuv, nb, cudaMemcpyDeviceToDevice, s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.v_new, I.xuv + n, nb, cudaMemcpyDeviceToDevice, s));
    } else {
    launch_mom_rhs(I.g, I.P, I.u, I.v, I.mom, I.bu, I.bv, s);
    fork_coefficient();
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.u_new, I.u, nb, cudaMemcpyDeviceToDevice, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.v_new, I.v, nb, cudaMemcpyDeviceToDevice, s));
    if (!host && I.split_v) {
        // graph mode: the u and v solves are parallel branches (fork, join)
        CAHN_CUDA_TRY(cudaEventRecord(I.ev_fork, s));
        CAHN_CUDA_TRY(cudaStreamWaitEvent(I.vbranch, I.ev_fork, 0));
        Driver dv = d;
        dv.s = I.vbranch;
        solve_h(I, CAHN_SYS_U, I.u_new, I.bu, d, st);
        solve_h(I, CAHN_SYS_V, I.v_new, I.bv, dv, st);
        CAHN_CUDA_TRY(cudaEventRecord(I.ev_join, I.vbranch));
        CAHN_CUDA_TRY(cudaStreamWaitEvent(s, I.ev_join, 0));
    } else {
        if ((code = solve_h(I, CAHN_SYS_U, I.u_new, I.bu, d, st)) && host) return code;
        if ((code = solve_h(I, CAHN_SYS_V, I.v_new, I.bv, d, st)) && host) return code;
    }
    }
    // 6. pressure (projection bookkeeping in the p system's scalars)
    use_sys(I, CAHN_SYS_P);
    launch_div(I.g, I.P.rho, I.u_new, I.v_new, I.d, s);
    launch_wdot<double>(I.g, I.d, (const double*)nullptr, I.kw.sd, S_TMP3, I.inv_sumw, nullptr, s);
    launch_sub_scalar<double>(I.d, n, I.kw.sd.scal + S_TMP3, nullptr, s);
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.p_new, I.p, nb, cudaMemcpyDeviceToDevice, s));
    if ((code = solve_p(I, I.p_new, I.d, d, st)) && host) return code;
    // 7. correction, then commit the pressure
    launch_correct(I.g, 1.0 / I.P.rho, I.p_new, I.u_new, I.v_new, s);
    note_launch();
    launch_k(k_commit_p, vec_blocks(n), RED_THREADS, 0, s, n, I.p_new, I.p, I.d_sys);
    if (I.nut) {
        note_launch();
        launch_k(k_commit_mass, dim3(1), dim3(32), 0, s, (const SysBlock*)I.d_sys, I.d_mass);
    }
    if (host) {
        rotate(I);
        st.steps += 1;
    } else {
        CAHN_CUDA_TRY(cudaStreamWaitEvent(s, I.ev_cjoin, 0));
    }
    return CAHN_OK;
}

// Capture one step (for the current buffer phase) into a graph.
void capture_step(Instance& I, GraphSlot& G) {
    cudaStream_t cs = I.cap[0];
    const int64_t noted = g_launches.load();   // capture is not execution
    G.gc.top = 0;
    G.gc.body.clear();
    CAHN_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    Driver d;
    d.s = cs;
    d.graph = true;
    d.pool = &I.cap;
    d.depth = 0;
    d.gc = &G.gc;
    cahn_stats dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    set_launch_frame(&G.gc.top);
    try {
        CAHN_CUDA_TRY(cudaMemsetAsync(G.gc.d_counters, 0, GRAPH_LOOPS * sizeof(unsigned), cs));
        CAHN_CUDA_TRY(cudaMemsetAsync(I.d_sys, 0, sizeof(SysBlock), cs));
        step_body(I, d, dummy);
    } catch (...) {
        set_launch_frame(nullptr);
        cudaGraph_t broken = nullptr;
        cudaStreamEndCapture(cs, &broken);
        if (broken) cudaGraphDestroy(broken);
        cudaGetLastError();
        throw;
    }
    set_launch_frame(nullptr);
    g_launches.store(noted);
    cudaGraph_t graph = nullptr;
    CAHN_CUDA_TRY(cudaStreamEndCapture(cs, &graph));
    cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    CAHN_CUDA_TRY(e);
}

// Statistics of one replayed step of instance I (its SysBlock and loop
// counters already copied to the host); rotates the buffers on success.
int collect_graph_step(Instance& I, GraphSlot& G, cahn_stats& st, int64_t& launches) {
    int64_t l = G.gc.top;
    for (size_t k = 0; k < G.gc.body.size(); ++k) l += G.gc.body[k] * (int64_t)G.h_counters[k];
    launches += l;
    const SysBlock& B = *I.h_sys;
    int code = CAHN_OK;
    if (B.status & CTL_DOMAIN) {
        code = CAHN_ERR_DOMAIN;
        st.failed_system = CAHN_SYS_PHI;
    } else if (B.nut_status & CTL_DOMAIN) {
        code = CAHN_ERR_DOMAIN;
        st.failed_system = CAHN_SYS_C;
    }
    for (int sys = 0; sys < CAHN_NSYS; ++sys) {
        const Ctl& c64 = B.ctl64[sys];
        if (I.mixed) {
            st.outer[sys] += c64.total;
            st.iters[sys] += B.ctl32[sys].total;
        } else {
            st.iters[sys] += c64.total;
        }
        const double bn = B.scal64[sys][S_BN];
        st.resid[sys] = bn > 0 ? B.scal64[sys][S_RES0] / bn : 0.0;
        const int c = status_code(c64.status | (I.mixed ? (B.ctl32[sys].status & CTL_NAN) : 0));
        if (c != CAHN_OK && code == CAHN_OK) {
            code = c;
            st.failed_system = sys;
        }
    }
    const double target = I.nut ? B.scal64[CAHN_SYS_PHI][S_TMP0] : I.m0;
    st.mass_drift = target != 0.0 ? (B.scal64[CAHN_SYS_PHI][S_MASS] - target) / target : 0.0;
    if (code != CAHN_OK) return code;
    rotate(I);
    st.steps += 1;
    return CAHN_OK;
}

void queue_readback(Instance& I, GraphSlot& G, cudaStream_t s) {
    CAHN_CUDA_TRY(cudaMemcpyAsync(I.h_sys, I.d_sys, sizeof(SysBlock), cudaMemcpyDeviceToHost, s));
    CAHN_CUDA_TRY(cudaMemcpyAsync(G.h_counters, G.gc.d_counters, GRAPH_LOOPS * sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, s));
}

// Graph mode: the coefficient of the current state, stream-ordered before
// the step graph, unless the previous step's graph formed it (its domain
// check into coef_status either way).
void graph_coefficient(Instance& I, cudaStream_t s) {
    if (I.coef_valid) return;
    CAHN_CUDA_TRY(cudaMemsetAsync(I.d_coef_status, 0, sizeof(int), s));
    coefficient(I, s, I.phi, I.phi_prev, I.d_coef_status);
    I.coef_valid = true;
}
// The branch of the step about to run forms the next coefficient unless
// this is the call's last step (nothing would use it: the next call starts
// from copy_in).
void graph_coefficient_branch(Instance& I, cudaStream_t s, bool last) {
    CAHN_CUDA_TRY(cudaMemsetAsync(I.d_coef_skip, last ? 1 : 0, sizeof(int), s));
}
// After a graph step: the coefficient its branch formed belongs to the new
// state if the step succeeded and the branch ran.
void graph_step_done(Instance& I, int code, bool last) { I.coef_valid = code == CAHN_OK && !last; }

// Graph mode: replay the captured step, then read every statistic back
// with one copy; the buffers rotate only after a successful step.  last:
// the call's last step (its coefficient branch returns at once).
int step_graph(Instance& I, cudaStream_t s, cahn_stats& st, int64_t& launches, bool last) {
    graph_coefficient(I, s);
    graph_coefficient_branch(I, s, last);
    GraphSlot& G = I.slot[I.phase];
    if (!G.exec) capture_step(I, G);
    CAHN_CUDA_TRY(cudaGraphLaunch(G.exec, s));
    queue_readback(I, G, s);
    CAHN_CUDA_TRY(cudaStreamSynchronize(s));
    const int code = collect_graph_step(I, G, st, launches);
    graph_step_done(I, code, last);
    if (code == CAHN_OK) I.phase = (I.phase + 1) % 3;
    return code;
}

// Capture one step of every instance into one graph: a fork event on the
// capture stream, one branch per instance on its own capture streams, a
// join back.
void capture_batch(cahn_ctx* c, int ph) {
    cudaStream_t cs = c->bcap;
    const int64_t noted = g_launches.load();
    CAHN_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        CAHN_CUDA_TRY(cudaEventRecord(c->fork, cs));
        for (size_t k = 0; k < c->inst.size(); ++k) {
            Instance& I = *c->inst[k];
            GraphSlot& G = I.slot[ph];
            G.gc.top = 0;
            G.gc.body.clear();
            cudaStream_t sk = I.cap[0];
            CAHN_CUDA_TRY(cudaStreamWaitEvent(sk, c->fork, 0));
            Driver d;
            d.s = sk;
            d.graph = true;
            d.pool = &I.cap;
            d.gc = &G.gc;
            set_launch_frame(&G.gc.top);
            CAHN_CUDA_TRY(cudaMemsetAsync(G.gc.d_counters, 0, GRAPH_LOOPS * sizeof(unsigned), sk));
            CAHN_CUDA_TRY(cudaMemsetAsync(I.d_sys, 0, sizeof(SysBlock), sk));
            cahn_stats dummy;
            std::memset(&dummy, 0, sizeof(dummy));
            step_body(I, d, dummy);
            set_launch_frame(nullptr);
            CAHN_CUDA_TRY(cudaEventRecord(c->join[k], sk));
            CAHN_CUDA_TRY(cudaStreamWaitEvent(cs, c->join[k], 0));
        }
    } catch (...) {
        set_launch_frame(nullptr);
        cudaGraph_t broken = nullptr;
        cudaStreamEndCapture(cs, &broken);
        if (broken) cudaGraphDestroy(broken);
        cudaGetLastError();
        g_launches.store(noted);
        throw;
    }
    g_launches.store(noted);
    cudaGraph_t graph = nullptr;
    CAHN_CUDA_TRY(cudaStreamEndCapture(cs, &graph));
    cudaError_t e = cudaGraphInstantiate(&c->bexec[ph], graph, 0);
    cudaGraphDestroy(graph);
    CAHN_CUDA_TRY(e);
}

// Batched graph mode: one graph launch advances every instance one step.
// An instance whose step failed keeps its step-start state; the batch
// graphs are then dropped and recaptured with the current buffers.
int step_batch(cahn_ctx* c, cahn_stats* sts, int64_t& launches, int& failed, bool last) {
    const int ph = c->bphase;
    // the coefficients the previous step did not form, one instance per
    // branch stream, joined back before the graph
    CAHN_CUDA_TRY(cudaEventRecord(c->cfork, c->s));
    for (Instance* I : c->inst) {
        if (!I->coef_valid) {
            CAHN_CUDA_TRY(cudaStreamWaitEvent(I->cbranch, c->cfork, 0));
            graph_coefficient(*I, I->cbranch);
            CAHN_CUDA_TRY(cudaEventRecord(I->ev_ejoin, I->cbranch));
            CAHN_CUDA_TRY(cudaStreamWaitEvent(c->s, I->ev_ejoin, 0));
        }
        graph_coefficient_branch(*I, c->s, last);
    }
    if (!c->bexec[ph]) capture_batch(c, ph);
    CAHN_CUDA_TRY(cudaGraphLaunch(c->bexec[ph], c->s));
    for (Instance* I : c->inst) queue_readback(*I, I->slot[ph], c->s);
    CAHN_CUDA_TRY(cudaStreamSynchronize(c->s));
    int ret = CAHN_OK;
    for (size_t k = 0; k < c->inst.size(); ++k) {
        const int code = collect_graph_step(*c->inst[k], c->inst[k]->slot[ph], sts[k], launches);
        sts[k].status = code;
        if (code != CAHN_OK && ret == CAHN_OK) {
            ret = code;
            failed = (int)k;
        }
    }
    // after a failed batch step every instance forms its coefficient again
    for (Instance* I : c->inst) graph_step_done(*I, ret, last);
    if (ret == CAHN_OK)
        c->bphase = (ph + 1) % 3;
    else
        c->drop_batch_graphs();
    return ret;
}

void reset_stats(cahn_stats& st) {
    std::memset(&st, 0, sizeof(st));
    st.failed_system = -1;
}

// ------------------------------------------------------------------ adjoint
// Vector-Jacobian product of nsteps steps started afresh from (phi0, u0,
// v0, p0) (previous levels equal to these, m0 = <phi0, 1>_W).  The forward
// pass stores the state every `K` steps; the reverse pass recomputes each
// segment from its checkpoint, keeping its time levels and mass-correction
// constants, and reverses its steps last to first.  Recomputation repeats
// the forward bit for bit (same kernels, same initial guesses,
// deterministic reductions).  The instance's own state, history and buffer
// arrangement are put back at the end.
struct VjpRun {
    Instance& I;
    cudaStream_t s;
    std::vector<void*> allocs;
    explicit VjpRun(Instance& inst, cudaStream_t st) : I(inst), s(st) {}
    ~VjpRun() {
        cudaStreamSynchronize(s);
        for (void* q : allocs) cudaFree(q);
    }
    double* F() { return dalloc<double>(allocs, I.n); }
};

struct StateRef {   // the seven fields a step starts from
    double* f[7];
};

StateRef live_state(Instance& I) {
    return StateRef{{I.phi, I.phi_prev, I.u, I.u_prev, I.v, I.v_prev, I.p}};
}
void copy_state(const StateRef& dst, const StateRef& src, size_t n, cudaStream_t s) {
    for (int k = 0; k < 7; ++k)
        CAHN_CUDA_TRY(cudaMemcpyAsync(dst.f[k], src.f[k], n * 8, cudaMemcpyDeviceToDevice, s));
}

int run_vjp(Instance& I, cudaStream_t s, const double* phi0, const double* u0, const double* v0,
            const double* p0, int N, int K, const double* jbar, double* out, double* theta,
            cahn_stats& st) {
    const size_t n = I.n, nb = n * sizeof(double);
    const Grid& g = I.g;
    VjpRun R(I, s);
    Driver d;
    d.s = s;
    // the instance's own state, to put back
    double* const arrangement[11] = {I.phi, I.phi_prev, I.phi_new, I.u, I.u_prev, I.u_new,
                                     I.v, I.v_prev, I.v_new, I.p, I.p_new};
    const double m0_saved = I.m0;
    const int phase_saved = I.phase;
    StateRef saved;
    for (double*& f : saved.f) f = R.F();
    copy_state(saved, live_state(I), n, s);
    auto restore = [&]() {
        double** slots[11] = {&I.phi, &I.phi_prev, &I.phi_new, &I.u, &I.u_prev, &I.u_new,
                              &I.v, &I.v_prev, &I.v_new, &I.p, &I.p_new};
        for (int k = 0; k < 11; ++k) *slots[k] = arrangement[k];
        copy_state(live_state(I), saved, n, s);
        I.m0 = m0_saved;
        I.phase = phase_saved;
        I.coef_valid = false;
    };
    try {
        // fresh start: q^{-1} = q^0, m0 = <phi0, 1>_W
        const double* init[7] = {phi0, phi0, u0, u0, v0, v0, p0};
        StateRef live = live_state(I);
        for (int k = 0; k < 7; ++k)
            CAHN_CUDA_TRY(cudaMemcpyAsync(live.f[k], init[k], nb, cudaMemcpyDeviceToDevice, s));
        I.coef_valid = false;
        use_sys(I, CAHN_SYS_PHI);
        launch_wdot<double>(g, I.phi, (const double*)nullptr, I.kw.sd, S_MASS, 1.0, nullptr, s);
        I.kw.read_back(s);
        I.m0 = I.kw.h_scal[S_MASS];

        const int nseg = N > 0 ? (N + K - 1) / K : 0;
        std::vector<StateRef> ck(nseg);
        for (StateRef& c : ck)
            for (double*& f : c.f) f = R.F();
        std::vector<double*> lphi(K + 2), lu(K + 2), lv(K + 2);
        for (int m = 0; m < K + 2; ++m) {
            lphi[m] = R.F();
            lu[m] = R.F();
            lv[m] = R.F();
        }
        double* cseg = dalloc<double>(R.allocs, (size_t)K);
        double* acc3 = dalloc<double>(R.allocs, 4);
        CAHN_CUDA_TRY(cudaMemsetAsync(acc3, 0, 4 * sizeof(double), s));
        cahn_stats fwd;
        reset_stats(fwd);
        auto level = [&](int m) {
            CAHN_CUDA_TRY(cudaMemcpyAsync(lphi[m], I.phi, nb, cudaMemcpyDeviceToDevice, s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(lu[m], I.u, nb, cudaMemcpyDeviceToDevice, s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(lv[m], I.v, nb, cudaMemcpyDeviceToDevice, s));
        };
        // steps k K .. k K + L - 1; with levels, level k K - 1 + m goes to slot m
        auto run_seg = [&](int k, bool levels) -> int {
            const int L = std::min(K, N - k * K);
            if (levels) {
                CAHN_CUDA_TRY(cudaMemcpyAsync(lphi[0], I.phi_prev, nb, cudaMemcpyDeviceToDevice, s));
                CAHN_CUDA_TRY(cudaMemcpyAsync(lu[0], I.u_prev, nb, cudaMemcpyDeviceToDevice, s));
                CAHN_CUDA_TRY(cudaMemcpyAsync(lv[0], I.v_prev, nb, cudaMemcpyDeviceToDevice, s));
                level(1);
            }
            for (int t = 0; t < L; ++t) {
                // graph-mode instances replay their captured step (same results)
                int64_t gl = 0;
                const int code =
                    I.use_graph ? step_graph(I, s, fwd, gl, t + 1 == L) : step_body(I, d, fwd);
                if (I.use_graph) g_launches.fetch_add(gl);
                if (code != CAHN_OK) {
                    st.failed_system = fwd.failed_system;
                    return code;
                }
                if (levels) {
                    launch_adj_save_c(I.d_sys->scal64[CAHN_SYS_PHI], I.m0, I.inv_sumw, cseg + t, s);
                    level(t + 2);
                }
            }
            return CAHN_OK;
        };
        for (int k = 0; k < nseg; ++k) {
            copy_state(ck[k], live_state(I), n, s);
            const int code = run_seg(k, k == nseg - 1);
            if (code != CAHN_OK) {
                restore();
                return code;
            }
        }

        // bars of three consecutive levels (phi, u, v), rolling
        double* B[3][3];
        for (auto& b3 : B)
            for (double*& f : b3) {
                f = R.F();
                CAHN_CUDA_TRY(cudaMemsetAsync(f, 0, nb, s));
            }
        auto bars = [&](int lev) { return B[((lev % 3) + 3) % 3]; };
        CAHN_CUDA_TRY(cudaMemcpyAsync(bars(N)[0], jbar, nb, cudaMemcpyDeviceToDevice, s));
        double *pb = R.F(), *q = R.F(), *xp = R.F(), *bub = R.F(), *bvb = R.F(), *rhs = R.F(),
               *mu = R.F();
        AdjFields A{};
        A.wf = I.wr;
        A.gxb = R.F(); A.gyb = R.F(); A.exb = R.F(); A.eyb = R.F();
        A.phb = R.F(); A.usb = R.F(); A.vsb = R.F(); A.wb = R.F(); A.psit = R.F();
        Op opw = I.op_ch;
        opw.kind = OP_CH13_WADJ;
        opw.a = I.a;
        int predict_phi = 8;
        const double rho = I.P.rho;

        for (int k = nseg - 1; k >= 0; --k) {
            if (k != nseg - 1) {
                copy_state(live_state(I), ck[k], n, s);
                I.coef_valid = false;
                const int code = run_seg(k, true);
                if (code != CAHN_OK) {
                    restore();
                    return code;
                }
            }
            const int s0 = k * K, L = std::min(K, N - s0);
            for (int t = L - 1; t >= 0; --t) {
                const int nn = s0 + t;   // reversing step nn -> nn + 1 (levels t, t+1, t+2)
                double** Bn1 = bars(nn + 1);
                double** Bn = bars(nn);
                double** Bm = bars(nn - 1);
                for (int f = 0; f < 3; ++f) CAHN_CUDA_TRY(cudaMemsetAsync(Bm[f], 0, nb, s));
                A.phi_new = lphi[t + 2];
                A.phi = lphi[t + 1];
                A.phi_prev = lphi[t];
                A.u = lu[t + 1];
                A.u_prev = lu[t];
                A.v = lv[t + 1];
                A.v_prev = lv[t];
                int code;
                // correction and pressure: d_bar = W S (W^-1 p_bar), S the projected Poisson solve
                launch_adj_correct(g, 1.0 / rho, Bn1[1], Bn1[2], pb, s);
                launch_adj_div_w(g, pb, q, s);
                use_sys(I, CAHN_SYS_P);
                launch_wdot<double>(g, q, (const double*)nullptr, I.kw.sd, S_TMP3, I.inv_sumw, nullptr, s);
                launch_sub_scalar<double>(q, n, I.kw.sd.scal + S_TMP3, nullptr, s);
                CAHN_CUDA_TRY(cudaMemsetAsync(xp, 0, nb, s));
                if ((code = solve_p(I, xp, q, d, st))) { restore(); return code; }
                launch_adj_div(g, rho, xp, Bn1[1], Bn1[2], s);
                // predictor: H is symmetric on the interior rows; wall rows are constants
                launch_adj_zero_walls(g, Bn1[1], s);
                launch_adj_zero_walls(g, Bn1[2], s);
                CAHN_CUDA_TRY(cudaMemsetAsync(bub, 0, nb, s));
                CAHN_CUDA_TRY(cudaMemsetAsync(bvb, 0, nb, s));
                if ((code = solve_h(I, CAHN_SYS_U, bub, Bn1[1], d, st))) { restore(); return code; }
                if ((code = solve_h(I, CAHN_SYS_V, bvb, Bn1[2], d, st))) { restore(); return code; }
                // momentum rhs, then mass correction
                launch_adj_mom(g, I.P, A, bub, bvb, Bn[1], Bn[2], s);
                use_sys(I, CAHN_SYS_PHI);
                launch_adj_mass(g, Bn1[0], Bn[0], A.phb, I.kw.sd, rhs, I.inv_sumw, acc3, s);
                // phase-field solve: A_phi^T b_bar = phit_bar  <=>  A* (b_bar / w) = phit_bar / w
                launch_ch_prep(g, I.P, A.phi, A.phi_prev, I.a, nullptr, I.wr, I.d_status, nullptr, s);
                launch_ch13_diag<double>(opw, I.dinv_ch, s);
                launch_invert<double>(n, I.dinv_ch, s);
                CAHN_CUDA_TRY(cudaMemsetAsync(mu, 0, nb, s));
                SolveResult r = gmres_solve<double>(I.kw, opw, mu, rhs, I.dinv_ch, nullptr,
                                                    I.prm.rtol, I.prm.max_iters, predict_phi, d);
                if ((code = record(I, CAHN_SYS_PHI, r, st))) { restore(); return code; }
                launch_adj_mul_w(g, mu, s);
                // phase-field rhs and coefficient
                launch_adj_ch(g, I.P, A, mu, I.a, cseg + t, Bn[0], Bm[0], Bn[1], Bm[1], Bn[2],
                              Bm[2], I.kw.sd, acc3, s);
            }
        }
        launch_adj_final(g, bars(0)[0], bars(-1)[0], acc3, out, s);
        double h3[4];
        CAHN_CUDA_TRY(cudaMemcpyAsync(h3, acc3, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CAHN_CUDA_TRY(cudaStreamSynchronize(s));
        theta[0] = h3[0];
        theta[1] = h3[1];
        st.steps = N;
        restore();
    } catch (...) {
        cudaGetLastError();
        try {
            restore();
        } catch (...) {
        }
        throw;
    }
    return CAHN_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int cahn_abi_version(void) { return CAHN_ABI_VERSION; }

const char* cahn_last_error(const cahn_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

int64_t cahn_last_launch_count(const cahn_ctx* ctx) { return ctx ? ctx->launches : 0; }

int cahn_init(cahn_ctx** out, int32_t batch, const cahn_params* params, double* const* phi,
              double* const* u, double* const* v, double* const* p, void* stream) {
    if (!out) return fail(nullptr, CAHN_ERR_ARG, "ctx pointer is NULL");
    *out = nullptr;
    if (batch < 1 || batch > 1024) return fail(nullptr, CAHN_ERR_ARG, "batch must be in 1..1024");
    if (!params || !phi || !u || !v || !p) return fail(nullptr, CAHN_ERR_ARG, "NULL argument");
    for (int k = 0; k < batch; ++k) {
        std::string e = check_params(params[k]);
        if (!e.empty()) return fail(nullptr, CAHN_ERR_ARG, "instance " + std::to_string(k) + ": " + e);
        if (!phi[k] || !u[k] || !v[k] || !p[k])
            return fail(nullptr, CAHN_ERR_ARG, "instance " + std::to_string(k) + ": NULL field");
    }
    cahn_ctx* c = new cahn_ctx();
    c->s = static_cast<cudaStream_t>(stream);
    try {
        for (int k = 0; k < batch; ++k) {
            Instance* I = new Instance();
            c->inst.push_back(I);
            setup_instance(*I, params[k], phi[k], u[k], v[k], p[k], c->s, batch > 1);
        }
        if (batch > 1) batch_coop(c->inst);
        bool all_graph = batch > 1;
        for (Instance* I : c->inst) all_graph = all_graph && I->use_graph;
        if (all_graph) {
            c->batch_graph = true;
            CAHN_CUDA_TRY(cudaStreamCreateWithFlags(&c->bcap, cudaStreamNonBlocking));
            CAHN_CUDA_TRY(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
            CAHN_CUDA_TRY(cudaEventCreateWithFlags(&c->cfork, cudaEventDisableTiming));
            for (int k = 0; k < batch; ++k) {
                cudaEvent_t e;
                CAHN_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                c->join.push_back(e);
            }
        }
        CAHN_CUDA_TRY(cudaStreamSynchronize(c->s));
    } catch (const std::bad_alloc&) {
        delete c;
        return fail(nullptr, CAHN_ERR_NOMEM, "device allocation failed");
    } catch (const std::exception& e) {
        delete c;
        return fail(nullptr, CAHN_ERR_CUDA, e.what());
    }
    *out = c;
    return CAHN_OK;
}

int cahn_step(cahn_ctx* ctx, int32_t nsteps, cahn_stats* stats) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, CAHN_ERR_ARG, "nsteps < 0");
    for (size_t k = 0; k < ctx->inst.size(); ++k)
        if (ctx->inst[k]->nut && !ctx->inst[k]->nut_ready)
            return fail(ctx, CAHN_ERR_ARG, "instance " + std::to_string(k) +
                                               ": nutrient on but no c registered (cahn_attach_nutrient)");
    Driver d;
    d.s = ctx->s;
    int ret = CAHN_OK;
    const int64_t l0 = g_launches.load();
    struct Tally {
        cahn_ctx* c;
        int64_t l0;
        ~Tally() { c->launches = g_launches.load() - l0; }
    } tally{ctx, l0};
    try {
        if (ctx->batch_graph) {
            const size_t nb = ctx->inst.size();
            std::vector<cahn_stats> sts(nb);
            for (cahn_stats& st : sts) reset_stats(st);
            for (Instance* I : ctx->inst) copy_in(*I, d.s);
            int64_t glaunch = 0;
            int failed = -1;
            for (int t = 0; t < nsteps && ret == CAHN_OK; ++t)
                ret = step_batch(ctx, sts.data(), glaunch, failed, t + 1 == nsteps);
            g_launches.fetch_add(glaunch);
            for (Instance* I : ctx->inst) copy_out(*I, d.s);
            CAHN_CUDA_TRY(cudaStreamSynchronize(d.s));
            for (size_t k = 0; k < nb; ++k) {
                if (sts[k].status == 0 && (int)k != failed) sts[k].status = CAHN_OK;
                if (stats) stats[k] = sts[k];
            }
            if (ret != CAHN_OK)
                fail(ctx, ret, "instance " + std::to_string(failed) + ": system " +
                                   sys_name(sts[failed].failed_system < 0 ? 0 : sts[failed].failed_system) +
                                   " failed (code " + std::to_string(ret) + ")");
            return ret;
        }
        for (size_t k = 0; k < ctx->inst.size(); ++k) {
            Instance& I = *ctx->inst[k];
            cahn_stats st;
            reset_stats(st);
            copy_in(I, d.s);
            int code = CAHN_OK;
            int64_t glaunch = 0;
            for (int t = 0; t < nsteps && code == CAHN_OK; ++t)
                code = I.use_graph ? step_graph(I, d.s, st, glaunch, t + 1 == nsteps)
                                   : step_body(I, d, st);
            if (I.use_graph) g_launches.fetch_add(glaunch);
            copy_out(I, d.s);
            CAHN_CUDA_TRY(cudaStreamSynchronize(d.s));
            st.status = code;
            if (stats) stats[k] = st;
            if (code != CAHN_OK && ret == CAHN_OK) {
                ret = code;
                fail(ctx, code, "instance " + std::to_string(k) + ": system " +
                                    sys_name(st.failed_system < 0 ? 0 : st.failed_system) +
                                    " failed (code " + std::to_string(code) + ")");
            }
        }
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    return ret;
}

int cahn_step_host(cahn_ctx* ctx, int32_t nsteps, double* const* phi_h, double* const* u_h,
                   double* const* v_h, double* const* p_h, cahn_stats* stats) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (!phi_h || !u_h || !v_h || !p_h) return fail(ctx, CAHN_ERR_ARG, "NULL argument");
    try {
        for (Instance* I : ctx->inst) (void)I;
        for (size_t k = 0; k < ctx->inst.size(); ++k) {
            Instance& I = *ctx->inst[k];
            if (!phi_h[k] || !u_h[k] || !v_h[k] || !p_h[k])
                return fail(ctx, CAHN_ERR_ARG, "NULL host field");
            const size_t b = I.n * sizeof(double);
            CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi_c, phi_h[k], b, cudaMemcpyHostToDevice, ctx->s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(I.u_c, u_h[k], b, cudaMemcpyHostToDevice, ctx->s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(I.v_c, v_h[k], b, cudaMemcpyHostToDevice, ctx->s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(I.p_c, p_h[k], b, cudaMemcpyHostToDevice, ctx->s));
        }
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    int ret = cahn_step(ctx, nsteps, stats);
    try {
        for (size_t k = 0; k < ctx->inst.size(); ++k) {
            Instance& I = *ctx->inst[k];
            const size_t b = I.n * sizeof(double);
            CAHN_CUDA_TRY(cudaMemcpyAsync(phi_h[k], I.phi_c, b, cudaMemcpyDeviceToHost, ctx->s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(u_h[k], I.u_c, b, cudaMemcpyDeviceToHost, ctx->s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(v_h[k], I.v_c, b, cudaMemcpyDeviceToHost, ctx->s));
            CAHN_CUDA_TRY(cudaMemcpyAsync(p_h[k], I.p_c, b, cudaMemcpyDeviceToHost, ctx->s));
        }
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    return ret;
}

int cahn_solve(cahn_ctx* ctx, int32_t instance, int32_t system, const double* rhs, double* x,
               cahn_stats* stats) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (system < CAHN_SYS_PHI || system > CAHN_SYS_UV) return fail(ctx, CAHN_ERR_ARG, "bad system");
    if (!rhs || !x) return fail(ctx, CAHN_ERR_ARG, "NULL rhs or x");
    Instance& I = *ctx->inst[instance];
    if (system == CAHN_SYS_C && !I.nut)
        return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_C needs an instance with the nutrient on");
    if (system == CAHN_SYS_UV && !I.impl_mom)
        return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_UV needs momentum = CAHN_MOM_IMPLICIT");
    Driver d;
    d.s = ctx->s;
    cahn_stats st;
    reset_stats(st);
    int code = CAHN_OK;
    const int64_t l0 = g_launches.load();
    struct Tally {
        cahn_ctx* c;
        int64_t l0;
        ~Tally() { c->launches = g_launches.load() - l0; }
    } tally{ctx, l0};
    try {
        copy_in(I, d.s);
        if (system == CAHN_SYS_PHI) {
            CAHN_CUDA_TRY(cudaMemsetAsync(I.d_status, 0, sizeof(int), d.s));
            coefficient(I, d.s);
            if (domain_status(I, d.s) & CTL_DOMAIN) {
                code = CAHN_ERR_DOMAIN;
                st.failed_system = CAHN_SYS_PHI;
            } else {
                code = solve_phi(I, x, rhs, d, st);
            }
        } else if (system == CAHN_SYS_P) {
            CAHN_CUDA_TRY(cudaMemcpyAsync(I.d, rhs, I.n * 8, cudaMemcpyDeviceToDevice, d.s));
            launch_wdot<double>(I.g, I.d, (const double*)nullptr, I.kw.sd, S_TMP3, I.inv_sumw, nullptr, d.s);
            launch_sub_scalar<double>(I.d, I.n, I.kw.sd.scal + S_TMP3, nullptr, d.s);
            code = solve_p(I, x, I.d, d, st);
        } else if (system == CAHN_SYS_C) {
            nut_coefficients(I, d.s);
            if (I.N.dtop) launch_nut_top(I.g, x, rhs, I.prm.dt, d.s);
            code = solve_c(I, x, rhs, d, st);
        } else if (system == CAHN_SYS_UV) {
            uv_coefficient(I, d.s);
            code = solve_uv(I, x, rhs, d, st);
        } else {
            code = solve_h(I, system, x, rhs, d, st);
        }
        CAHN_CUDA_TRY(cudaStreamSynchronize(d.s));
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    st.status = code;
    if (stats) *stats = st;
    if (code != CAHN_OK) fail(ctx, code, std::string("solve of ") + sys_name(system) + " failed");
    return code;
}

int cahn_apply(cahn_ctx* ctx, int32_t instance, int32_t system, const double* x, double* y) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (system < CAHN_SYS_PHI || system > CAHN_SYS_UV) return fail(ctx, CAHN_ERR_ARG, "bad system");
    if (!x || !y) return fail(ctx, CAHN_ERR_ARG, "NULL x or y");
    Instance& I = *ctx->inst[instance];
    if (system == CAHN_SYS_C && !I.nut)
        return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_C needs an instance with the nutrient on");
    if (system == CAHN_SYS_UV && !I.impl_mom)
        return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_UV needs momentum = CAHN_MOM_IMPLICIT");
    const int64_t l0 = g_launches.load();
    try {
        const Op* op = &I.op_p;
        if (system == CAHN_SYS_PHI) {
            if (!I.coef_valid) coefficient(I, ctx->s);
            op = &I.op_ch;
        } else if (system == CAHN_SYS_C) {
            nut_coefficients(I, ctx->s);
            op = &I.op_c;
        } else if (system == CAHN_SYS_UV) {
            uv_coefficient(I, ctx->s);
            op = &I.op_uv;
        } else if (system != CAHN_SYS_P) {
            op = &I.op_h;
        }
        launch_op<double>(*op, EPI_APPLY, x, nullptr, y, I.kw.sd, nullptr, 0.0, ctx->s);
        CAHN_CUDA_TRY(cudaGetLastError());
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    ctx->launches = g_launches.load() - l0;
    return CAHN_OK;
}

int cahn_apply32(cahn_ctx* ctx, int32_t instance, int32_t system, const float* x, float* y) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (system < CAHN_SYS_PHI || system > CAHN_SYS_UV) return fail(ctx, CAHN_ERR_ARG, "bad system");
    if (!x || !y) return fail(ctx, CAHN_ERR_ARG, "NULL x or y");
    Instance& I = *ctx->inst[instance];
    if (!I.mixed) return fail(ctx, CAHN_ERR_ARG, "cahn_apply32 needs a CAHN_MIXED instance");
    if (system == CAHN_SYS_C && !I.nut)
        return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_C needs an instance with the nutrient on");
    const int64_t l0 = g_launches.load();
    try {
        const Op* op = &I.op32_p;
        if (system == CAHN_SYS_PHI) {
            if (!I.coef_valid) coefficient(I, ctx->s);
            op = &I.op32_ch;
        } else if (system == CAHN_SYS_C) {
            nut_coefficients(I, ctx->s);
            op = &I.op32_c;
        } else if (system == CAHN_SYS_UV) {
            if (!I.impl_mom)
                return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_UV needs momentum = CAHN_MOM_IMPLICIT");
            uv_coefficient(I, ctx->s);
            op = &I.op32_uv;
        } else if (system != CAHN_SYS_P) {
            op = &I.op32_h;
        }
        launch_op<float>(*op, EPI_APPLY, x, nullptr, y, I.kw32.sd, nullptr, 0.0, ctx->s);
        CAHN_CUDA_TRY(cudaGetLastError());
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    ctx->launches = g_launches.load() - l0;
    return CAHN_OK;
}

int cahn_smooth32(cahn_ctx* ctx, int32_t instance, int32_t system, int32_t k, const float* x,
                  const float* b, float* d, float* y) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (system < CAHN_SYS_PHI || system > CAHN_SYS_C) return fail(ctx, CAHN_ERR_ARG, "bad system");
    if (k < 0 || k >= 16) return fail(ctx, CAHN_ERR_ARG, "k outside [0, 16)");
    if (!x || !b || !d || !y) return fail(ctx, CAHN_ERR_ARG, "NULL x, b, d or y");
    if (x == y || d == y || d == x || d == b)
        return fail(ctx, CAHN_ERR_ARG, "y and d must not alias each other, x or b");
    Instance& I = *ctx->inst[instance];
    if (!I.mixed) return fail(ctx, CAHN_ERR_ARG, "cahn_smooth32 needs a CAHN_MIXED instance");
    if (!I.use_mg) return fail(ctx, CAHN_ERR_ARG, "cahn_smooth32 needs the multigrid preconditioner");
    if (system == CAHN_SYS_C && !I.nut)
        return fail(ctx, CAHN_ERR_ARG, "CAHN_SYS_C needs an instance with the nutrient on");
    const int64_t l0 = g_launches.load();
    try {
        Multigrid<float>* mg = &I.mg32_p;
        if (system == CAHN_SYS_PHI) {
            if (!I.coef_valid) coefficient(I, ctx->s);
            mg = &I.mg32_ch;
        } else if (system == CAHN_SYS_C) {
            nut_coefficients(I, ctx->s);
            mg = &I.mg32_c;
        } else if (system != CAHN_SYS_P) {
            mg = &I.mg32_h;
        }
        mg->fine_step(x, b, d, y, k, ctx->s);
        CAHN_CUDA_TRY(cudaGetLastError());
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    ctx->launches = g_launches.load() - l0;
    return CAHN_OK;
}

int cahn_mg_down32(cahn_ctx* ctx, int32_t instance, int32_t system, const float* b, float* x) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (system != CAHN_SYS_U && system != CAHN_SYS_V && system != CAHN_SYS_P)
        return fail(ctx, CAHN_ERR_ARG, "cahn_mg_down32: CAHN_SYS_U, CAHN_SYS_V or CAHN_SYS_P");
    if (!x || !b) return fail(ctx, CAHN_ERR_ARG, "NULL b or x");
    if ((const float*)x == b) return fail(ctx, CAHN_ERR_ARG, "x must not alias b");
    Instance& I = *ctx->inst[instance];
    if (!I.mixed) return fail(ctx, CAHN_ERR_ARG, "cahn_mg_down32 needs a CAHN_MIXED instance");
    if (!I.use_mg || I.prm.precond != CAHN_PC_MG)
        return fail(ctx, CAHN_ERR_ARG, "cahn_mg_down32 needs the multigrid preconditioner");
    Multigrid<float>& mg = system == CAHN_SYS_P ? I.mg32_p : I.mg32_h;
    if (mg.lv.size() < 2) return fail(ctx, CAHN_ERR_ARG, "cahn_mg_down32: one-level hierarchy");
    const int64_t l0 = g_launches.load();
    try {
        mg.down_pass(b, x, ctx->s);
        CAHN_CUDA_TRY(cudaGetLastError());
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    ctx->launches = g_launches.load() - l0;
    return CAHN_OK;
}

int cahn_lap5_coarse_inverse(int32_t nx, int32_t ny, int32_t walls, double c0, double cx,
                             double cy, double* P) {
    if (nx < 2 || ny < 1) return fail(nullptr, CAHN_ERR_ARG, "cahn_lap5_coarse_inverse: nx >= 2, ny >= 1");
    if ((int64_t)nx * (ny + 1) > 4096) return fail(nullptr, CAHN_ERR_ARG, "cahn_lap5_coarse_inverse: n > 4096");
    if (walls != 0 && walls != 1) return fail(nullptr, CAHN_ERR_ARG, "cahn_lap5_coarse_inverse: walls 0 or 1");
    if (!(c0 >= 0.0 && cx >= 0.0 && cy >= 0.0) || !std::isfinite(c0) || !std::isfinite(cx) ||
        !std::isfinite(cy) || !(cx + cy > 0.0))
        return fail(nullptr, CAHN_ERR_ARG, "cahn_lap5_coarse_inverse: bad coefficients");
    if (!P) return fail(nullptr, CAHN_ERR_ARG, "P is NULL");
    Op o{};
    o.g = Grid{nx, ny, 1.0, 1.0};
    o.kind = walls ? OP_LAP5_DIRICHLET : OP_LAP5_NEUMANN;
    o.c0 = c0;
    o.cx = cx;
    o.cy = cy;
    std::vector<double> m;
    if (!dense_solve_matrix(o, walls ? 1 : 0, m))
        return fail(nullptr, CAHN_ERR_ARG, "cahn_lap5_coarse_inverse: singular system");
    std::copy(m.begin(), m.end(), P);
    return CAHN_OK;
}

int cahn_vjp(cahn_ctx* ctx, int32_t instance, const double* phi0, const double* u0,
             const double* v0, const double* p0, int32_t nsteps, int32_t checkpoint,
             const double* phiN_bar, double* phi0_bar, double* theta_bar, cahn_stats* stats) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (nsteps < 0) return fail(ctx, CAHN_ERR_ARG, "nsteps < 0");
    if (checkpoint < 1) return fail(ctx, CAHN_ERR_ARG, "checkpoint must be >= 1");
    if (!phi0 || !u0 || !v0 || !p0 || !phiN_bar || !phi0_bar || !theta_bar)
        return fail(ctx, CAHN_ERR_ARG, "NULL argument");
    Instance& I = *ctx->inst[instance];
    if (I.nut) return fail(ctx, CAHN_ERR_ARG, "the adjoint does not cover the nutrient");
    if (I.impl_mom)
        return fail(ctx, CAHN_ERR_ARG, "the adjoint covers the eta_bar split momentum only");
    cahn_stats st;
    reset_stats(st);
    const int64_t l0 = g_launches.load();
    struct Tally {
        cahn_ctx* c;
        int64_t l0;
        ~Tally() { c->launches = g_launches.load() - l0; }
    } tally{ctx, l0};
    int code;
    try {
        const int K = std::max(1, std::min((int)checkpoint, (int)nsteps));
        code = run_vjp(I, ctx->s, phi0, u0, v0, p0, nsteps, K, phiN_bar, phi0_bar, theta_bar, st);
    } catch (const std::bad_alloc&) {
        return fail(ctx, CAHN_ERR_NOMEM, "device allocation failed");
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    st.status = code;
    if (stats) *stats = st;
    if (code != CAHN_OK)
        fail(ctx, code, std::string("adjoint: system ") +
                            sys_name(st.failed_system < 0 ? 0 : st.failed_system) + " failed");
    return code;
}

int cahn_get_history(cahn_ctx* ctx, int32_t instance, double* phi_prev, double* u_prev,
                     double* v_prev, double* m0) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (!phi_prev || !u_prev || !v_prev || !m0) return fail(ctx, CAHN_ERR_ARG, "NULL argument");
    Instance& I = *ctx->inst[instance];
    const size_t b = I.n * sizeof(double);
    try {
        CAHN_CUDA_TRY(cudaMemcpyAsync(phi_prev, I.phi_prev, b, cudaMemcpyDeviceToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(u_prev, I.u_prev, b, cudaMemcpyDeviceToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(v_prev, I.v_prev, b, cudaMemcpyDeviceToDevice, ctx->s));
        double m = I.m0;
        if (I.nut)
            CAHN_CUDA_TRY(cudaMemcpyAsync(&m, I.d_mass, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
        *m0 = m;
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    return CAHN_OK;
}

int cahn_set_history(cahn_ctx* ctx, int32_t instance, const double* phi_prev, const double* u_prev,
                     const double* v_prev, double m0) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (!phi_prev || !u_prev || !v_prev) return fail(ctx, CAHN_ERR_ARG, "NULL argument");
    if (!std::isfinite(m0)) return fail(ctx, CAHN_ERR_ARG, "m0 is not finite");
    Instance& I = *ctx->inst[instance];
    const size_t b = I.n * sizeof(double);
    try {
        // a captured step holds m0 as a kernel argument: recapture after the change
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
        for (GraphSlot& G : I.slot) {
            if (G.exec) CAHN_CUDA_TRY(cudaGraphExecDestroy(G.exec));
            G.exec = nullptr;
        }
        ctx->drop_batch_graphs();
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.phi_prev, phi_prev, b, cudaMemcpyDeviceToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.u_prev, u_prev, b, cudaMemcpyDeviceToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.v_prev, v_prev, b, cudaMemcpyDeviceToDevice, ctx->s));
        if (I.nut)
            CAHN_CUDA_TRY(cudaMemcpyAsync(I.d_mass, &m0, sizeof(double), cudaMemcpyHostToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    I.m0 = m0;
    I.coef_valid = false;
    return CAHN_OK;
}

int cahn_attach_nutrient(cahn_ctx* ctx, int32_t instance, double* c, const double* c_prev) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (!c) return fail(ctx, CAHN_ERR_ARG, "c is NULL");
    Instance& I = *ctx->inst[instance];
    if (!I.nut) return fail(ctx, CAHN_ERR_ARG, "the instance was created with nutrient = 0");
    const size_t b = I.n * sizeof(double);
    try {
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
        for (GraphSlot& G : I.slot) {
            if (G.exec) CAHN_CUDA_TRY(cudaGraphExecDestroy(G.exec));
            G.exec = nullptr;
        }
        ctx->drop_batch_graphs();
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.c, c, b, cudaMemcpyDeviceToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(I.c_prev, c_prev ? c_prev : c, b, cudaMemcpyDeviceToDevice, ctx->s));
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    I.c_c = c;
    I.nut_ready = true;
    return CAHN_OK;
}

int cahn_get_nutrient_history(cahn_ctx* ctx, int32_t instance, double* c_prev) {
    if (!ctx) return fail(nullptr, CAHN_ERR_ARG, "ctx is NULL");
    if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, CAHN_ERR_ARG, "bad instance");
    if (!c_prev) return fail(ctx, CAHN_ERR_ARG, "c_prev is NULL");
    Instance& I = *ctx->inst[instance];
    if (!I.nut_ready) return fail(ctx, CAHN_ERR_ARG, "no nutrient registered");
    try {
        CAHN_CUDA_TRY(cudaMemcpyAsync(c_prev, I.c_prev, I.n * sizeof(double), cudaMemcpyDeviceToDevice,
                                      ctx->s));
        CAHN_CUDA_TRY(cudaStreamSynchronize(ctx->s));
    } catch (const std::exception& e) {
        return fail(ctx, CAHN_ERR_CUDA, e.what());
    }
    return CAHN_OK;
}

int cahn_tile_height(const cahn_ctx* ctx, int32_t instance, int32_t system, int32_t level) {
    if (!ctx || instance < 0 || instance >= (int)ctx->inst.size()) return -1;
    if (system < CAHN_SYS_PHI || system > CAHN_SYS_C || level < 0) return -1;
    const Instance& I = *ctx->inst[instance];
    if (system == CAHN_SYS_C) {
        if (!I.nut) return -1;
        if (I.use_mg) {
            if (I.mixed) return level < (int)I.mg32_c.lv.size() ? I.mg32_c.lv[level].op.ty : -1;
            return level < (int)I.mg_c.lv.size() ? I.mg_c.lv[level].op.ty : -1;
        }
        if (level > 0) return -1;
        return I.mixed ? I.op32_c.ty : I.op_c.ty;
    }
    const int k = system == CAHN_SYS_PHI ? 0 : (system == CAHN_SYS_P ? 2 : 1);
    if (I.use_mg) {
        if (I.mixed) {
            const Multigrid<float>* m[3] = {&I.mg32_ch, &I.mg32_h, &I.mg32_p};
            return level < (int)m[k]->lv.size() ? m[k]->lv[level].op.ty : -1;
        }
        const Multigrid<double>* m[3] = {&I.mg_ch, &I.mg_h, &I.mg_p};
        return level < (int)m[k]->lv.size() ? m[k]->lv[level].op.ty : -1;
    }
    if (level > 0) return -1;
    const Op* o[3] = {I.mixed ? &I.op32_ch : &I.op_ch, I.mixed ? &I.op32_h : &I.op_h,
                      I.mixed ? &I.op32_p : &I.op_p};
    return o[k]->ty;
}

int cahn_free(cahn_ctx* ctx) {
    if (!ctx) return CAHN_OK;
    cudaStreamSynchronize(ctx->s);
    delete ctx;
    return CAHN_OK;
}

}  // extern "C"
