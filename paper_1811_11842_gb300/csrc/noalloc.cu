// Allocation-free pressure solve.
//
// Some callers cannot allocate device memory at the time they need a solve:
// a host application whose memory manager has already reserved the GPU's
// memory for its own pool, code running in a latency-critical loop where
// cudaMalloc / cudaFree would stall (they can synchronise the device), or
// a plugin that may only use memory set aside at load time.  This entry
// point serves them: it solves the pressure system of cahn_solve
// (CAHN_SYS_P, Jacobi-preconditioned CG) with every intermediate held in
// one file-scope device array, so it calls no allocating routine.  The
// caller passes the right-hand side and the solution array.
//
// The array is a fixed 3.3 MB per GPU that loads the library, held until
// the process exits.  It bounds the grid to nx * (ny + 1) <= 66,560 nodes
// (256 x 256 intervals fit).  All calls share it, and it keeps the last
// call's contents, so calls that overlap on the GPU (two streams, two
// threads) race and must be serialised by the caller.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/cahn.h"
#include "solver.h"

namespace {

using namespace cahn;

constexpr size_t NA_MAX_NODES = 66560;
constexpr int NA_MAX_BLOCKS = 4096;
constexpr int NA_VECS = 6;   // r, z, p, q, projected rhs, Jacobi scaling
constexpr size_t NA_SCAL_OFF = NA_VECS * NA_MAX_NODES;
constexpr size_t NA_CTL_OFF = NA_SCAL_OFF + S_COUNT;
constexpr size_t NA_PART_OFF = NA_CTL_OFF + 8;                  // Ctl fits in 8 doubles
constexpr size_t NA_CNT_OFF = NA_PART_OFF + 2 * (size_t)NA_MAX_BLOCKS;
constexpr size_t NA_TOTAL = NA_CNT_OFF + 8;
static_assert(sizeof(Ctl) <= 8 * sizeof(double), "Ctl slot too small");

// The scratch: in host code this name is only a stand-in for the device
// address, which comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};
Ctl g_na_hctl[NA_MAX_DEVICES];
double g_na_hscal[NA_MAX_DEVICES][S_COUNT];
thread_local std::string g_na_error;

int na_fail(int code, const std::string& msg) {
    g_na_error = msg;
    return code;
}

// Once per device, with that device current: look up the scratch address
// and clear the reduction counter.
int na_setup(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        double* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return na_fail(CAHN_ERR_CUDA, cudaGetErrorString(e));
        e = cudaMemset(p + NA_CNT_OFF, 0, 8 * sizeof(double));
        if (e != cudaSuccess) return na_fail(CAHN_ERR_CUDA, cudaGetErrorString(e));
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return na_fail(CAHN_ERR_CUDA, cudaGetErrorString(e));
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return CAHN_OK;
}

}  // namespace

extern "C" {

const char* cahn_noalloc_last_error(void) { return g_na_error.c_str(); }

int cahn_solve_p_noalloc(int32_t nx, int32_t ny, double lx, double ly, double rtol,
                         int32_t max_iters, const double* rhs, double* x, void* stream,
                         cahn_stats* stats) {
    if (nx < 4 || nx % 2 || ny < 4 || ny % 2) return na_fail(CAHN_ERR_ARG, "nx, ny must be even and >= 4");
    if (!(lx > 0) || !(ly > 0)) return na_fail(CAHN_ERR_ARG, "lx, ly must be > 0");
    if (!(rtol > 0) || !(rtol < 1)) return na_fail(CAHN_ERR_ARG, "rtol must be in (0,1)");
    if (max_iters < 1) return na_fail(CAHN_ERR_ARG, "max_iters must be >= 1");
    if (!rhs || !x) return na_fail(CAHN_ERR_ARG, "NULL rhs or x");
    const size_t n = (size_t)nx * (ny + 1);
    if (n > NA_MAX_NODES)
        return na_fail(CAHN_ERR_ARG, "grid too large for the allocation-free solve: nx*(ny+1) = " +
                                         std::to_string(n) + " > 66560 nodes");
    const int blocks = std::max(tile_blocks(nx, ny), vec_blocks(n));
    if (blocks > NA_MAX_BLOCKS) return na_fail(CAHN_ERR_ARG, "grid shape needs too many blocks");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(CAHN_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(CAHN_ERR_ARG, "device index too large");
    double* base = nullptr;
    int code = na_setup(dev, &base);
    if (code != CAHN_OK) return code;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Grid g{nx, ny, lx / nx, ly / ny};
    const double gx = 1.0 / (g.hx * g.hx), gy = 1.0 / (g.hy * g.hy);
    Op op{};
    op.g = g;
    op.kind = OP_LAP5_NEUMANN;
    op.c0 = 0.0;
    op.cx = gx;
    op.cy = gy;

    KrylovWs<double> W;   // views into the scratch; W.alloc() is never called
    W.g = g;
    W.n = n;
    W.r = base + 0 * NA_MAX_NODES;
    W.z = base + 1 * NA_MAX_NODES;
    W.p = base + 2 * NA_MAX_NODES;
    W.q = base + 3 * NA_MAX_NODES;
    double* d = base + 4 * NA_MAX_NODES;
    double* dinv = base + 5 * NA_MAX_NODES;
    W.sd.scal = base + NA_SCAL_OFF;
    W.sd.ctl = reinterpret_cast<Ctl*>(base + NA_CTL_OFF);
    W.sd.red.partials = base + NA_PART_OFF;
    W.sd.red.counter = reinterpret_cast<unsigned*>(base + NA_CNT_OFF);
    W.sd.red.stride = blocks;
    W.h_ctl = &g_na_hctl[dev];
    W.h_scal = g_na_hscal[dev];

    const double sumw = (double)nx * ny;   // interior rows + two half-weight wall rows
    int predict = 8;
    Driver drv;
    drv.s = s;
    SolveResult res;
    try {
        // the counter must start at zero; everything else is written before it is read
        CAHN_CUDA_TRY(cudaMemsetAsync(W.sd.red.counter, 0, sizeof(unsigned), s));
        CAHN_CUDA_TRY(cudaMemcpyAsync(d, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        launch_wdot<double>(g, d, (const double*)nullptr, W.sd, S_TMP3, 1.0 / sumw, nullptr, s);
        launch_sub_scalar<double>(d, n, W.sd.scal + S_TMP3, nullptr, s);
        launch_fill(dinv, 1.0 / (2.0 * gx + 2.0 * gy), n, s);
        res = cg_solve<double>(W, op, x, d, dinv, nullptr, rtol, max_iters, true, 1.0 / sumw,
                               predict, drv);
        CAHN_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (const std::exception& ex) {
        return na_fail(CAHN_ERR_CUDA, ex.what());
    }
    code = CAHN_OK;
    if (res.status & CTL_NAN)
        code = CAHN_ERR_NAN;
    else if (res.status & CTL_NOT_CONVERGED)
        code = CAHN_ERR_NOT_CONVERGED;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->iters[CAHN_SYS_P] = res.it;
        stats->resid[CAHN_SYS_P] = res.rel_res;
        stats->failed_system = code == CAHN_OK ? -1 : CAHN_SYS_P;
        stats->status = code;
    }
    if (code != CAHN_OK) na_fail(code, "pressure solve failed");
    return code;
}

}  // extern "C"
