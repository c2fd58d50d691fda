// Shared internals of the CUDA library: grid descriptors, launch helpers and
// the deterministic two-stage block reduction used by every fused dot.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace cahn {

// One structured grid level: nx periodic columns, ny+1 rows (walls 0, ny).
struct Grid {
    int nx, ny;
    double hx, hy;
    __host__ __device__ size_t n() const { return (size_t)nx * (ny + 1); }
};

// Slots of the per-solve device scalar block (doubles).  Kernels that end
// in a reduction write derived scalars (alpha, beta, ...) from their last
// block, so the next kernel reads them without a host round trip.
enum ScalarSlot {
    S_BN = 0,      // ||b||_W
    S_RR,          // <r,r>_W (latest)
    S_RZ,          // <r,z>_W
    S_PQ,          // <p,Ap>_W
    S_ALPHA,
    S_BETA,
    S_TOL2,        // (rtol ||b||)^2
    S_MASS,        // generic reduction result
    S_TMP0, S_TMP1, S_TMP2, S_TMP3,
    S_OMEGA, S_RHO, S_ALPHA2, S_RES0,
    S_IRLAST,      // refinement: residual norm of the previous sweep
    S_COUNT
};

// Per-solve control block in device memory.
struct Ctl {
    int done;       // loop finished (converged, failed or capped)
    int it;         // iterations of this solve
    int status;     // 0 ok, else CTL_* bits
    int cycle_end;  // GMRES: the current restart cycle is over
    int k;          // GMRES: current Arnoldi column
    int maxit;
    int cycles;     // GMRES restart cycles started; refinement: stalled sweeps
    int idle;       // GMRES: no restart cycle in progress
    int total;      // iterations summed over every solve since the last clear
};
enum { CTL_NOT_CONVERGED = 1, CTL_NAN = 2, CTL_DOMAIN = 4 };

constexpr int RED_THREADS = 256;
constexpr int VEC_MAX_BLOCKS = 1216;    // 152 SMs x 8 resident blocks of 256
constexpr int MAX_MULTI = 66;           // GMRES(64) + 2 reduction slots
constexpr int TILE_X = 32, TILE_Y = 32; // stencil output tile per block (32 x 8 threads)

// Workspace of the two-stage reductions: per-block partial sums and a
// completion counter.  One per instance (its kernels are stream-ordered).
struct RedWs {
    double* partials;     // [MAX_MULTI][stride]
    unsigned* counter;    // 1 counter, reset to 0 by the last block
    int stride;           // >= blocks of any reducing launch on this instance
};

inline int vec_blocks(size_t items, int threads = RED_THREADS) {
    size_t b = (items + threads - 1) / threads;
    if (b > (size_t)VEC_MAX_BLOCKS) b = VEC_MAX_BLOCKS;
    if (b < 1) b = 1;
    return (int)b;
}
inline dim3 tile_grid(int nx, int ny, int ty = TILE_Y) {
    return dim3((unsigned)((nx + TILE_X - 1) / TILE_X), (unsigned)((ny + 1 + ty - 1) / ty));
}
inline int tile_blocks(int nx, int ny) {
    dim3 g = tile_grid(nx, ny);
    return (int)(g.x * g.y);
}

// ---------------------------------------------------------------- device
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (1-D or 2-D blocks, whole warps); result valid in every
// thread.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = t & 31, wid = t >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = (t < nw) ? sh[t] : 0.0;
    if (wid == 0) r = warp_sum(r);
    if (t == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int flat_tid() { return threadIdx.x + blockDim.x * threadIdx.y; }
__device__ __forceinline__ int flat_bid() { return blockIdx.x + gridDim.x * blockIdx.y; }
__device__ __forceinline__ int nblocks() { return gridDim.x * gridDim.y; }

// Publish this block's partial (thread 0 of the block).  The final sum is
// taken in block order by the last block to finish (`last_block` +
// `final_sum`), so results are deterministic.
__device__ __forceinline__ void publish_partial(RedWs ws, int slot, double part) {
    if (flat_tid() == 0) ws.partials[(size_t)slot * ws.stride + flat_bid()] = part;
}

__device__ __forceinline__ bool last_block(RedWs ws) {
    __shared__ unsigned s_last;
    __threadfence();
    __syncthreads();
    if (flat_tid() == 0) {
        unsigned t = atomicAdd(ws.counter, 1u);
        s_last = (t == (unsigned)nblocks() - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

__device__ __forceinline__ double final_sum(RedWs ws, int slot, double* sh) {
    double v = 0.0;
    const double* p = ws.partials + (size_t)slot * ws.stride;
    const int nt = blockDim.x * blockDim.y, nb = nblocks();
    for (int b = flat_tid(); b < nb; b += nt) v += __ldcg(p + b);
    return block_sum(v, sh);
}

__device__ __forceinline__ void reset_counter(RedWs ws) {
    if (flat_tid() == 0) *ws.counter = 0u;
}

// Products that must stay rounded on their own (never contracted into an
// FMA by the compiler): with every multiply-add of a stencil written as an
// explicit fma or one of these, each template instantiation of a kernel
// (tile heights, epilogues) rounds a node's value identically.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// One thread's share of a weighted dot product, sum of w a b over its
// nodes (w = 1/2 or 1).  FP64 operands: FP64 FMAs.  FP32 operands: a
// double-float accumulator (s + c) built from error-free transformations
// in FP32 only -- the product split exactly as p + e with an FMA, the sum
// by Knuth's TwoSum -- so each thread's partial carries ~2^-44 relative
// accuracy and is converted to FP64 once, for the FP64 block and grid
// sums.  GB300's FP64 pipe (2 FMA/clk/SM) would otherwise bound every FP32
// reduction kernel: a per-node conversion and FP64 FMA cost more than the
// node's memory traffic.  Every operation is rounded on its own (_rn), so
// no FMA contraction or reassociation can change the result.
template <typename T>
struct WSum;
template <>
struct WSum<double> {
    // interior rows (w = 1) and wall rows (w = 1/2) apart, so a node costs
    // one FP64 FMA (the weight is uniform along a row: no divergence)
    double v = 0.0, vw = 0.0;
    __device__ __forceinline__ void add(double w, double a, double b) {
        if (w == 1.0)
            v = fma(a, b, v);
        else
            vw = fma(a, b, vw);
    }
    __device__ __forceinline__ double get() const { return fma(0.5, vw, v); }
};
template <>
struct WSum<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float w, float a, float b) {
        const float wa = __fmul_rn(w, a);   // exact: w is 1/2 or 1
        const float p = __fmul_rn(wa, b);
        const float e = fmaf(wa, b, -p);    // p + e = wa b exactly
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// Block and grid reduction of WSum partials.  FP64 partials: FP64 warp
// shuffles and sums.  FP32 partials stay double-float pairs (s, c) through
// the warp, block and grid stages -- each addition Knuth's TwoSum of the
// leading parts with the trailing parts and its error added -- and are
// converted to FP64 once, at the end.  GB300's FP64 pipe issues 2 lanes per
// clock and SM, so an FP64 warp shuffle tree in every block cost ~4 us of
// FP64 issue per reduction kernel on a 1024^2 grid.  TwoSum is error free,
// so the two lanes of every butterfly step compute the same pair and all
// lanes end with identical values: the result is deterministic.
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    s = t;
    c = __fadd_rn(__fadd_rn(c, c2), err);
}
__device__ __forceinline__ void warp_sum_pair(float& s, float& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
        pair_add(s, c, s2, c2);
    }
}
// block-wide pair sum, result in every thread; `shd` holds >= 32 doubles
__device__ __forceinline__ void block_sum_pair(float& s, float& c, double* shd) {
    float2* sh = reinterpret_cast<float2*>(shd);
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = t & 31, wid = t >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    warp_sum_pair(s, c);
    __syncthreads();
    if (lane == 0) sh[wid] = make_float2(s, c);
    __syncthreads();
    float rs = 0.0f, rc = 0.0f;
    if (t < nw) {
        rs = sh[t].x;
        rc = sh[t].y;
    }
    if (wid == 0) warp_sum_pair(rs, rc);
    if (t == 0) sh[0] = make_float2(rs, rc);
    __syncthreads();
    s = sh[0].x;
    c = sh[0].y;
    __syncthreads();
}

// this block's partial of acc into slot (all threads call)
template <typename T>
__device__ __forceinline__ void publish_wsum(RedWs ws, int slot, const WSum<T>& acc, double* sh) {
    if constexpr (sizeof(T) == 4) {
        float s = acc.s, c = acc.c;
        block_sum_pair(s, c, sh);
        if (flat_tid() == 0)
            reinterpret_cast<float2*>(ws.partials + (size_t)slot * ws.stride)[flat_bid()] =
                make_float2(s, c);
    } else {
        publish_partial(ws, slot, block_sum(acc.get(), sh));
    }
}
// pair partial (s, c) of this block into slot (thread 0 writes)
__device__ __forceinline__ void publish_pair(RedWs ws, int slot, int block, float s, float c) {
    reinterpret_cast<float2*>(ws.partials + (size_t)slot * ws.stride)[block] = make_float2(s, c);
}
// the grid total of slot (the last block; all its threads get it)
template <typename T>
__device__ __forceinline__ double final_wsum(RedWs ws, int slot, double* sh) {
    if constexpr (sizeof(T) == 4) {
        const float2* p = reinterpret_cast<const float2*>(ws.partials + (size_t)slot * ws.stride);
        const int nt = blockDim.x * blockDim.y, nb = nblocks();
        float s = 0.0f, c = 0.0f;
        for (int b = flat_tid(); b < nb; b += nt) {
            const float2 v = __ldcg(p + b);
            pair_add(s, c, v.x, v.y);
        }
        block_sum_pair(s, c, sh);
        return (double)s + (double)c;
    } else {
        return final_sum(ws, slot, sh);
    }
}

// Block-uniform scalars of a kernel: thread 0 converts src[idx[k]] to T once
// per block.  A conversion from FP64 runs on the FP64 pipe (2 lanes per clock
// and SM on GB300); once per thread it cost about a microsecond per launch on
// a 1024^2 grid.  Call with every thread of the block.
template <typename T, int N>
__device__ __forceinline__ void block_scalars(const double* src, const int (&idx)[N], T (&out)[N]) {
    __shared__ T sh[N];
    if (threadIdx.x + blockDim.x * threadIdx.y == 0)
        for (int k = 0; k < N; ++k) sh[k] = (T)src[idx[k]];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = sh[k];
}

// trapezoid weight of flat index e (row-major [ny+1][nx])
__device__ __forceinline__ double wgt(size_t e, const Grid& g) {
    return (e < (size_t)g.nx || e >= g.n() - g.nx) ? 0.5 : 1.0;
}
// the same in the precision T of a kernel (no FP64 conversion in FP32 kernels)
template <typename T>
__device__ __forceinline__ T wgt_t(size_t e, const Grid& g) {
    return (e < (size_t)g.nx || e >= g.n() - g.nx) ? (T)0.5 : (T)1;
}

__device__ __forceinline__ int wrapx(int i, int nx) {
    i %= nx;
    return i < 0 ? i + nx : i;
}
// periodic wrap of a column index within [-nx, 2nx) (no division)
__device__ __forceinline__ int wrapx_near(int i, int nx) {
    return i < 0 ? i + nx : (i >= nx ? i - nx : i);
}
// even reflection of a row index about the walls, clamped into [0, ny]
__device__ __forceinline__ int refly(int j, int ny) {
    if (j < 0) j = -j;
    if (j > ny) j = 2 * ny - j;
    return j < 0 ? 0 : (j > ny ? ny : j);
}

}  // namespace cahn

// ---------------------------------------------------------------- host
#define CAHN_CUDA_TRY(expr)                                              \
    do {                                                                 \
        cudaError_t _e = (expr);                                         \
        if (_e != cudaSuccess) throw ::cahn::CudaError(_e, #expr, __FILE__, __LINE__); \
    } while (0)

#include <atomic>
#include <stdexcept>
#include <string>
namespace cahn {
// Host-side count of kernel launches issued by this library.  While a
// graph is being captured, launches are also attributed to g_frame (the
// graph's top level or the loop body being captured).
extern std::atomic<int64_t> g_launches;
extern thread_local int64_t* g_frame;
inline void note_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_frame) ++*g_frame;
}
struct CudaError : std::runtime_error {
    cudaError_t code;
    CudaError(cudaError_t e, const char* what, const char* file, int line)
        : std::runtime_error(std::string(cudaGetErrorString(e)) + " in " + what + " at " +
                             file + ":" + std::to_string(line)),
          code(e) {}
};
struct ArgError : std::runtime_error {
    using std::runtime_error::runtime_error;
};
}  // namespace cahn
