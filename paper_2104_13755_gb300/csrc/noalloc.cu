// Residual norms of a caller-supplied CSR system without any allocation.
//
// Some callers cannot allocate device memory at the moment they need this:
// real-time frame loops, where cudaMalloc or cudaFree may synchronise the
// device and stall the frame, and host applications that give a plug-in a
// fixed device budget and own every allocation themselves.  This entry point
// serves them:
// the caller passes the matrix and vectors it already owns, and the only
// scratch -- one partial sum per block of the first kernel -- lives in the
// fixed-size array below, which is part of the library image and stays
// resident on every GPU that loads the library until the process exits.
//
// The reduction is the same two-phase, fixed-order one the solver uses for its
// stopping test, so repeated calls on the same data give identical bits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/smg.h"
#include "plan.hpp"

namespace {

constexpr int kBlocks = 608;   // grid of the first kernel
constexpr int kThreads = 256;
constexpr int kMaxRhs = 4;
// partial sums: kBlocks rows of (||r_q||^2, ||b_q||^2) for q < kMaxRhs
constexpr int kScratchDoubles = kBlocks * 2 * kMaxRhs;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

template <int K>
__global__ void __launch_bounds__(kThreads) csr_resnorm_partial(int64_t n, const int64_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ col,
                                                                const double* __restrict__ vals,
                                                                const double* __restrict__ x,
                                                                const double* __restrict__ b,
                                                                double* __restrict__ scratch) {
    double rr[K], bb[K];
#pragma unroll
    for (int q = 0; q < K; q++) rr[q] = bb[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        double acc[K];
#pragma unroll
        for (int q = 0; q < K; q++) acc[q] = b[i * K + q];
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const double a = vals[p];
            const int64_t j = col[p];
#pragma unroll
            for (int q = 0; q < K; q++) acc[q] -= a * x[j * K + q];
        }
#pragma unroll
        for (int q = 0; q < K; q++) {
            const double bv = b[i * K + q];
            rr[q] += acc[q] * acc[q];
            bb[q] += bv * bv;
        }
    }
    __shared__ double red[kThreads / 32][2 * K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < K; q++)
        for (int o = 16; o > 0; o >>= 1) {
            rr[q] += __shfl_xor_sync(0xffffffffu, rr[q], o);
            bb[q] += __shfl_xor_sync(0xffffffffu, bb[q], o);
        }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; q++) {
            red[wid][q] = rr[q];
            red[wid][K + q] = bb[q];
        }
    __syncthreads();
    if (threadIdx.x < 2 * K) {  // every slot of this block is overwritten: no clearing needed
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; w++) s += red[w][threadIdx.x];
        scratch[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = s;
    }
}

template <int K>
__global__ void __launch_bounds__(kThreads) csr_resnorm_final(const double* __restrict__ scratch,
                                                              double* __restrict__ out) {
    __shared__ double red[kThreads][2 * K];
    double acc[2 * K];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) acc[q] = 0.0;
    for (int blk = threadIdx.x; blk < kBlocks; blk += kThreads)
#pragma unroll
        for (int q = 0; q < 2 * K; q++) acc[q] += scratch[(int64_t)blk * 2 * K + q];
#pragma unroll
    for (int q = 0; q < 2 * K; q++) red[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 2 * K; q++) red[threadIdx.x][q] += red[threadIdx.x + w][q];
        __syncthreads();
    }
    if (threadIdx.x < 2 * K) out[threadIdx.x] = red[0][threadIdx.x];
}

// Device address of g_scratch, looked up once per device and context (the
// host-side symbol is only a stand-in and must never be handed to a kernel).
// The address belongs to the context the module was loaded in: after
// cudaDeviceReset, or with another context current on the device, the
// lookup is repeated.  The current context comes from the driver's
// cuCtxGetCurrent, reached through the runtime (no link to the driver
// library); where that is unavailable the address is looked up on every call.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
struct ScratchAddr {
    void* ctx = nullptr;
    double* ptr = nullptr;
};
ScratchAddr g_scratch_dev[kMaxDevices];

typedef int (*CtxGetCurrentFn)(void**);  // CUresult cuCtxGetCurrent(CUcontext*)

CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (CtxGetCurrentFn)f;
    }();
    return fn;
}

void* current_context() {
    CtxGetCurrentFn fn = ctx_get_current();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

int scratch_for_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        smg::set_error("no usable current CUDA device");
        return SMG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> guard(g_lock);
    ScratchAddr& a = g_scratch_dev[dev];
    void* ctx = current_context();
    if (!a.ptr || !ctx || ctx != a.ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);  // also makes the primary context current
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            smg::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SMG_ERR_CUDA;
        }
        a.ptr = (double*)p;
        a.ctx = current_context();
    }
    *out = a.ptr;
    return SMG_OK;
}

template <int K>
cudaError_t run(int64_t n, const int64_t* rowptr, const int32_t* col, const double* vals, const double* x,
                const double* b, double* out, double* scratch, cudaStream_t s) {
    csr_resnorm_partial<K><<<kBlocks, kThreads, 0, s>>>(n, rowptr, col, vals, x, b, scratch);
    csr_resnorm_final<K><<<1, kThreads, 0, s>>>(scratch, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" int smg_residual_norms_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col, const double* vals,
                                          const double* x, const double* b, int nrhs, double* out,
                                          smg_stream stream) {
    if (!rowptr || !col || !vals || !x || !b || !out || n < 1) {
        smg::set_error("smg_residual_norms_noalloc: null pointer or empty system");
        return SMG_ERR_INVALID_ARG;
    }
    if (nrhs < 1 || nrhs > kMaxRhs) {
        smg::set_error("smg_residual_norms_noalloc: nrhs must be 1..4 (the fixed scratch holds " +
                       std::to_string(kBlocks) + " blocks x 2 x 4 partial sums)");
        return SMG_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st != SMG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (nrhs) {
        case 1: e = run<1>(n, rowptr, col, vals, x, b, out, scratch, s); break;
        case 2: e = run<2>(n, rowptr, col, vals, x, b, out, scratch, s); break;
        case 3: e = run<3>(n, rowptr, col, vals, x, b, out, scratch, s); break;
        default: e = run<4>(n, rowptr, col, vals, x, b, out, scratch, s); break;
    }
    if (e != cudaSuccess) {
        smg::set_error(std::string("smg_residual_norms_noalloc: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    return SMG_OK;
}
