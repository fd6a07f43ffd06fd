// Machine-peak probes (Sec. 1.6 of the paper: own micro-benchmarks for the
// bandwidth and FP64 ceilings of the roofline model).
#include "tsm_internal.h"
#include "tsm_probe.h"

namespace tsm {
namespace {

constexpr int kChains = 16;  // independent FMA chains per thread

// DFMA peak in the form the products run: a TM x 4 register tile updated by
// the outer product of two register vectors (acc[m][n] += a[m] * b[n]), so
// every operand is a register (no constant-bank operand) and 4 TM
// independent accumulator chains per thread hide the pipe latency.  The
// operands come from the kernel argument, so nothing can be folded at
// compile time.
template <int TM>
__global__ void k_dfma_tile(int64_t iters, double seed, double* out) {
    double a[TM], b[4], acc[TM][4];
#pragma unroll
    for (int i = 0; i < TM; ++i) a[i] = seed + threadIdx.x * 1e-9 + i * 1e-3;
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = seed - threadIdx.x * 1e-9 - j * 1e-3;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
#pragma unroll 2
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s += acc[i][j];
    if (s == 12345.678) out[0] = s;  // keeps the chains alive
}

// The first form of the probe, kept for comparison: each chain multiplies
// its own running value by a compile-time constant (x = x * m + a).
__global__ void k_dfma_chain(int64_t iters, double seed, double* out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed + threadIdx.x * 1e-7 + c;
    const double m = 0.999999999, a = 1e-9;
#pragma unroll 4
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], m, a);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;
}

__global__ void k_dmma_peak(int64_t iters, double seed, double* out) {
    double acc[4][2];
    double av = seed + threadIdx.x * 1e-9, bv = 1.0 - threadIdx.x * 1e-9;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = 0.0;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            asm volatile(
                "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                : "+d"(acc[c][0]), "+d"(acc[c][1])
                : "d"(av), "d"(bv));
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
    if (s == 12345.678) out[0] = s;
}

// Read-only stream.  Each CTA takes contiguous chunks of ILP x blockDim
// 16-byte vectors (chunk c, then c + gridDim.x, ...), so the ILP loads a
// thread keeps in flight are coalesced and fall in the same DRAM pages.
// The loaded bits are folded with integer XOR so that the FP64 pipe (slow
// on this part) never limits the measured bandwidth.
template <int ILP>
__global__ void k_read(const double2* __restrict__ x, int64_t n, double* out) {
    unsigned long long s0 = 0, s1 = 0;
    const int64_t chunk = (int64_t)ILP * blockDim.x;
    const int64_t nfull = n / chunk;
    for (int64_t c = blockIdx.x; c < nfull; c += gridDim.x) {
        const double2* p = x + c * chunk + threadIdx.x;
        double2 v[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) v[u] = __ldcs(p + u * blockDim.x);
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            s0 ^= __double_as_longlong(v[u].x);
            s1 ^= __double_as_longlong(v[u].y);
        }
    }
    for (int64_t i = nfull * chunk + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = __ldcs(x + i);
        s0 ^= __double_as_longlong(v.x);
        s1 ^= __double_as_longlong(v.y);
    }
    if ((s0 ^ s1) == 0x123456789abcdefull) out[0] = (double)s0;
}

// Read-modify-write stream with the same chunking (the STREAM "scale"
// kernel with factor 1, which leaves the buffer unchanged).
template <int ILP>
__global__ void k_scale_stream(double2* x, int64_t n) {
    const int64_t chunk = (int64_t)ILP * blockDim.x;
    const int64_t nfull = n / chunk;
    for (int64_t c = blockIdx.x; c < nfull; c += gridDim.x) {
        double2* p = x + c * chunk + threadIdx.x;
        double2 v[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) v[u] = __ldcs(p + u * blockDim.x);
#pragma unroll
        for (int u = 0; u < ILP; ++u) __stcs(p + u * blockDim.x, make_double2(v[u].x * 1.0, v[u].y * 1.0));
    }
    for (int64_t i = nfull * chunk + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        __stcs(x + i, __ldcs(x + i));
}

struct Timer {
    cudaEvent_t a, b;
    cudaStream_t s;
    bool ok;
    explicit Timer(cudaStream_t st) : s(st) {
        ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, s); }
    float stop() {
        cudaEventRecord(b, s);
        float ms = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return -1.f;
        return ms;
    }
};

}  // namespace
}  // namespace tsm

using namespace tsm;

extern "C" tsm_status tsm_probe_fp64(int mode, int64_t iters, double* gflops, tsm_stream_t stream) {
    if (mode < 0 || mode > 2 || !gflops || iters < 1) return TSM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    const int sm = device_info().sm_count;
    double* dummy = nullptr;
    if (cudaMalloc(&dummy, 64) != cudaSuccess) return TSM_ERR_ALLOC;
    Timer t(s);
    if (!t.ok) {
        cudaFree(dummy);
        return TSM_ERR_LAUNCH;
    }
    // mode 0 tries 1, 2 and 4 CTAs of 256 threads per SM with 16 and 32
    // chains per thread (the products run 1-2 CTAs of 256 threads per SM)
    // and keeps the fastest; modes 1 and 2 run 4 CTAs per SM
    double best_gflops = 0.0;
    const int nshape = mode == 0 ? 6 : 1;
    for (int shape = 0; shape < nshape; ++shape) {
        const int cps = mode == 0 ? (1 << (shape % 3)) : 4;
        const int tm = mode == 0 && shape >= 3 ? 8 : 4;
        const int blocks = sm * cps, threads = 256;
        // the same number of FMAs per SM for every shape
        const int64_t it = mode == 0 ? iters * 4 / cps * 4 / tm : iters;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {  // the first pass warms up the clocks
            t.start();
            if (mode == 0 && tm == 4)
                k_dfma_tile<4><<<blocks, threads, 0, s>>>(it, 1.0, dummy);
            else if (mode == 0)
                k_dfma_tile<8><<<blocks, threads, 0, s>>>(it, 1.0, dummy);
            else if (mode == 1)
                k_dmma_peak<<<blocks, threads, 0, s>>>(it, 1.0, dummy);
            else
                k_dfma_chain<<<blocks, threads, 0, s>>>(it, 1.0, dummy);
            const float ms = t.stop();
            if (rep > 0 && ms > 0.f && ms < best) best = ms;
        }
        if (best >= 1e29f) break;
        double flops;
        if (mode == 1)
            flops = 2.0 * 8 * 8 * 4 * 4 * (double)it * blocks * (threads / 32);
        else
            flops = 2.0 * (mode == 0 ? 4 * tm : kChains) * (double)it * blocks * threads;  // 2 flops per FMA
        const double g = flops / (best * 1e-3) / 1e9;
        if (g > best_gflops) best_gflops = g;
    }
    cudaFree(dummy);
    if (best_gflops <= 0.0 || cudaGetLastError() != cudaSuccess) return TSM_ERR_LAUNCH;
    *gflops = best_gflops;
    return TSM_OK;
}

extern "C" tsm_status tsm_probe_bandwidth(void* buffer, size_t bytes, int mode, int ilp, int blocks_in,
                                          int threads_in, double* gbs, tsm_stream_t stream) {
    if (!buffer || !gbs || bytes < 16 || (bytes % 16) || ((uintptr_t)buffer % 16)) return TSM_ERR_INVALID_VALUE;
    if ((mode != 0 && mode != 1) || (ilp != 1 && ilp != 4 && ilp != 16) || blocks_in < 0) return TSM_ERR_INVALID_VALUE;
    if (threads_in != 0 && (threads_in < 32 || threads_in > 1024 || threads_in % 32)) return TSM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    const int sm = device_info().sm_count;
    const int blocks = blocks_in > 0 ? blocks_in : sm * 8;
    const int threads = threads_in > 0 ? threads_in : 256;
    const int64_t n = (int64_t)(bytes / 16);
    double* dummy = nullptr;
    if (cudaMalloc(&dummy, 64) != cudaSuccess) return TSM_ERR_ALLOC;
    Timer t(s);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        t.start();
        if (mode == 0) {
            if (ilp == 1) k_read<1><<<blocks, threads, 0, s>>>((const double2*)buffer, n, dummy);
            if (ilp == 4) k_read<4><<<blocks, threads, 0, s>>>((const double2*)buffer, n, dummy);
            if (ilp == 16) k_read<16><<<blocks, threads, 0, s>>>((const double2*)buffer, n, dummy);
        } else {
            if (ilp == 1) k_scale_stream<1><<<blocks, threads, 0, s>>>((double2*)buffer, n);
            if (ilp == 4) k_scale_stream<4><<<blocks, threads, 0, s>>>((double2*)buffer, n);
            if (ilp == 16) k_scale_stream<16><<<blocks, threads, 0, s>>>((double2*)buffer, n);
        }
        const float ms = t.stop();
        if (ms > 0.f && ms < best) best = ms;
    }
    cudaFree(dummy);
    if (best >= 1e29f || cudaGetLastError() != cudaSuccess) return TSM_ERR_LAUNCH;
    *gbs = (double)bytes * (mode == 1 ? 2.0 : 1.0) / (best * 1e-3) / 1e9;
    return TSM_OK;
}
