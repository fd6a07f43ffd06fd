// One block Gram-Schmidt step in a single cooperative kernel (the use of
// TSMTTSM followed by TSMM that Sec. 1.2 of the paper describes):
//     C = op(A)^T B     (op = conjugate transpose for complex data)
//     B = B - A C
// Every CTA owns one contiguous range of rows for the whole step:
//   1. it forms its partial of C over its rows (register tiles, Sec. 3) and
//      sums its row lanes in a fixed order into a partial slot;
//   2. grid barrier; CTA b sums a slice of C's entries over all partial
//      slots in slot order and stores those entries of C;
//   3. grid barrier; it stages -C in shared memory and updates its own rows
//      of B (TSMM with beta = 1, Sec. 4).
// At small K the rows a CTA updates in step 3 are the rows it read in step 1,
// still in L2, and the step costs one launch instead of two.
//
// The barriers are a counter and a flag in the stream workspace: the
// arrival that completes a barrier publishes the launch's generation number
// in the flag, and the CTAs poll the flag with a clock budget.  The launch is
// cooperative, so every CTA is resident and each barrier completes; the
// budget only turns an impossible hang into an error word (tsm_gs_status).
// Every CTA arrives at both barriers even after a wait gave up, so the
// counter is back at zero for the next launch.
#include <cstdint>

#include "fp64_common.cuh"
#include "tsm_internal.h"

namespace tsm {
namespace gsf {

constexpr int kThreads = 256;
constexpr long long kDefaultTimeout = 4000000000LL;  // SM clock cycles, about two seconds
long long g_timeout = kDefaultTimeout;

// Words of the stream workspace's ticket array used here.
constexpr int kCountWord = 48, kFlagWord = 49, kErrWord = 50;

struct Args {
    int M, N, cplx;
    int64_t K;
    const double* A;
    int64_t lda;
    double* B;
    int64_t ldb;
    double* C;
    int64_t ldc;
    double* parts;       // grid x M x N (x 2) partial slots
    unsigned* words;     // the workspace ticket array
    unsigned gen;        // this launch's barrier generations are gen + 1, gen + 2
    long long timeout;   // clock budget of one barrier wait
};

__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier j (0 or 1) with a bounded wait.  Thread 0 of each CTA takes
// an arrival index i from the launch's counter; arrivals G - 1 and 2G - 1
// release barriers 0 and 1 by raising the flag to gen + 1 and gen + 2 (a
// maximum, so it never moves back), and arrival 2G - 1 -- the launch's last
// -- also returns the counter to zero for the next launch.  Every CTA
// arrives exactly twice, so this holds even when a wait gave up and the
// arrivals of the two barriers interleave.  Returns false (and sets the
// error word) if this CTA's wait gave up.
__device__ bool grid_barrier(const Args& a, unsigned j) {
    __shared__ int s_ok;
    __threadfence();  // every thread's writes, before the CTA arrives
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned G = gridDim.x;
        const unsigned target = a.gen + j + 1u;
        const unsigned i = atomicAdd(&a.words[kCountWord], 1u);
        if (i % G == G - 1u) {
            if (i == 2u * G - 1u) a.words[kCountWord] = 0u;
            __threadfence();
            atomicMax(&a.words[kFlagWord], a.gen + i / G + 1u);
        }
        const long long t0 = clock64();
        while ((int)(load_acquire(&a.words[kFlagWord]) - target) < 0) {
            if (clock64() - t0 > a.timeout) {
                atomicExch(&a.words[kErrWord], 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Step 1: this CTA's partial of op(A)^T B over rows [k0, k1).  Thread
// (lane, p) holds the TM x TN tile at C[pm + i*PM][pn + j*PN]; lanes take
// rows k0 + lane, k0 + lane + L, ...; the lanes of each entry are summed
// by a fixed-pairing tree in shared memory.
template <int TM, int TN, bool CPLX>
__device__ void partial_tile(const Args& a, int64_t k0, int64_t k1, double* part, double* red) {
    constexpr int CC = CPLX ? 2 : 1;
    const int M = a.M, N = a.N;
    const int PM = (M + TM - 1) / TM, PN = (N + TN - 1) / TN, P = PM * PN;
    const int L = kThreads / P;
    const int t = threadIdx.x;
    const int lane = t / P, p = t - lane * P;
    const int pm = p % PM, pn = p / PM;
    const bool active = lane < L;
    int mi[TM], nj[TN];
    bool mok[TM], nok[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        mi[i] = pm + i * PM;
        mok[i] = mi[i] < M;
        if (!mok[i]) mi[i] = 0;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        nj[j] = pn + j * PN;
        nok[j] = nj[j] < N;
        if (!nok[j]) nj[j] = 0;
    }
    double acc[TM][TN][CC];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
#pragma unroll
            for (int c = 0; c < CC; ++c) acc[i][j][c] = 0.0;
    const int64_t sa = a.lda * CC, sb = a.ldb * CC;
    if (active) {
        for (int64_t k = k0 + lane; k < k1; k += L) {
            const double* ar = a.A + k * sa;
            const double* br = a.B + k * sb;
            double av[TM][CC], bv[TN][CC];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int c = 0; c < CC; ++c) av[i][c] = mok[i] ? ar[mi[i] * CC + c] : 0.0;
#pragma unroll
            for (int j = 0; j < TN; ++j)
#pragma unroll
                for (int c = 0; c < CC; ++c) bv[j][c] = nok[j] ? br[nj[j] * CC + c] : 0.0;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    if (!CPLX) {
                        acc[i][j][0] = fma(av[i][0], bv[j][0], acc[i][j][0]);
                    } else {
                        // conj(a) * b
                        const double ar_ = av[i][0], ai = av[i][CC - 1];
                        const double br_ = bv[j][0], bi = bv[j][CC - 1];
                        acc[i][j][0] = fma(ar_, br_, acc[i][j][0]);
                        acc[i][j][0] = fma(ai, bi, acc[i][j][0]);
                        acc[i][j][CC - 1] = fma(ar_, bi, acc[i][j][CC - 1]);
                        acc[i][j][CC - 1] = fma(-ai, br_, acc[i][j][CC - 1]);
                    }
                }
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
#pragma unroll
            for (int c = 0; c < CC; ++c) {
                if (active) red[lane * P + p] = acc[i][j][c];
                __syncthreads();
                for (int n = L; n > 1;) {
                    const int h = (n + 1) >> 1;
                    if (active && lane + h < n) red[lane * P + p] += red[(lane + h) * P + p];
                    __syncthreads();
                    n = h;
                }
                if (t < P) {
                    const int m = (t % PM) + i * PM, n = (t / PM) + j * PN;
                    if (m < M && n < N) part[(m * N + n) * CC + c] = red[t];
                }
                __syncthreads();
            }
}

// Step 2: entries [e0, e1) of C summed over the G partial slots.  S threads
// share an entry (thread s takes slots s, s + S, ... in order); the S slice
// sums are combined by a fixed-pairing tree in shared memory.
template <bool CPLX>
__device__ void reduce_slice(const Args& a, int e0, int e1, double* red) {
    constexpr int CC = CPLX ? 2 : 1;
    const int G = gridDim.x, MNc = a.M * a.N * CC;
    const int t = threadIdx.x;
    const int ne = e1 - e0;
    if (ne <= 0) return;
    int S = 1;
    while (S < 32 && S * 2 * ne <= kThreads && S * 2 <= G) S *= 2;
    for (int base = 0; base < ne * S; base += kThreads) {
        const int w = base + t;
        const bool mine = w < ne * S;
        const int e = e0 + (mine ? w / S : 0), s = w % S;
        double v[CC];
#pragma unroll
        for (int c = 0; c < CC; ++c) v[c] = 0.0;
        if (mine)
            for (int g = s; g < G; g += S)
#pragma unroll
                for (int c = 0; c < CC; ++c) v[c] += __ldcg(a.parts + (int64_t)g * MNc + e * CC + c);
#pragma unroll
        for (int c = 0; c < CC; ++c) red[t * CC + c] = v[c];
        __syncthreads();
        for (int h = S >> 1; h >= 1; h >>= 1) {
            if (mine && s < h)
#pragma unroll
                for (int c = 0; c < CC; ++c) red[t * CC + c] += red[(t + h) * CC + c];
            __syncthreads();
        }
        if (mine && s == 0) {
            const int m = e / a.N, n = e - m * a.N;
#pragma unroll
            for (int c = 0; c < CC; ++c) a.C[((int64_t)m * a.ldc + n) * CC + c] = red[t * CC + c];
        }
        __syncthreads();
    }
}

// Step 3: rows [k0, k1) of B updated with -C staged in shared memory.  N
// threads per row (one result each), kThreads / N rows per pass.
template <bool CPLX>
__device__ void update_rows(const Args& a, int64_t k0, int64_t k1, double* cs) {
    constexpr int CC = CPLX ? 2 : 1;
    const int M = a.M, N = a.N;
    for (int o = threadIdx.x; o < M * N; o += kThreads) {
        const int m = o / N, n = o - m * N;
#pragma unroll
        for (int c = 0; c < CC; ++c) cs[o * CC + c] = -__ldcg(a.C + ((int64_t)m * a.ldc + n) * CC + c);
    }
    __syncthreads();
    const int rpc = kThreads / N;
    const int r = threadIdx.x / N, n = threadIdx.x - r * N;
    if (r >= rpc) return;
    const int64_t sa = a.lda * CC, sb = a.ldb * CC;
    for (int64_t k = k0 + r; k < k1; k += rpc) {
        const double* ar = a.A + k * sa;
        double* br = a.B + k * sb + n * CC;
        double acc[CC];
#pragma unroll
        for (int c = 0; c < CC; ++c) acc[c] = br[c];
        for (int m = 0; m < M; ++m) {
            const double cr = cs[(m * N + n) * CC], ci = cs[(m * N + n) * CC + CC - 1];
            if (!CPLX) {
                acc[0] = fma(ar[m], cr, acc[0]);
            } else {
                const double xr = ar[2 * m], xi = ar[2 * m + 1];
                acc[0] = fma(xr, cr, acc[0]);
                acc[0] = fma(-xi, ci, acc[0]);
                acc[CC - 1] = fma(xr, ci, acc[CC - 1]);
                acc[CC - 1] = fma(xi, cr, acc[CC - 1]);
            }
        }
#pragma unroll
        for (int c = 0; c < CC; ++c) br[c] = acc[c];
    }
}

template <int TM, int TN, bool CPLX>
__global__ void __launch_bounds__(kThreads) k_gs_fused(const Args a) {
    constexpr int CC = CPLX ? 2 : 1;
    extern __shared__ double dyn[];  // max(2 * kThreads, M * N) * CC doubles
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int64_t k0 = a.K * b / G, k1 = a.K * (b + 1) / G;
    const int MNc = a.M * a.N * CC;
    partial_tile<TM, TN, CPLX>(a, k0, k1, a.parts + b * MNc, dyn);
    bool ok = grid_barrier(a, 0u);
    const int E = a.M * a.N;
    if (ok) reduce_slice<CPLX>(a, (int)(E * b / G), (int)(E * (b + 1) / G), dyn);
    ok = grid_barrier(a, 1u) && ok;
    if (ok) update_rows<CPLX>(a, k0, k1, dyn);
}

}  // namespace gsf
}  // namespace tsm

namespace tsm {
namespace gsf {

typedef void (*Kernel)(const Args);

// Register tile T x T (T in 1, 2, 4), among those that need at most
// kThreads threads per row lane (4 x 4 always does for M, N <= 64).  For
// M N <= kThreads the 1 x 1 tile: the lane reduction after step 1 (TM TN
// entries, log2 L levels each) then costs more than the loads a larger tile
// saves.  Above that the least padded work ceil(M/T) T ceil(N/T) T, ties to
// the larger tile, which loads less per FMA.
int tile_for(int M, int N) {
    if (M * N <= kThreads) return 1;
    int best = 4;
    long long bw = 1LL << 60;
    for (int t = 2; t <= 4; t *= 2) {
        if ((long long)((M + t - 1) / t) * ((N + t - 1) / t) > kThreads) continue;
        const long long w = (long long)((M + t - 1) / t) * t * ((N + t - 1) / t) * t;
        if (w <= bw) {
            bw = w;
            best = t;
        }
    }
    return best;
}

Kernel kernel_for(int tile, int cplx) {
    if (cplx) return tile == 4 ? k_gs_fused<4, 4, true> : (tile == 2 ? k_gs_fused<2, 2, true> : k_gs_fused<1, 1, true>);
    return tile == 4 ? k_gs_fused<4, 4, false> : (tile == 2 ? k_gs_fused<2, 2, false> : k_gs_fused<1, 1, false>);
}

size_t smem_for(int M, int N, int cplx) {
    const size_t cc = cplx ? 2 : 1;
    const size_t need = (size_t)M * N * cc;
    const size_t red = 2 * (size_t)kThreads;
    return (need > red ? need : red) * sizeof(double);
}

tsm_status run(tsm_dtype dtype, int M, int N, int64_t K, const void* A, int64_t lda, void* B, int64_t ldb,
               void* C, int64_t ldc, cudaStream_t s) {
    const int cplx = dtype == TSM_C64;
    const DeviceInfo& di = device_info();
    const Kernel k = kernel_for(tile_for(M, N), cplx);
    const size_t smem = smem_for(M, N, cplx);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TSM_ERR_LAUNCH;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, smem) != cudaSuccess || occ < 1)
        return TSM_ERR_LAUNCH;
    // at most two CTAs per SM, and about 4096 FMAs of each product per CTA
    // at least (1 to 128 rows): products with many FMAs per row spread over
    // every SM even at small K, narrow ones meet at the barriers with fewer
    // CTAs
    int64_t grid = (int64_t)di.sm_count * (occ < 2 ? occ : 2);
    int64_t rmin = 4096 / ((int64_t)M * N * (cplx ? 4 : 1));
    if (rmin < 1) rmin = 1;
    if (rmin > 128) rmin = 128;
    const int64_t by_rows = (K + rmin - 1) / rmin;
    if (grid > by_rows) grid = by_rows;
    if (grid < 1) grid = 1;
    Workspace* ws = nullptr;
    const size_t pbytes = (size_t)grid * M * N * (cplx ? 2 : 1) * sizeof(double);
    tsm_status st = workspace_get(s, pbytes, 64, &ws);
    if (st != TSM_OK) return st;
    Args a;
    a.M = M;
    a.N = N;
    a.cplx = cplx;
    a.K = K;
    a.A = (const double*)A;
    a.lda = lda;
    a.B = (double*)B;
    a.ldb = ldb;
    a.C = (double*)C;
    a.ldc = ldc;
    a.parts = ws->partials;
    a.words = ws->tickets;
    a.gen = ws->gs_gen;
    a.timeout = g_timeout;
    void* params[] = {&a};
    if (cudaLaunchCooperativeKernel((const void*)k, dim3((unsigned)grid), dim3(kThreads), params, smem, s) !=
        cudaSuccess)
        return TSM_ERR_LAUNCH;
    ws->gs_gen += 2u;
    return TSM_OK;
}

}  // namespace gsf

tsm_status gs_fused_run(tsm_dtype dtype, int M, int N, int64_t K, const void* A, int64_t lda, void* B,
                        int64_t ldb, void* C, int64_t ldc, cudaStream_t s) {
    return gsf::run(dtype, M, N, K, A, lda, B, ldb, C, ldc, s);
}

// Fused up to 2^15 rows.  Measured on 12 shapes (real and complex, 1 x 1
// to 64 x 64 and 37 x 53) at K = 1, 3000, 10^4 and 2^15, the fused step was
// faster or within 2 % at 46 of the 48 points (up to 3.3x faster: complex
// 64 x 64 at K = 3000); the two exceptions are real 16 x 16 and 37 x 53 at
// 2^15 (12 % and 2.4 % slower).  Above 2^15 the tuned product kernels win.
bool gs_fused_preferred(tsm_dtype, int, int, int64_t K) { return K <= (1 << 15); }

}  // namespace tsm

using namespace tsm;

extern "C" {

tsm_status tsm_gs_status(tsm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    Workspace* ws = nullptr;
    tsm_status st = workspace_get(s, 256, 64, &ws);
    if (st != TSM_OK) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TSM_ERR_LAUNCH;
    unsigned err = 0;
    unsigned* p = ws->tickets + gsf::kErrWord;
    if (cudaMemcpy(&err, p, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return TSM_ERR_LAUNCH;
    if (err) {
        const unsigned zero = 0;
        if (cudaMemcpy(p, &zero, sizeof(unsigned), cudaMemcpyHostToDevice) != cudaSuccess) return TSM_ERR_LAUNCH;
        return TSM_ERR_TIMEOUT;
    }
    return TSM_OK;
}

tsm_status tsm_gs_set_timeout(int64_t timeout_cycles) {
    gsf::g_timeout = timeout_cycles > 0 ? (long long)timeout_cycles : gsf::kDefaultTimeout;
    return TSM_OK;
}

}  // extern "C"
