// Hand-written FP64 kernel families for TSMTTSM and TSMM (binary64 on the
// FP64 pipe, no tensor cores).
//
// TSMTTSM (Sec. 3): the long K loop is split into one contiguous row range
// per CTA; inside a CTA, P = ceil(M/T_M) * ceil(N/T_N) threads each own a
// T_M x T_N register tile of C (Listing 5) and L = 256 / P row lanes walk the
// range with stride L, U rows per iteration (the loads of U rows are issued
// before their FMAs, which plays the role of the paper's leap frogging,
// Sec. 3.1).  Tiles use the transposed mapping of Fig. 10: tile entry (i, j)
// of thread (pm, pn) is C[pm + i*PM][pn + j*PN], so neighbouring threads load
// neighbouring addresses.  Tile entries past M or N are guarded (Sec. 2.1).
//
// Reduction (Sec. 3.2, replaced by a deterministic scheme): lanes of a CTA
// are summed through shared memory in lane order; each CTA writes its M x N
// partial to a workspace; the last CTA to take a ticket sums the partials in
// CTA order, applies alpha/beta and resets the ticket.  No floating-point
// atomics, so results repeat bit for bit.
//
// TSMM (Sec. 4): alpha*C is staged once per CTA in shared memory (Sec. 4.2);
// TPR threads share one row of B and each computes up to NPT results,
// interleaved (Fig. 12) so that consecutive threads store consecutive
// elements; U rows per thread per iteration reuse every C value U times
// (Sec. 4.2, Fig. 13).  The grid is persistent (a multiple of the SM count)
// and walks K with a grid stride.
#include <cstdio>
#include <cstring>

#include "fp64_common.cuh"
#include "fp64_tsmttsm.cuh"
#include "tsm_internal.h"

namespace tsm {
namespace {

// --------------------------------------------------------------------- TSMM

template <int TPR, int NPT, int U, bool CPLX, bool GEN>
__global__ void __launch_bounds__(kBlock) k_tsmm(const TsmmArgs a) {
    constexpr int CC = CPLX ? 2 : 1;
    constexpr int RPC = kBlock / TPR;  // rows per CTA per unrolled step
    extern __shared__ double cs[];     // alpha * C, M x N (x CC)
    const int N = a.N, M = a.M;
    tsmm_begin(a);
    tsmm_stage_c<CC>(a, cs);

    const int r = threadIdx.x / TPR, q = threadIdx.x - r * TPR;
    const int npt = (N + TPR - 1) / TPR;  // result slots in use, <= NPT
    const double* __restrict__ A = a.A;
    const int64_t sa = a.lda * CC, sb = a.ldb * CC;
    const int64_t step = (int64_t)gridDim.x * RPC * U;
    for (int64_t base = (int64_t)blockIdx.x * RPC * U; base < a.K; base += step) {
        int64_t row[U];
        bool rok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            row[u] = base + r + (int64_t)u * RPC;
            rok[u] = row[u] < a.K;
            if (!rok[u]) row[u] = 0;
        }
        double acc[U][NPT][CC], ob[U][NPT][CC];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < NPT; ++j)
#pragma unroll
                for (int c = 0; c < CC; ++c) acc[u][j][c] = ob[u][j][c] = 0.0;
        if (!a.beta_zero) {
            // old B values first, so their latency overlaps the FMAs; the
            // beta term then opens each FMA chain (tsmm_acc_init)
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < NPT; ++j) {
                    if (j >= npt) break;
                    const int n = q + j * TPR;
                    if (rok[u] && n < N)
#pragma unroll
                        for (int c = 0; c < CC; ++c) ob[u][j][c] = a.B[row[u] * sb + n * CC + c];
                    tsmm_acc_init<CC, GEN>(a, ob[u][j][0], ob[u][j][CC - 1], acc[u][j][0], acc[u][j][CC - 1]);
                }
        }
#pragma unroll 2
        for (int m = 0; m < M; ++m) {
            double av[U][CC];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < CC; ++c) av[u][c] = rok[u] ? __ldg(A + row[u] * sa + m * CC + c) : 0.0;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                // CTA-uniform bound: unused result slots are branched around
                // (predicated-off FMAs still occupy the FP64 pipe)
                if (j >= npt) break;
                const int n = q + j * TPR;
                if (n < N) {
                    const double cr = cs[(m * N + n) * CC];
                    const double ci = cs[(m * N + n) * CC + CC - 1];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (!CPLX) {
                            acc[u][j][0] = fma(av[u][0], cr, acc[u][j][0]);
                        } else {
                            const double ar = av[u][0], ai = av[u][CC - 1];
                            acc[u][j][0] = fma(ar, cr, acc[u][j][0]);
                            acc[u][j][0] = fma(-ai, ci, acc[u][j][0]);
                            acc[u][j][CC - 1] = fma(ar, ci, acc[u][j][CC - 1]);
                            acc[u][j][CC - 1] = fma(ai, cr, acc[u][j][CC - 1]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!rok[u]) continue;
            double* out = a.B + row[u] * sb;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                if (j >= npt) break;
                const int n = q + j * TPR;
                if (n >= N) continue;
                tsmm_store_plain<CC>(out, n, acc[u][j][0], acc[u][j][CC - 1]);
            }
        }
    }
}

template <int TPR, int NPT, int U, bool CPLX>
size_t tsmm_smem(int M, int N) {
    return (size_t)M * N * (CPLX ? 2 : 1) * sizeof(double);
}

template <int TPR, int NPT, int U, bool CPLX, bool GEN>
cudaError_t launch_tsmm_as(const TsmmArgs& a, int grid, cudaStream_t s) {
    const size_t smem = tsmm_smem<TPR, NPT, U, CPLX>(a.M, a.N);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tsmm<TPR, NPT, U, CPLX, GEN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k_tsmm<TPR, NPT, U, CPLX, GEN>, grid, kBlock, smem, s, a);
}

template <int TPR, int NPT, int U, bool CPLX>
cudaError_t launch_tsmm(const TsmmArgs& a, int grid, cudaStream_t s) {
    return tsmm_general_beta(a) ? launch_tsmm_as<TPR, NPT, U, CPLX, true>(a, grid, s)
                                : launch_tsmm_as<TPR, NPT, U, CPLX, false>(a, grid, s);
}

template <int TPR, int NPT, int U, bool CPLX>
int occ_tsmm(int M, int N) {
    if (N > TPR * NPT) return 0;
    const size_t smem = tsmm_smem<TPR, NPT, U, CPLX>(M, N);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_tsmm<TPR, NPT, U, CPLX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tsmm<TPR, NPT, U, CPLX, false>, kBlock, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

// ------------------------------------------------------------ scale kernels

__global__ void k_scale(double* X, int64_t rows, int cols, int64_t ld, int cplx, double br, double bi,
                        int beta_zero) {
    const int64_t total = rows * cols;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = o / cols, c = o - r * cols;
        if (!cplx) {
            double* p = X + r * ld + c;
            *p = beta_zero ? 0.0 : br * *p;
        } else {
            double* p = X + (r * ld + c) * 2;
            if (beta_zero) {
                p[0] = 0.0;
                p[1] = 0.0;
            } else {
                const double xr = p[0], xi = p[1];
                p[0] = br * xr - bi * xi;
                p[1] = br * xi + bi * xr;
            }
        }
    }
}

// ----------------------------------------------------------- registration

template <int TPR, int NPT, int U, bool CPLX>
Variant make_tsmm() {
    Variant v;
    memset(&v, 0, sizeof(v));
    snprintf(v.info.name, sizeof(v.info.name), "tsmm_%s_smemc_tpr%d_npt%d_u%d", CPLX ? "c64" : "r64", TPR,
             NPT, U);
    v.info.kind = TSM_KIND_TSMM;
    v.info.dtype = CPLX ? TSM_C64 : TSM_R64;
    v.info.tile_n = NPT;
    v.info.threads_per_row = TPR;
    v.info.unroll = U;
    v.info.block = kBlock;
    v.tsmm = launch_tsmm<TPR, NPT, U, CPLX>;
    v.occupancy = occ_tsmm<TPR, NPT, U, CPLX>;
    return v;
}

template <bool CPLX>
void add_tsmttsm(std::vector<Variant>& t) {
    t.push_back(make_tsmttsm<1, 1, 4, CPLX>());
    t.push_back(make_tsmttsm<2, 2, 2, CPLX>());
    t.push_back(make_tsmttsm<2, 2, 4, CPLX>());
    t.push_back(make_tsmttsm<4, 4, 1, CPLX>());
    t.push_back(make_tsmttsm<4, 4, 2, CPLX>());
    t.push_back(make_tsmttsm<8, 4, 1, CPLX>());
    t.push_back(make_tsmttsm<4, 8, 1, CPLX>());
    if (!CPLX) t.push_back(make_tsmttsm<8, 8, 1, CPLX>());
}

template <bool CPLX>
void add_tsmm(std::vector<Variant>& t) {
    t.push_back(make_tsmm<1, 1, 4, CPLX>());
    t.push_back(make_tsmm<1, 2, 4, CPLX>());
    t.push_back(make_tsmm<1, 4, 2, CPLX>());
    t.push_back(make_tsmm<2, 1, 4, CPLX>());
    t.push_back(make_tsmm<2, 2, 4, CPLX>());
    t.push_back(make_tsmm<2, 4, 2, CPLX>());
    t.push_back(make_tsmm<4, 1, 4, CPLX>());
    t.push_back(make_tsmm<4, 2, 4, CPLX>());
    t.push_back(make_tsmm<4, 4, 2, CPLX>());
    t.push_back(make_tsmm<4, 8, 1, CPLX>());
    t.push_back(make_tsmm<4, 16, 1, CPLX>());
    t.push_back(make_tsmm<8, 1, 4, CPLX>());
    t.push_back(make_tsmm<8, 2, 2, CPLX>());
    t.push_back(make_tsmm<8, 4, 2, CPLX>());
    t.push_back(make_tsmm<8, 8, 1, CPLX>());
    t.push_back(make_tsmm<16, 1, 4, CPLX>());
    t.push_back(make_tsmm<16, 2, 2, CPLX>());
    t.push_back(make_tsmm<16, 4, 1, CPLX>());
    t.push_back(make_tsmm<16, 4, 2, CPLX>());
    t.push_back(make_tsmm<32, 1, 2, CPLX>());
    t.push_back(make_tsmm<32, 2, 1, CPLX>());
}

}  // namespace

void register_fp64_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm) {
    add_tsmttsm<false>(tsmttsm);
    add_tsmttsm<true>(tsmttsm);
    add_tsmm<false>(tsmm);
    add_tsmm<true>(tsmm);
}

namespace {

// Final pass of the TSMTTSM reduction: S consecutive lanes of a warp share
// entry o of C (S a power of two <= 32); lane s sums the CTA partials s,
// s + S, ... in order (eight interleaved running sums, combined by a fixed
// tree), the S slice sums are combined by a fixed shuffle tree, and the
// first lane stores alpha * sum + beta * C.  With S chosen so that each
// lane takes a few dozen partials, the pass is a handful of L2 round trips
// however many CTAs wrote partials.
template <int CC>
__global__ void __launch_bounds__(256) k_tsmttsm_final(const TsmttsmArgs a, int G, int S) {
    pdl_trigger();
    pdl_wait();  // the partials of the launch before
    const int MN = a.M * a.N;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int o = gt / S, s = gt - o * S;  // S divides 32: an entry's lanes share a warp
    double v[CC];
    if (o < MN) {
        sum_partials<CC>(a.ws, MN * CC, o, G, s, S, v);
    } else {
#pragma unroll
        for (int c = 0; c < CC; ++c) v[c] = 0.0;
    }
    for (int h = S >> 1; h >= 1; h >>= 1)
#pragma unroll
        for (int c = 0; c < CC; ++c) v[c] += __shfl_down_sync(0xffffffffu, v[c], h, S);
    if (o < MN && s == 0) tsmttsm_store_entry<CC>(a, o, v);
}

}  // namespace

cudaError_t launch_tsmttsm_final(const TsmttsmArgs& a, int grid, int cplx, cudaStream_t s) {
    const int MN = a.M * a.N;
    int S = 1;
    while (S < 32 && grid >= 16 * S) S *= 2;  // at least 8 partials per lane
    const int threads = MN * S;
    const int blocks = (threads + 255) / 256;
    if (cplx) return launch_pdl(k_tsmttsm_final<2>, blocks, 256, 0, s, a, grid, S);
    return launch_pdl(k_tsmttsm_final<1>, blocks, 256, 0, s, a, grid, S);
}

cudaError_t launch_scale_small(double* C, int rows, int cols, int64_t ld, int cplx, double br, double bi,
                               int beta_zero, cudaStream_t s) {
    const int64_t total = (int64_t)rows * cols;
    const int grid = (int)((total + 255) / 256);
    k_scale<<<grid > 0 ? grid : 1, 256, 0, s>>>(C, rows, cols, ld, cplx, br, bi, beta_zero);
    return cudaGetLastError();
}

cudaError_t launch_scale_tall(double* B, int64_t rows, int cols, int64_t ld, int cplx, double br, double bi,
                              int beta_zero, cudaStream_t s) {
    const int grid = device_info().sm_count * 8;
    k_scale<<<grid, 256, 0, s>>>(B, rows, cols, ld, cplx, br, bi, beta_zero);
    return cudaGetLastError();
}

}  // namespace tsm
