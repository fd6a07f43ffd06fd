// FP64 variants for the widths the power-of-two families of kernels_fp64.cu
// cover badly (the non-square shapes of the batched workload and of the full
// (M, N) grid).  A guarded tile entry or result slot past M or N still issues
// its FMAs (on zeros), and on GB300 the FP64 pipe (about 2 FMA/clk/SM) is the
// bound, so padding costs its full share of time.
//
// TSMTTSM (Sec. 3): more tile shapes of the register-tiled kernel
// (fp64_tsmttsm.cuh) -- 3x3, 3x5, 5x3, 5x2, 2x5, 2x7, 7x2, 5x5 -- picked
// greedily as those that most reduce the padded work summed over all
// M, N <= 64 (12.5 % -> 6.4 % over the existing tiles).
//
// TSMM (Sec. 4): t threads per row, any value from 1 to 64 (not only powers
// of two), each computing up to NPT interleaved results (Fig. 12); chosen per
// N at launch so that npt * t covers N with the least padding, e.g. N = 39
// as 13 threads x 3 results.  Its loop bound over the result slots is
// warp-uniform, so unused slots cost nothing.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fp64_common.cuh"
#include "fp64_tsmttsm.cuh"
#include "tsm_internal.h"

namespace tsm {

// Threads per row for TSMM with at most `nptmax` results per thread: the
// least padding npt * t - N, then the most results per thread (each A value
// loaded feeds more FMAs).
void rt_tsmm_tpr(int N, int nptmax, int* tpr_out, int* npt_out) {
    int bt = N, bn = 1, bw = 1 << 30;
    for (int npt = 1; npt <= nptmax; ++npt) {
        const int t = (N + npt - 1) / npt;
        if (t > 64) continue;
        const int waste = npt * t - N;
        if (waste < bw || (waste == bw && npt > bn)) {
            bw = waste;
            bt = t;
            bn = npt;
        }
    }
    *tpr_out = bt;
    *npt_out = bn;
}

namespace {

// --------------------------------------------------------------------- TSMM

template <int NPT, int U, bool CPLX, bool GEN>
__global__ void __launch_bounds__(kBlock) k_tsmm_rt(const TsmmArgs a, const int tpr) {
    constexpr int CC = CPLX ? 2 : 1;
    extern __shared__ double cs[];  // alpha * C, M x N (x CC)
    const int N = a.N, M = a.M;
    tsmm_begin(a);
    tsmm_stage_c<CC>(a, cs);

    const int rpc = kBlock / tpr;  // rows per CTA per unrolled step
    const int r = threadIdx.x / tpr, q = threadIdx.x - r * tpr;
    const bool live = r < rpc;     // threads past rpc * tpr hold no row
    const int npt = (N + tpr - 1) / tpr;
    const double* __restrict__ A = a.A;
    const int64_t sa = a.lda * CC, sb = a.ldb * CC;
    const int64_t step = (int64_t)gridDim.x * rpc * U;
    for (int64_t base = (int64_t)blockIdx.x * rpc * U; base < a.K; base += step) {
        int64_t row[U];
        bool rok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            row[u] = base + r + (int64_t)u * rpc;
            rok[u] = live && row[u] < a.K;
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
                    const int n = q + j * tpr;
                    if (rok[u] && n < N)
#pragma unroll
                        for (int c = 0; c < CC; ++c) ob[u][j][c] = a.B[row[u] * sb + n * CC + c];
                    tsmm_acc_init<CC, GEN>(a, ob[u][j][0], ob[u][j][CC - 1], acc[u][j][0], acc[u][j][CC - 1]);
                }
        }
        if (live) {
#pragma unroll 2
            for (int m = 0; m < M; ++m) {
                double av[U][CC];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < CC; ++c) av[u][c] = rok[u] ? __ldg(A + row[u] * sa + m * CC + c) : 0.0;
#pragma unroll
                for (int j = 0; j < NPT; ++j) {
                    if (j >= npt) break;  // warp-uniform
                    const int n = q + j * tpr;
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
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!rok[u]) continue;
            double* out = a.B + row[u] * sb;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                if (j >= npt) break;
                const int n = q + j * tpr;
                if (n >= N) continue;
                tsmm_store_plain<CC>(out, n, acc[u][j][0], acc[u][j][CC - 1]);
            }
        }
    }
}

template <int NPT, int U, bool CPLX, bool GEN>
cudaError_t launch_tsmm_rt_as(const TsmmArgs& a, int grid, cudaStream_t s) {
    int tpr = 1, npt = 1;
    rt_tsmm_tpr(a.N, NPT, &tpr, &npt);
    const size_t smem = (size_t)a.M * a.N * (CPLX ? 2 : 1) * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tsmm_rt<NPT, U, CPLX, GEN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(k_tsmm_rt<NPT, U, CPLX, GEN>, grid, kBlock, smem, s, a, tpr);
}

template <int NPT, int U, bool CPLX>
cudaError_t launch_tsmm_rt(const TsmmArgs& a, int grid, cudaStream_t s) {
    return tsmm_general_beta(a) ? launch_tsmm_rt_as<NPT, U, CPLX, true>(a, grid, s)
                                : launch_tsmm_rt_as<NPT, U, CPLX, false>(a, grid, s);
}

template <int NPT, int U, bool CPLX>
int occ_tsmm_rt(int M, int N) {
    const size_t smem = (size_t)M * N * (CPLX ? 2 : 1) * sizeof(double);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_tsmm_rt<NPT, U, CPLX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tsmm_rt<NPT, U, CPLX, false>, kBlock, smem) != cudaSuccess)
        return 0;
    return n;
}

// ----------------------------------------------------------- registration

template <int NPT, int U, bool CPLX>
Variant make_tsmm_rt() {
    Variant v;
    memset(&v, 0, sizeof(v));
    snprintf(v.info.name, sizeof(v.info.name), "tsmm_%s_rt_npt%d_u%d", CPLX ? "c64" : "r64", NPT, U);
    v.info.kind = TSM_KIND_TSMM;
    v.info.dtype = CPLX ? TSM_C64 : TSM_R64;
    v.info.tile_n = NPT;
    v.info.threads_per_row = 64;  // the largest; the launch picks the value
    v.info.unroll = U;
    v.info.block = kBlock;
    v.info.runtime_tile = 1;
    v.tsmm = launch_tsmm_rt<NPT, U, CPLX>;
    v.occupancy = occ_tsmm_rt<NPT, U, CPLX>;
    return v;
}

}  // namespace

void register_rt_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm) {
    for (int cplx = 0; cplx < 2; ++cplx) {
        const bool c = cplx != 0;
        tsmttsm.push_back(c ? make_tsmttsm<3, 3, 2, true>() : make_tsmttsm<3, 3, 2, false>());
        tsmttsm.push_back(c ? make_tsmttsm<3, 5, 1, true>() : make_tsmttsm<3, 5, 1, false>());
        tsmttsm.push_back(c ? make_tsmttsm<5, 3, 1, true>() : make_tsmttsm<5, 3, 1, false>());
        tsmttsm.push_back(c ? make_tsmttsm<5, 2, 2, true>() : make_tsmttsm<5, 2, 2, false>());
        tsmttsm.push_back(c ? make_tsmttsm<2, 5, 2, true>() : make_tsmttsm<2, 5, 2, false>());
        tsmttsm.push_back(c ? make_tsmttsm<2, 7, 1, true>() : make_tsmttsm<2, 7, 1, false>());
        tsmttsm.push_back(c ? make_tsmttsm<7, 2, 1, true>() : make_tsmttsm<7, 2, 1, false>());
        tsmttsm.push_back(c ? make_tsmttsm<5, 5, 1, true>() : make_tsmttsm<5, 5, 1, false>());
    }
    tsmm.push_back(make_tsmm_rt<4, 2, false>());
    tsmm.push_back(make_tsmm_rt<8, 1, false>());
    tsmm.push_back(make_tsmm_rt<2, 4, false>());
    tsmm.push_back(make_tsmm_rt<4, 2, true>());
    tsmm.push_back(make_tsmm_rt<2, 2, true>());
    tsmm.push_back(make_tsmm_rt<8, 1, true>());
}

}  // namespace tsm
