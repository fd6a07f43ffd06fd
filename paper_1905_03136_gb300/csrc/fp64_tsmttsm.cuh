// The register-tiled FP64 TSMTTSM kernel family (Sec. 3), shared by the
// translation units that instantiate its tile shapes.  P = ceil(M/T_M) *
// ceil(N/T_N) threads each own a T_M x T_N register tile of C (Listing 5) and
// L = 256 / P row lanes walk the CTA's contiguous row range with stride L, U
// rows per iteration (the loads of U rows are issued before their FMAs, the
// leap frogging of Sec. 3.1).  Tile entry (i, j) of thread (pm, pn) is
// C[pm + i*PM][pn + j*PN] (the transposed mapping of Fig. 10), and entries
// past M or N are guarded (Sec. 2.1).  The reduction is fp64_common.cuh's
// fixed-order scheme.
#pragma once

#include <cstdio>
#include <cstring>

#include "fp64_common.cuh"
#include "tsm_internal.h"

namespace tsm {
namespace {

// ------------------------------------------------------------------ TSMTTSM

template <int TM, int TN, int U, bool CPLX, bool CONJ>
__global__ void __launch_bounds__(kBlock) k_tsmttsm(const TsmttsmArgs a) {
    constexpr int CC = CPLX ? 2 : 1;
    tsmttsm_begin(a);
    const int M = a.M, N = a.N;
    const int PM = (M + TM - 1) / TM, PN = (N + TN - 1) / TN, P = PM * PN;
    const int L = kBlock / P;
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

    const int64_t G = gridDim.x;
    const int64_t k0 = a.K * (int64_t)blockIdx.x / G;
    const int64_t k1 = a.K * ((int64_t)blockIdx.x + 1) / G;
    const double* __restrict__ A = a.A;
    const double* __restrict__ B = a.B;
    const int64_t sa = a.lda * CC, sb = a.ldb * CC;

    if (active) {
        int64_t k = k0 + lane;
        for (; k + (int64_t)(U - 1) * L < k1; k += (int64_t)U * L) {
            double av[U][TM][CC], bv[U][TN][CC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double* ar = A + (k + (int64_t)u * L) * sa;
                const double* br = B + (k + (int64_t)u * L) * sb;
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int c = 0; c < CC; ++c) av[u][i][c] = mok[i] ? __ldg(ar + mi[i] * CC + c) : 0.0;
#pragma unroll
                for (int j = 0; j < TN; ++j)
#pragma unroll
                    for (int c = 0; c < CC; ++c) bv[u][j][c] = nok[j] ? __ldg(br + nj[j] * CC + c) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        if (!CPLX) {
                            acc[i][j][0] = fma(av[u][i][0], bv[u][j][0], acc[i][j][0]);
                        } else {
                            const double ar = av[u][i][0], ai = av[u][i][CC - 1];
                            const double br = bv[u][j][0], bi = bv[u][j][CC - 1];
                            acc[i][j][0] = fma(ar, br, acc[i][j][0]);
                            acc[i][j][0] = fma(CONJ ? ai : -ai, bi, acc[i][j][0]);
                            acc[i][j][CC - 1] = fma(ar, bi, acc[i][j][CC - 1]);
                            acc[i][j][CC - 1] = fma(CONJ ? -ai : ai, br, acc[i][j][CC - 1]);
                        }
                    }
        }
        for (; k < k1; k += L) {
            const double* ar = A + k * sa;
            const double* br = B + k * sb;
            double av[TM][CC], bv[TN][CC];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int c = 0; c < CC; ++c) av[i][c] = mok[i] ? __ldg(ar + mi[i] * CC + c) : 0.0;
#pragma unroll
            for (int j = 0; j < TN; ++j)
#pragma unroll
                for (int c = 0; c < CC; ++c) bv[j][c] = nok[j] ? __ldg(br + nj[j] * CC + c) : 0.0;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    if (!CPLX) {
                        acc[i][j][0] = fma(av[i][0], bv[j][0], acc[i][j][0]);
                    } else {
                        const double ar_ = av[i][0], ai = av[i][CC - 1];
                        const double br_ = bv[j][0], bi = bv[j][CC - 1];
                        acc[i][j][0] = fma(ar_, br_, acc[i][j][0]);
                        acc[i][j][0] = fma(CONJ ? ai : -ai, bi, acc[i][j][0]);
                        acc[i][j][CC - 1] = fma(ar_, bi, acc[i][j][CC - 1]);
                        acc[i][j][CC - 1] = fma(CONJ ? -ai : ai, br_, acc[i][j][CC - 1]);
                    }
                }
        }
    }

    tsmttsm_finish<TM, TN, CC>(a, &acc[0][0][0], PM, PN, L, lane, p, active);
}

template <int TM, int TN, int U, bool CPLX>
cudaError_t launch_tsmttsm(const TsmttsmArgs& a, int grid, cudaStream_t s) {
    if (CPLX && a.conj) return launch_pdl(k_tsmttsm<TM, TN, U, CPLX, true>, grid, kBlock, 0, s, a);
    return launch_pdl(k_tsmttsm<TM, TN, U, CPLX, false>, grid, kBlock, 0, s, a);
}

template <int TM, int TN, int U, bool CPLX>
int occ_tsmttsm(int M, int N) {
    const int P = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    if (P > kBlock) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tsmttsm<TM, TN, U, CPLX, false>, kBlock, 0) !=
        cudaSuccess)
        return 0;
    return n;
}


template <int TM, int TN, int U, bool CPLX>
Variant make_tsmttsm() {
    Variant v;
    memset(&v, 0, sizeof(v));
    snprintf(v.info.name, sizeof(v.info.name), "tsmttsm_%s_direct_t%dx%d_u%d", CPLX ? "c64" : "r64", TM, TN,
             U);
    v.info.kind = TSM_KIND_TSMTTSM;
    v.info.dtype = CPLX ? TSM_C64 : TSM_R64;
    v.info.tile_m = TM;
    v.info.tile_n = TN;
    v.info.unroll = U;
    v.info.block = kBlock;
    v.tsmttsm = launch_tsmttsm<TM, TN, U, CPLX>;
    v.occupancy = occ_tsmttsm<TM, TN, U, CPLX>;
    return v;
}

}  // namespace
}  // namespace tsm
