// Narrow-width FP64 kernels: TSMTTSM and TSMM for the shapes whose rows are
// only a few doubles wide (real M, N <= 4, complex M, N <= 2).
//
// At these widths the work per row is a handful of FMAs, so the products are
// bound by HBM bandwidth (real 1 x 1, Eq. 1 intensity 1/8 flop/B) or need
// about 5 TB/s of it while the FP64 pipe runs flat out (real 2 x 2, complex
// 1 x 1).  The paper's remedy for the narrow end is to give each thread more
// independent loads (Sec. 3.1, 5.3); here the rows are streamed as whole
// 16- or 32-byte vectors instead of 8-byte scalars:
//
//  - with lda == M and ldb == N (block vectors stored without padding, the
//    layout of Sec. 1.2) A and B are single contiguous arrays, so each thread
//    owns a GROUP of R consecutive rows whose A and B bytes are whole vectors
//    (R = the least row count making R*M*c and R*N*c multiples of the vector
//    width).  A warp's load instruction then covers 32 consecutive groups,
//    fully coalesced, and U groups per thread are loaded before any FMA
//    (leap frogging, Sec. 3.1, with U*(R*(M+N)*c*8) bytes in flight per
//    thread);
//  - any other leading dimension or an unaligned pointer takes the scalar
//    row loop of the same kernel (warp-uniform branch), so every layout is
//    served; only the speed differs;
//  - TSMTTSM: the group loop accumulates the M x N tile in registers; the
//    CTA sums its threads with a fixed butterfly of warp shuffles and then
//    the warps in warp order, and the last CTA sums all CTA partials in CTA
//    order (the deterministic replacement of Sec. 3.2's atomics, shared with
//    the other TSMTTSM kernels);
//  - TSMM: alpha*C (at most 16 doubles) lives in registers (Sec. 4.2 "data
//    from C": registers instead of shared memory) and each thread writes its
//    group of R output rows with vector stores.
// Two orders of the group loop.  Contiguous: CTA b of G takes groups
// [NG*b/G, NG*(b+1)/G), every CTA streaming the same bytes (+-1 group).
// Window: chunks of U blocks of 256 groups, CTA b taking chunks b, b + G,
// ..., so the grid moves through the arrays together (better DRAM page
// locality when reads and writes mix, as in TSMM, which always uses it).
#include <cstdio>
#include <cstring>

#include "fp64_common.cuh"
#include "tsm_internal.h"

namespace tsm {
namespace {

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// Rows per group so that R * w * CC doubles are a whole number of VW-double
// vectors for both widths.
template <int M, int N, int CC, int VW>
struct Group {
    static constexpr int R = lcm_c(VW / gcd_c(VW, M * CC), VW / gcd_c(VW, N * CC));
    static constexpr int EA = R * M * CC;  // doubles of A per group
    static constexpr int EB = R * N * CC;  // doubles of B per group
};

// Streaming loads of VW consecutive doubles (read-only data, used once: no L1
// allocation).  Not volatile, so the compiler may schedule them freely.
template <int VW>
__device__ __forceinline__ void ldv(const double* p, double* v);
template <>
__device__ __forceinline__ void ldv<2>(const double* p, double* v) {
    asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p));
}
template <>
__device__ __forceinline__ void ldv<4>(const double* p, double* v) {
    asm("ld.global.nc.L1::no_allocate.v4.f64 {%0, %1, %2, %3}, [%4];"
        : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
        : "l"(p));
}

template <int VW>
__device__ __forceinline__ void ldv_rw(const double* p, double* v);  // output B (beta != 0): coherent load
template <>
__device__ __forceinline__ void ldv_rw<2>(const double* p, double* v) {
    asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p) : "memory");
}
template <>
__device__ __forceinline__ void ldv_rw<4>(const double* p, double* v) {
    asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
}

template <int VW>
__device__ __forceinline__ void stv(double* p, const double* v);
template <>
__device__ __forceinline__ void stv<2>(double* p, const double* v) {
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v[0]), "d"(v[1]) : "memory");
}
template <>
__device__ __forceinline__ void stv<4>(double* p, const double* v) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]),
                 "d"(v[3])
                 : "memory");
}

// acc[(i*N + j)*CC + c] += op(a[i]) * b[j] over one row (a: M*CC, b: N*CC).
template <int M, int N, int CC, bool CONJ>
__device__ __forceinline__ void row_fma(const double* a, const double* b, double* acc) {
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double* c = acc + (i * N + j) * CC;
            if (CC == 1) {
                c[0] = fma(a[i], b[j], c[0]);
            } else {
                const double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * j], bi = b[2 * j + 1];
                c[0] = fma(ar, br, c[0]);
                c[0] = fma(CONJ ? ai : -ai, bi, c[0]);
                c[1] = fma(ar, bi, c[1]);
                c[1] = fma(CONJ ? -ai : ai, br, c[1]);
            }
        }
}

// --------------------------------------------------------------- TSMTTSM

template <int M, int N, int CC, bool CONJ, int VW, int U, bool PF, bool WIN>
__global__ void __launch_bounds__(kBlock) k_tsmttsm_narrow(const TsmttsmArgs a, int vec) {
    typedef Group<M, N, CC, VW> Gp;
    constexpr int R = Gp::R, EA = Gp::EA, EB = Gp::EB, MNC = M * N * CC;
    constexpr int VP = next_pow2(MNC);  // values per lane, padded for the warp reduction
    tsmttsm_begin(a);
    double acc[VP];
#pragma unroll
    for (int e = 0; e < VP; ++e) acc[e] = 0.0;
    const int t = threadIdx.x;
    const int64_t G = gridDim.x, b = blockIdx.x;

    if (vec && WIN) {
        // Window order: the NB whole blocks of 256 groups are cut into
        // G * T chunks of at most U blocks; CTA b takes chunks b, b + G,
        // ..., so at any moment the grid streams one window of consecutive
        // chunks (DRAM pages shared by neighbouring CTAs).  A chunk's block
        // count is CTA-uniform, so no warp diverges.
        const int64_t NG = a.K / R, NB = NG / kBlock;
        const int64_t T = (NB + G * U - 1) / (G * U), NC = G * T;
        auto load = [&](int64_t c, double (*av)[EA], double (*bv)[EB]) -> int {
            const int64_t blk0 = NB * c / NC;
            const int nb = (int)(NB * (c + 1) / NC - blk0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u >= nb) break;
                const int64_t g = (blk0 + u) * kBlock + t;
#pragma unroll
                for (int v = 0; v < EA / VW; ++v) ldv<VW>(a.A + g * EA + v * VW, &av[u][v * VW]);
#pragma unroll
                for (int v = 0; v < EB / VW; ++v) ldv<VW>(a.B + g * EB + v * VW, &bv[u][v * VW]);
            }
            return nb;
        };
        auto compute = [&](int nb, double (*av)[EA], double (*bv)[EB]) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u >= nb) break;
#pragma unroll
                for (int r = 0; r < R; ++r) row_fma<M, N, CC, CONJ>(&av[u][r * M * CC], &bv[u][r * N * CC], acc);
            }
        };
        if (PF) {
            int64_t c = b;
            if (c < NC) {
                double av[U][EA], bv[U][EB];
                int nb = load(c, av, bv);
                for (;;) {
                    const int64_t cn = c + G;
                    if (cn < NC) {
                        double an[U][EA], bn[U][EB];
                        const int nn = load(cn, an, bn);
                        compute(nb, av, bv);
#pragma unroll
                        for (int u = 0; u < U; ++u) {
#pragma unroll
                            for (int e = 0; e < EA; ++e) av[u][e] = an[u][e];
#pragma unroll
                            for (int e = 0; e < EB; ++e) bv[u][e] = bn[u][e];
                        }
                        nb = nn;
                        c = cn;
                    } else {
                        compute(nb, av, bv);
                        break;
                    }
                }
            }
        } else {
            for (int64_t c = b; c < NC; c += G) {
                double av[U][EA], bv[U][EB];
                const int nb = load(c, av, bv);
                compute(nb, av, bv);
            }
        }
        // the groups after the last whole block and the rows after the last
        // whole group
        if (b == G - 1) {
            for (int64_t g = NB * kBlock + t; g < NG; g += kBlock) {
                double av[EA], bv[EB];
#pragma unroll
                for (int v = 0; v < EA / VW; ++v) ldv<VW>(a.A + g * EA + v * VW, &av[v * VW]);
#pragma unroll
                for (int v = 0; v < EB / VW; ++v) ldv<VW>(a.B + g * EB + v * VW, &bv[v * VW]);
#pragma unroll
                for (int r = 0; r < R; ++r) row_fma<M, N, CC, CONJ>(&av[r * M * CC], &bv[r * N * CC], acc);
            }
            for (int64_t k = NG * R + t; k < a.K; k += kBlock) {
                double av[M * CC], bv[N * CC];
#pragma unroll
                for (int e = 0; e < M * CC; ++e) av[e] = __ldg(a.A + k * (M * CC) + e);
#pragma unroll
                for (int e = 0; e < N * CC; ++e) bv[e] = __ldg(a.B + k * (N * CC) + e);
                row_fma<M, N, CC, CONJ>(av, bv, acc);
            }
        }
    } else if (vec) {
        const int64_t NG = a.K / R;
        const int64_t g1 = NG * (b + 1) / G;
        int64_t g = NG * b / G + t;
        auto load = [&](int64_t g0, double (*av)[EA], double (*bv)[EB]) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double* pa = a.A + (g0 + (int64_t)u * kBlock) * EA;
                const double* pb = a.B + (g0 + (int64_t)u * kBlock) * EB;
#pragma unroll
                for (int v = 0; v < EA / VW; ++v) ldv<VW>(pa + v * VW, &av[u][v * VW]);
#pragma unroll
                for (int v = 0; v < EB / VW; ++v) ldv<VW>(pb + v * VW, &bv[u][v * VW]);
            }
        };
        auto compute = [&](double (*av)[EA], double (*bv)[EB]) {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) row_fma<M, N, CC, CONJ>(&av[u][r * M * CC], &bv[u][r * N * CC], acc);
        };
        const int64_t step = (int64_t)U * kBlock;
        if (PF) {
            // register double buffering: the loads of the next U groups are
            // in flight while the FMAs of the current ones run
            if (g + (int64_t)(U - 1) * kBlock < g1) {
                double av[U][EA], bv[U][EB];
                load(g, av, bv);
                for (;;) {
                    const int64_t gn = g + step;
                    if (gn + (int64_t)(U - 1) * kBlock < g1) {
                        double an[U][EA], bn[U][EB];
                        load(gn, an, bn);
                        compute(av, bv);
#pragma unroll
                        for (int u = 0; u < U; ++u) {
#pragma unroll
                            for (int e = 0; e < EA; ++e) av[u][e] = an[u][e];
#pragma unroll
                            for (int e = 0; e < EB; ++e) bv[u][e] = bn[u][e];
                        }
                        g = gn;
                    } else {
                        compute(av, bv);
                        g = gn;
                        break;
                    }
                }
            }
        } else {
            for (; g + (int64_t)(U - 1) * kBlock < g1; g += step) {
                double av[U][EA], bv[U][EB];
                load(g, av, bv);
                compute(av, bv);
            }
        }
        for (; g < g1; g += kBlock) {
            double av[EA], bv[EB];
#pragma unroll
            for (int v = 0; v < EA / VW; ++v) ldv<VW>(a.A + g * EA + v * VW, &av[v * VW]);
#pragma unroll
            for (int v = 0; v < EB / VW; ++v) ldv<VW>(a.B + g * EB + v * VW, &bv[v * VW]);
#pragma unroll
            for (int r = 0; r < R; ++r) row_fma<M, N, CC, CONJ>(&av[r * M * CC], &bv[r * N * CC], acc);
        }
        // the K - NG*R < R rows after the last whole group
        if (b == G - 1) {
            for (int64_t k = NG * R + t; k < a.K; k += kBlock) {
                double av[M * CC], bv[N * CC];
#pragma unroll
                for (int e = 0; e < M * CC; ++e) av[e] = __ldg(a.A + k * (M * CC) + e);
#pragma unroll
                for (int e = 0; e < N * CC; ++e) bv[e] = __ldg(a.B + k * (N * CC) + e);
                row_fma<M, N, CC, CONJ>(av, bv, acc);
            }
        }
    } else {
        // any leading dimension: one row per thread per step
        const int64_t k1 = a.K * (b + 1) / G;
        const int64_t sa = a.lda * CC, sb = a.ldb * CC;
        for (int64_t k = a.K * b / G + t; k < k1; k += kBlock) {
            double av[M * CC], bv[N * CC];
#pragma unroll
            for (int e = 0; e < M * CC; ++e) av[e] = __ldg(a.A + k * sa + e);
#pragma unroll
            for (int e = 0; e < N * CC; ++e) bv[e] = __ldg(a.B + k * sb + e);
            row_fma<M, N, CC, CONJ>(av, bv, acc);
        }
    }

    pdl_trigger();  // the main loop is done: the next launch may be scheduled

    // In-CTA reduction: recursive halving across the 32 lanes (about VP
    // adds per lane instead of 5 per value), then the 8 warp sums in warp
    // order.  Every pairing is fixed, so the CTA partial repeats bit for bit.
    __shared__ double red[kBlock * CC];
    const int lane = t & 31, warp = t >> 5;
    constexpr int L = log2_pow2(VP);
    warp_reduce_scatter<VP>(acc, lane);
    const int e = lane >> (5 - L);
    if ((lane & ((32 >> L) - 1)) == 0 && e < MNC) red[warp * MNC + e] = acc[0];
    __syncthreads();
    pdl_wait();  // the previous launch on the stream may still use the workspace
    if (t < MNC) {
        double s = red[t];
#pragma unroll
        for (int w = 1; w < kBlock / 32; ++w) s += red[w * MNC + t];
        a.ws[b * MNC + t] = s;
    }
    tsmttsm_cross_cta<CC>(a, red);
}

template <int M, int N, int CC, int VW>
bool narrow_vec_ok(const double* A, int64_t lda, const double* B, int64_t ldb) {
    return lda == M && ldb == N && ((uintptr_t)A % (VW * 8)) == 0 && ((uintptr_t)B % (VW * 8)) == 0;
}

template <int M, int N, int CC, int VW, int U, bool PF, bool WIN>
cudaError_t launch_tsmttsm_narrow(const TsmttsmArgs& a, int grid, cudaStream_t s) {
    if (a.M != M || a.N != N) return cudaErrorInvalidValue;
    const int vec = narrow_vec_ok<M, N, CC, VW>(a.A, a.lda, a.B, a.ldb) ? 1 : 0;
    if (CC == 2 && a.conj)
        return launch_pdl(k_tsmttsm_narrow<M, N, CC, true, VW, U, PF, WIN>, grid, kBlock, 0, s, a, vec);
    return launch_pdl(k_tsmttsm_narrow<M, N, CC, false, VW, U, PF, WIN>, grid, kBlock, 0, s, a, vec);
}

template <int M, int N, int CC, int VW, int U, bool PF, bool WIN>
int occ_tsmttsm_narrow(int, int) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tsmttsm_narrow<M, N, CC, false, VW, U, PF, WIN>,
                                                      kBlock, 0) != cudaSuccess)
        return 0;
    return n;
}

// ------------------------------------------------------------------ TSMM

template <int M, int N, int CC, int VW, int U, bool PF>
__global__ void __launch_bounds__(kBlock) k_tsmm_narrow(const TsmmArgs a, int vec) {
    typedef Group<M, N, CC, VW> Gp;
    constexpr int R = Gp::R, EA = Gp::EA, EB = Gp::EB;
    tsmm_begin(a);
    // alpha * C in registers
    double cr[M * N * CC];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const double* src = a.Cm + ((int64_t)m * a.ldc + n) * CC;
            if (CC == 1) {
                cr[m * N + n] = a.alpha_r * __ldg(src);
            } else {
                const double xr = __ldg(src), xi = __ldg(src + 1);
                cr[(m * N + n) * 2] = a.alpha_r * xr - a.alpha_i * xi;
                cr[(m * N + n) * 2 + 1] = a.alpha_r * xi + a.alpha_i * xr;
            }
        }
    const int t = threadIdx.x;
    const int64_t G = gridDim.x, b = blockIdx.x;
    const bool bz = a.beta_zero != 0;

    // out[n*CC + c] = sum_m in[m] * cr[m][n] (+ beta * old, which opens the
    // FMA chain: no extra FP64 operation for beta = 1)
    auto row_out = [&](const double* in, const double* old, double* out) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            double xr = 0.0, xi = 0.0;
            if (!bz) tsmm_acc_init_kept<CC>(a, old[n * CC], old[n * CC + CC - 1], xr, xi);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (CC == 1) {
                    xr = fma(in[m], cr[m * N + n], xr);
                } else {
                    const double ar = in[2 * m], ai = in[2 * m + 1];
                    const double c0 = cr[(m * N + n) * 2], c1 = cr[(m * N + n) * 2 + 1];
                    xr = fma(ar, c0, xr);
                    xr = fma(-ai, c1, xr);
                    xi = fma(ar, c1, xi);
                    xi = fma(ai, c0, xi);
                }
            }
            if (CC == 1) {
                out[n] = xr;
            } else {
                out[2 * n] = xr;
                out[2 * n + 1] = xi;
            }
        }
    };

    if (vec) {
        // Window order (as in the TSMTTSM kernel): G * T chunks of at most U
        // blocks of 256 groups, CTA b taking chunks b, b + G, ...; reads and
        // writes of the whole grid then move through one window of the
        // arrays, which keeps DRAM pages open for both directions (separate
        // per-CTA ranges interleave 2 G streams in the banks).
        const int64_t NG = a.K / R, NB = NG / kBlock;
        const int64_t T = (NB + G * U - 1) / (G * U), NC = G * T;
        auto load = [&](int64_t c, double (*av)[EA], double (*bo)[EB], int64_t* blk) -> int {
            const int64_t blk0 = NB * c / NC;
            const int nb = (int)(NB * (c + 1) / NC - blk0);
            *blk = blk0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u >= nb) break;
                const int64_t g = (blk0 + u) * kBlock + t;
#pragma unroll
                for (int v = 0; v < EA / VW; ++v) ldv<VW>(a.A + g * EA + v * VW, &av[u][v * VW]);
            }
            if (!bz) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (u >= nb) break;
                    const int64_t g = (blk0 + u) * kBlock + t;
#pragma unroll
                    for (int v = 0; v < EB / VW; ++v) ldv_rw<VW>(a.B + g * EB + v * VW, &bo[u][v * VW]);
                }
            }
            return nb;
        };
        auto compute_store = [&](int64_t blk0, int nb, double (*av)[EA], double (*bo)[EB]) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u >= nb) break;
                double out[EB];
#pragma unroll
                for (int r = 0; r < R; ++r) row_out(&av[u][r * M * CC], &bo[u][r * N * CC], &out[r * N * CC]);
                double* pb = a.B + ((blk0 + u) * kBlock + t) * EB;
#pragma unroll
                for (int v = 0; v < EB / VW; ++v) stv<VW>(pb + v * VW, &out[v * VW]);
            }
        };
        if (PF) {
            // the next chunk's loads are in flight while the current chunk
            // is computed and stored (register double buffer)
            int64_t c = b;
            if (c < NC) {
                double av[U][EA], bo[U][EB];
                int64_t blk;
                int nb = load(c, av, bo, &blk);
                for (;;) {
                    const int64_t cn = c + G;
                    if (cn < NC) {
                        double an[U][EA], bn[U][EB];
                        int64_t blkn;
                        const int nn = load(cn, an, bn, &blkn);
                        compute_store(blk, nb, av, bo);
#pragma unroll
                        for (int u = 0; u < U; ++u) {
#pragma unroll
                            for (int e = 0; e < EA; ++e) av[u][e] = an[u][e];
#pragma unroll
                            for (int e = 0; e < EB; ++e) bo[u][e] = bn[u][e];
                        }
                        nb = nn;
                        blk = blkn;
                        c = cn;
                    } else {
                        compute_store(blk, nb, av, bo);
                        break;
                    }
                }
            }
        } else {
            for (int64_t c = b; c < NC; c += G) {
                double av[U][EA], bo[U][EB];
                int64_t blk;
                const int nb = load(c, av, bo, &blk);
                compute_store(blk, nb, av, bo);
            }
        }
        // groups after the last whole block, rows after the last whole group
        if (b == G - 1) {
            for (int64_t g = NB * kBlock + t; g < NG; g += kBlock) {
                double av[EA], bo[EB], out[EB];
#pragma unroll
                for (int v = 0; v < EA / VW; ++v) ldv<VW>(a.A + g * EA + v * VW, &av[v * VW]);
                if (!bz) {
#pragma unroll
                    for (int v = 0; v < EB / VW; ++v) ldv_rw<VW>(a.B + g * EB + v * VW, &bo[v * VW]);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) row_out(&av[r * M * CC], &bo[r * N * CC], &out[r * N * CC]);
#pragma unroll
                for (int v = 0; v < EB / VW; ++v) stv<VW>(a.B + g * EB + v * VW, &out[v * VW]);
            }
            for (int64_t k = NG * R + t; k < a.K; k += kBlock) {
                double av[M * CC], bo[N * CC], out[N * CC];
#pragma unroll
                for (int e = 0; e < M * CC; ++e) av[e] = __ldg(a.A + k * (M * CC) + e);
                if (!bz) {
#pragma unroll
                    for (int e = 0; e < N * CC; ++e) bo[e] = a.B[k * (N * CC) + e];
                }
                row_out(av, bo, out);
#pragma unroll
                for (int e = 0; e < N * CC; ++e) a.B[k * (N * CC) + e] = out[e];
            }
        }
    } else {
        const int64_t k1 = a.K * (b + 1) / G;
        const int64_t sa = a.lda * CC, sb = a.ldb * CC;
        for (int64_t k = a.K * b / G + t; k < k1; k += kBlock) {
            double av[M * CC], bo[N * CC], out[N * CC];
#pragma unroll
            for (int e = 0; e < M * CC; ++e) av[e] = __ldg(a.A + k * sa + e);
            if (!bz) {
#pragma unroll
                for (int e = 0; e < N * CC; ++e) bo[e] = a.B[k * sb + e];
            }
            row_out(av, bo, out);
#pragma unroll
            for (int e = 0; e < N * CC; ++e) a.B[k * sb + e] = out[e];
        }
    }
}

template <int M, int N, int CC, int VW, int U, bool PF>
cudaError_t launch_tsmm_narrow(const TsmmArgs& a, int grid, cudaStream_t s) {
    if (a.M != M || a.N != N) return cudaErrorInvalidValue;
    const int vec = narrow_vec_ok<M, N, CC, VW>(a.A, a.lda, a.B, a.ldb) ? 1 : 0;
    return launch_pdl(k_tsmm_narrow<M, N, CC, VW, U, PF>, grid, kBlock, 0, s, a, vec);
}

template <int M, int N, int CC, int VW, int U, bool PF>
int occ_tsmm_narrow(int, int) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tsmm_narrow<M, N, CC, VW, U, PF>, kBlock, 0) !=
        cudaSuccess)
        return 0;
    return n;
}

// ----------------------------------------------------------- registration

template <int M, int N, int CC, int VW, int U, bool PF, bool WIN>
Variant make_tsmttsm_narrow() {
    Variant v;
    memset(&v, 0, sizeof(v));
    snprintf(v.info.name, sizeof(v.info.name), "tsmttsm_%s_narrow_m%dn%d_v%d_u%d%s%s", CC == 2 ? "c64" : "r64",
             M, N, VW, U, PF ? "_pf" : "", WIN ? "_win" : "");
    v.info.kind = TSM_KIND_TSMTTSM;
    v.info.dtype = CC == 2 ? TSM_C64 : TSM_R64;
    v.info.fixed_m = M;
    v.info.fixed_n = N;
    v.info.tile_m = M;
    v.info.tile_n = N;
    v.info.unroll = U;
    v.info.block = kBlock;
    v.tsmttsm = launch_tsmttsm_narrow<M, N, CC, VW, U, PF, WIN>;
    v.occupancy = occ_tsmttsm_narrow<M, N, CC, VW, U, PF, WIN>;
    return v;
}

template <int M, int N, int CC, int VW, int U, bool PF>
Variant make_tsmm_narrow() {
    Variant v;
    memset(&v, 0, sizeof(v));
    snprintf(v.info.name, sizeof(v.info.name), "tsmm_%s_narrow_m%dn%d_v%d_u%d%s", CC == 2 ? "c64" : "r64", M, N,
             VW, U, PF ? "_pf" : "");
    v.info.kind = TSM_KIND_TSMM;
    v.info.dtype = CC == 2 ? TSM_C64 : TSM_R64;
    v.info.fixed_m = M;
    v.info.fixed_n = N;
    v.info.tile_n = N;
    v.info.threads_per_row = 1;
    v.info.unroll = U;
    v.info.block = kBlock;
    v.tsmm = launch_tsmm_narrow<M, N, CC, VW, U, PF>;
    v.occupancy = occ_tsmm_narrow<M, N, CC, VW, U, PF>;
    return v;
}

// Variants per product and shape: 16-byte vectors with four groups in
// flight, 32-byte vectors with two and with four, and vectors with the next
// groups prefetched into a second register buffer ("_pf"); TSMTTSM also in
// window order ("_win"; TSMM always streams in window order).  TSMM
// holds its output group beside the loaded one, so wide groups (real 3 x 3:
// 12 doubles each) take a smaller unroll (MU) to stay clear of spills.
template <int M, int N, int CC, int MU>
void add_shape(std::vector<Variant>& t, std::vector<Variant>& m) {
    t.push_back(make_tsmttsm_narrow<M, N, CC, 2, 4, false, false>());
    t.push_back(make_tsmttsm_narrow<M, N, CC, 4, 2, false, false>());
    t.push_back(make_tsmttsm_narrow<M, N, CC, 4, 4, false, false>());
    t.push_back(make_tsmttsm_narrow<M, N, CC, 4, 1, true, false>());
    t.push_back(make_tsmttsm_narrow<M, N, CC, 4, 2, true, false>());
    t.push_back(make_tsmttsm_narrow<M, N, CC, 4, 1, true, true>());
    t.push_back(make_tsmttsm_narrow<M, N, CC, 4, 2, true, true>());
    m.push_back(make_tsmm_narrow<M, N, CC, 2, MU, false>());
    m.push_back(make_tsmm_narrow<M, N, CC, 4, (MU > 2 ? MU / 2 : 1), false>());
    m.push_back(make_tsmm_narrow<M, N, CC, 4, MU, false>());
    m.push_back(make_tsmm_narrow<M, N, CC, 4, 1, true>());
    m.push_back(make_tsmm_narrow<M, N, CC, 2, MU / 2, true>());
}

}  // namespace

void register_narrow_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm) {
    add_shape<1, 1, 1, 4>(tsmttsm, tsmm);
    add_shape<2, 2, 1, 4>(tsmttsm, tsmm);
    add_shape<3, 3, 1, 2>(tsmttsm, tsmm);
    add_shape<4, 4, 1, 4>(tsmttsm, tsmm);
    add_shape<1, 1, 2, 4>(tsmttsm, tsmm);
    add_shape<2, 2, 2, 4>(tsmttsm, tsmm);
}

}  // namespace tsm
