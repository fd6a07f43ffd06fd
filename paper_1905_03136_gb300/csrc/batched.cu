// Batched persistent launch: many uneven TSMTTSM / TSMM instances in one
// kernel, captured in a CUDA graph (see tsm_batched.h).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fp64_common.cuh"
#include "tsm_batched.h"
#include "tsm_internal.h"

namespace tsm {
tsm_status validate_common(int dtype, int M, int N, int64_t K, const double* alpha, const double* beta);

namespace batched {

struct Inst {
    int kind, cplx, conj, M, N, code, beta_zero, n_items;
    int tpr;           // TSMM code 4: threads per row (any value 1..64)
    int64_t K, lda, ldb, ldo;
    const double* A;
    const double* B;
    double* out;
    double ar, ai, br, bi;
    int64_t part_off;  // doubles: first partial slot of this instance (TSMTTSM)
};

struct Item {
    int inst, idx;
    int64_t r0, r1;
};

constexpr int kThreads = 256;
// Work items per persistent CTA the default split aims at.  Items of a few
// hundred milliseconds (4 per CTA) left SMs idle behind the last large items;
// 16 per CTA brought the 256-instance mixed batch from 1380 to 1232 ms.
constexpr double kItemsPerCta = 16.0;

// ----------------------------------------------------------- TSMTTSM item

// One row's rank-1 update of the register tile (complex: op T or C on A).
template <int TM, int TN, bool CPLX, bool CONJ>
__device__ __forceinline__ void item_fma(double (&acc)[TM][TN][CPLX ? 2 : 1], const double (&av)[TM][CPLX ? 2 : 1],
                                         const double (&bv)[TN][CPLX ? 2 : 1]) {
    constexpr int CC = CPLX ? 2 : 1;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            if (!CPLX) {
                acc[i][j][0] = fma(av[i][0], bv[j][0], acc[i][j][0]);
            } else {
                const double ar = av[i][0], ai = av[i][CC - 1];
                const double br = bv[j][0], bi = bv[j][CC - 1];
                acc[i][j][0] = fma(ar, br, acc[i][j][0]);
                acc[i][j][0] = fma(CONJ ? ai : -ai, bi, acc[i][j][0]);
                acc[i][j][CC - 1] = fma(ar, bi, acc[i][j][CC - 1]);
                acc[i][j][CC - 1] = fma(CONJ ? -ai : ai, br, acc[i][j][CC - 1]);
            }
        }
}

template <int TM, int TN, int U, bool CPLX, bool CONJ>
__device__ __noinline__ void tsmttsm_item(const Inst* __restrict__ ip, const Item it, double* parts,
                                          unsigned* tickets, double* red) {
    const Inst in = *ip;
    constexpr int CC = CPLX ? 2 : 1;
    __shared__ unsigned s_last;
    const int M = in.M, N = in.N;
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
    const int64_t sa = in.lda * CC, sb = in.ldb * CC;
    if (active) {
        // unguarded main loop over whole groups of U rows, then single rows
        int64_t k = it.r0 + lane;
        for (; k + (int64_t)(U - 1) * L < it.r1; k += (int64_t)L * U) {
            double av[U][TM][CC], bv[U][TN][CC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double* ar = in.A + (k + (int64_t)u * L) * sa;
                const double* br = in.B + (k + (int64_t)u * L) * sb;
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
            for (int u = 0; u < U; ++u) item_fma<TM, TN, CPLX, CONJ>(acc, av[u], bv[u]);
        }
        for (; k < it.r1; k += L) {
            const double* ar = in.A + k * sa;
            const double* br = in.B + k * sb;
            double av[TM][CC], bv[TN][CC];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int c = 0; c < CC; ++c) av[i][c] = mok[i] ? __ldg(ar + mi[i] * CC + c) : 0.0;
#pragma unroll
            for (int j = 0; j < TN; ++j)
#pragma unroll
                for (int c = 0; c < CC; ++c) bv[j][c] = nok[j] ? __ldg(br + nj[j] * CC + c) : 0.0;
            item_fma<TM, TN, CPLX, CONJ>(acc, av, bv);
        }
    }
    // lanes: fixed-pairing tree per tile entry, into this item's slot
    const int MNc = M * N * CC;
    double* part = parts + in.part_off + (int64_t)it.idx * MNc;
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
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = (atomicAdd(&tickets[it.inst], 1u) == (unsigned)in.n_items - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double* slots = parts + in.part_off;
    const int MN = M * N, G = in.n_items;
    int S = 1;
    while (S * 2 * MN <= kThreads && S * 2 <= G) S *= 2;
    for (int base = 0; base < MN * S; base += kThreads) {
        const int w = base + t;
        const bool mine = w < MN * S;
        double v[CC];
        if (mine) sum_partials<CC>(slots, MNc, w / S, G, w % S, S, v);
        if (S > 1) {
            // fixed pairwise tree over the S slice sums of one entry (a
            // serial chain would cost S - 1 FP64 issue slots in a row)
#pragma unroll
            for (int c = 0; c < CC; ++c) red[t * CC + c] = mine ? v[c] : 0.0;
            __syncthreads();
            for (int h = S >> 1; h >= 1; h >>= 1) {
                if (mine && (w % S) < h)
#pragma unroll
                    for (int c = 0; c < CC; ++c) red[t * CC + c] += red[(t + h) * CC + c];
                __syncthreads();
            }
#pragma unroll
            for (int c = 0; c < CC; ++c) v[c] = red[t * CC + c];
            __syncthreads();
        }
        if (!mine || (w % S) != 0) continue;
        const int o = w / S, m = o / N, n = o - m * N;
        double* out = in.out + ((int64_t)m * in.ldo + n) * CC;
        if (!CPLX) {
            double r = in.ar * v[0];
            if (!in.beta_zero) r = fma(in.br, out[0], r);
            out[0] = r;
        } else {
            double rr = in.ar * v[0] - in.ai * v[CC - 1];
            double ri = in.ar * v[CC - 1] + in.ai * v[0];
            if (!in.beta_zero) {
                const double orr = out[0], oi = out[CC - 1];
                rr += in.br * orr - in.bi * oi;
                ri += in.br * oi + in.bi * orr;
            }
            out[0] = rr;
            out[CC - 1] = ri;
        }
    }
    __syncthreads();
    if (t == 0) tickets[it.inst] = 0u;
}

// -------------------------------------------------------------- TSMM item

template <int TPR, int NPT, bool CPLX>
__device__ __noinline__ void tsmm_item(const Inst* __restrict__ ip, const Item it, double* cs) {
    const Inst in = *ip;
    constexpr int CC = CPLX ? 2 : 1;
    constexpr int RPC = kThreads / TPR;
    constexpr int U = 2;
    const int M = in.M, N = in.N;
    for (int o = threadIdx.x; o < M * N; o += kThreads) {
        const int m = o / N, n = o - m * N;
        const double* src = in.B + ((int64_t)m * in.ldb + n) * CC;
        if (!CPLX) {
            cs[o] = in.ar * src[0];
        } else {
            const double cr = src[0], ci = src[CC - 1];
            cs[o * CC] = in.ar * cr - in.ai * ci;
            cs[o * CC + CC - 1] = in.ar * ci + in.ai * cr;
        }
    }
    __syncthreads();
    const int r = threadIdx.x / TPR, q = threadIdx.x - r * TPR;
    const int npt = (N + TPR - 1) / TPR;  // result slots in use, <= NPT
    const int64_t sa = in.lda * CC, sb = in.ldo * CC;
    for (int64_t base = it.r0; base < it.r1; base += (int64_t)RPC * U) {
        int64_t row[U];
        bool rok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            row[u] = base + r + (int64_t)u * RPC;
            rok[u] = row[u] < it.r1;
            if (!rok[u]) row[u] = it.r0;
        }
        double acc[U][NPT][CC];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < NPT; ++j)
#pragma unroll
                for (int c = 0; c < CC; ++c) acc[u][j][c] = 0.0;
        // four columns of A per pass, their loads issued before the FMAs, so
        // each thread keeps 4 * U independent loads in flight
        for (int m0 = 0; m0 < M; m0 += 4) {
            double av[4][U][CC];
#pragma unroll
            for (int mm = 0; mm < 4; ++mm)
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < CC; ++c)
                        av[mm][u][c] = (rok[u] && m0 + mm < M) ? __ldg(in.A + row[u] * sa + (m0 + mm) * CC + c) : 0.0;
#pragma unroll
            for (int mm = 0; mm < 4; ++mm) {
                const int m = m0 + mm;
                if (m >= M) break;
#pragma unroll
                for (int j = 0; j < NPT; ++j) {
                    // CTA-uniform bound: result slots no thread needs are
                    // branched around (predicated-off FMAs still occupy the
                    // FP64 pipe); only the last, ragged slot is guarded
                    if (j >= npt) break;
                    const int n = q + j * TPR;
                    if (n < N) {
                        const double cr = cs[(m * N + n) * CC], ci = cs[(m * N + n) * CC + CC - 1];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (!CPLX) {
                                acc[u][j][0] = fma(av[mm][u][0], cr, acc[u][j][0]);
                            } else {
                                acc[u][j][0] = fma(av[mm][u][0], cr, acc[u][j][0]);
                                acc[u][j][0] = fma(-av[mm][u][CC - 1], ci, acc[u][j][0]);
                                acc[u][j][CC - 1] = fma(av[mm][u][0], ci, acc[u][j][CC - 1]);
                                acc[u][j][CC - 1] = fma(av[mm][u][CC - 1], cr, acc[u][j][CC - 1]);
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!rok[u]) continue;
            double* out = in.out + row[u] * sb;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                if (j >= npt) break;
                const int n = q + j * TPR;
                if (n >= N) continue;
                double vr = acc[u][j][0], vi = acc[u][j][CC - 1];
                if (!CPLX) {
                    if (!in.beta_zero) vr = fma(in.br, out[n], vr);
                    out[n] = vr;
                } else {
                    if (!in.beta_zero) {
                        const double orr = out[n * 2], oi = out[n * 2 + 1];
                        vr += in.br * orr - in.bi * oi;
                        vi += in.br * oi + in.bi * orr;
                    }
                    out[n * 2] = vr;
                    out[n * 2 + 1] = vi;
                }
            }
        }
    }
    __syncthreads();  // cs is reused by the next item
}

// TSMM item with any number of threads per row (in.tpr) and up to NPT
// results each: npt * tpr covers N with the least padding, and the loop over
// result slots has a warp-uniform bound, so no FMA is spent on padding.
template <int NPT, bool CPLX>
__device__ __noinline__ void tsmm_item_rt(const Inst* __restrict__ ip, const Item it, double* cs) {
    const Inst in = *ip;
    constexpr int CC = CPLX ? 2 : 1;
    constexpr int U = 2;
    const int M = in.M, N = in.N, tpr = in.tpr;
    for (int o = threadIdx.x; o < M * N; o += kThreads) {
        const int m = o / N, n = o - m * N;
        const double* src = in.B + ((int64_t)m * in.ldb + n) * CC;
        if (!CPLX) {
            cs[o] = in.ar * src[0];
        } else {
            const double cr = src[0], ci = src[CC - 1];
            cs[o * CC] = in.ar * cr - in.ai * ci;
            cs[o * CC + CC - 1] = in.ar * ci + in.ai * cr;
        }
    }
    __syncthreads();
    const int rpc = kThreads / tpr;
    const int r = threadIdx.x / tpr, q = threadIdx.x - r * tpr;
    const bool live = r < rpc;
    const int npt = (N + tpr - 1) / tpr;
    const int64_t sa = in.lda * CC, sb = in.ldo * CC;
    for (int64_t base = it.r0; base < it.r1; base += (int64_t)rpc * U) {
        int64_t row[U];
        bool rok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            row[u] = base + r + (int64_t)u * rpc;
            rok[u] = live && row[u] < it.r1;
            if (!rok[u]) row[u] = it.r0;
        }
        double acc[U][NPT][CC];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < NPT; ++j)
#pragma unroll
                for (int c = 0; c < CC; ++c) acc[u][j][c] = 0.0;
        if (live) {
            for (int m0 = 0; m0 < M; m0 += 4) {
                double av[4][U][CC];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm)
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int c = 0; c < CC; ++c)
                            av[mm][u][c] = (rok[u] && m0 + mm < M) ? __ldg(in.A + row[u] * sa + (m0 + mm) * CC + c) : 0.0;
#pragma unroll
                for (int mm = 0; mm < 4; ++mm) {
                    const int m = m0 + mm;
                    if (m >= M) break;
#pragma unroll
                    for (int j = 0; j < NPT; ++j) {
                        if (j >= npt) break;
                        const int n = q + j * tpr;
                        if (n < N) {
                            const double cr = cs[(m * N + n) * CC], ci = cs[(m * N + n) * CC + CC - 1];
#pragma unroll
                            for (int u = 0; u < U; ++u) {
                                if (!CPLX) {
                                    acc[u][j][0] = fma(av[mm][u][0], cr, acc[u][j][0]);
                                } else {
                                    acc[u][j][0] = fma(av[mm][u][0], cr, acc[u][j][0]);
                                    acc[u][j][0] = fma(-av[mm][u][CC - 1], ci, acc[u][j][0]);
                                    acc[u][j][CC - 1] = fma(av[mm][u][0], ci, acc[u][j][CC - 1]);
                                    acc[u][j][CC - 1] = fma(av[mm][u][CC - 1], cr, acc[u][j][CC - 1]);
                                }
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!rok[u]) continue;
            double* out = in.out + row[u] * sb;
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
                if (j >= npt) break;
                const int n = q + j * tpr;
                if (n >= N) continue;
                double vr = acc[u][j][0], vi = acc[u][j][CC - 1];
                if (!CPLX) {
                    if (!in.beta_zero) vr = fma(in.br, out[n], vr);
                    out[n] = vr;
                } else {
                    if (!in.beta_zero) {
                        const double orr = out[n * 2], oi = out[n * 2 + 1];
                        vr += in.br * orr - in.bi * oi;
                        vi += in.br * oi + in.bi * orr;
                    }
                    out[n * 2] = vr;
                    out[n * 2 + 1] = vi;
                }
            }
        }
    }
    __syncthreads();  // cs is reused by the next item
}

// -------------------------------------------------------- persistent kernel

// Accumulators stay at <= 32 doubles per thread for complex data (codes 4,
// 5 and 13 run as 4x4, code 14 as 3x3, and there is no 4-threads-per-row
// TSMM) and at <= 64 for real data (the 8x8 tile of code 13).
template <bool CPLX, bool CONJ>
__device__ void run_tsmttsm(const Inst* in, const Item& it, double* parts, unsigned* tickets, double* red) {
    switch (in->code) {
        case 1: tsmttsm_item<1, 1, 4, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 2: tsmttsm_item<2, 2, 2, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 4:
            if (!CPLX) {
                tsmttsm_item<4, 8, 1, CPLX, CONJ>(in, it, parts, tickets, red);
                break;
            }
            tsmttsm_item<4, 4, 1, CPLX, CONJ>(in, it, parts, tickets, red);
            break;
        case 5:
            if (!CPLX) {
                tsmttsm_item<8, 4, 1, CPLX, CONJ>(in, it, parts, tickets, red);
                break;
            }
            tsmttsm_item<4, 4, 1, CPLX, CONJ>(in, it, parts, tickets, red);
            break;
        case 6: tsmttsm_item<3, 3, 2, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 7: tsmttsm_item<2, 5, 2, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 8: tsmttsm_item<5, 2, 2, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 9: tsmttsm_item<3, 5, 1, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 10: tsmttsm_item<5, 3, 1, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 11: tsmttsm_item<2, 7, 1, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 12: tsmttsm_item<7, 2, 1, CPLX, CONJ>(in, it, parts, tickets, red); break;
        case 13:
            if (!CPLX) {
                tsmttsm_item<8, 8, 1, CPLX, CONJ>(in, it, parts, tickets, red);
                break;
            }
            tsmttsm_item<4, 4, 1, CPLX, CONJ>(in, it, parts, tickets, red);
            break;
        case 14:
            if (!CPLX) {
                tsmttsm_item<5, 5, 1, CPLX, CONJ>(in, it, parts, tickets, red);
                break;
            }
            tsmttsm_item<3, 3, 2, CPLX, CONJ>(in, it, parts, tickets, red);
            break;
        default: tsmttsm_item<4, 4, 1, CPLX, CONJ>(in, it, parts, tickets, red); break;
    }
}

template <bool CPLX>
__device__ void run_tsmm(const Inst* in, const Item& it, double* cs) {
    switch (in->code) {
        case 1:
            if (!CPLX) {
                tsmm_item<4, 16, CPLX>(in, it, cs);
                break;
            }
            tsmm_item<8, 8, CPLX>(in, it, cs);
            break;
        case 3: tsmm_item<16, 4, CPLX>(in, it, cs); break;
        case 4: tsmm_item_rt<4, CPLX>(in, it, cs); break;
        default: tsmm_item<8, 8, CPLX>(in, it, cs); break;
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_batched(const Inst* __restrict__ insts,
                                                      const Item* __restrict__ items, int n_items,
                                                      unsigned* counter, unsigned* tickets, double* parts) {
    extern __shared__ double dyn[];
    __shared__ int s_item;
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int w = s_item;
        __syncthreads();
        if (w >= n_items) break;
        const Item it = items[w];
        const Inst* in = insts + it.inst;
        if (in->kind == TSM_KIND_TSMTTSM) {
            if (!in->cplx)
                run_tsmttsm<false, false>(in, it, parts, tickets, dyn);
            else if (in->conj)
                run_tsmttsm<true, true>(in, it, parts, tickets, dyn);
            else
                run_tsmttsm<true, false>(in, it, parts, tickets, dyn);
        } else {
            if (!in->cplx)
                run_tsmm<false>(in, it, dyn);
            else
                run_tsmm<true>(in, it, dyn);
        }
    }
}

// TSMTTSM tiles by code and the default choice: the least FP64 issue work
// per useful product -- tile padding past M and N times the idle lanes of
// partly filled warps, ceil(P*L/32)*32 * TM*TN / (L*M*N) with P threads per
// lane and L = 256/P lanes -- then the larger tile.  (Complex data runs
// codes 4, 5 and 13 with a 4x4 tile and code 14 with a 3x3 one.)
constexpr int kTileCodes = 14;
const int kTile[kTileCodes + 1][2] = {{0, 0}, {1, 1}, {2, 2}, {4, 4}, {4, 8}, {8, 4}, {3, 3}, {2, 5},
                                      {5, 2}, {3, 5}, {5, 3}, {2, 7}, {7, 2}, {8, 8}, {5, 5}};

// The tile a code runs with (complex data: codes 4, 5, 13 as 4x4, 14 as 3x3).
void code_tile(int code, int cplx, int* tm, int* tn) {
    *tm = kTile[code][0];
    *tn = kTile[code][1];
    if (cplx && (code == 4 || code == 5 || code == 13)) *tm = *tn = 4;
    if (cplx && code == 14) *tm = *tn = 3;
}

bool tile_ok(int code, int M, int N, int cplx) {
    if (code < 1 || code > kTileCodes) return false;
    int tm, tn;
    code_tile(code, cplx, &tm, &tn);
    return ((M + tm - 1) / tm) * ((N + tn - 1) / tn) <= kThreads;
}

int default_tile(int M, int N, int cplx) {
    int best = 3;
    double bw = 1e30;
    int ba = 0;
    for (int c = 1; c <= kTileCodes; ++c) {
        if (!tile_ok(c, M, N, cplx)) continue;
        if (cplx && (c == 4 || c == 5 || c == 13 || c == 14)) continue;  // same as codes 3 and 6
        const int tm = kTile[c][0], tn = kTile[c][1];
        const int P = ((M + tm - 1) / tm) * ((N + tn - 1) / tn), L = kThreads / P;
        const double waste = (double)((P * L + 31) / 32 * 32) * tm * tn / ((double)L * M * N);
        if (waste < bw - 1e-9 || (waste < bw + 1e-9 && tm * tn > ba)) {
            best = c;
            bw = waste;
            ba = tm * tn;
        }
    }
    return best;
}

}  // namespace batched
}  // namespace tsm

struct tsm_batch {
    int n_items, n_inst, ctas;
    size_t smem;
    tsm::batched::Inst* d_inst;
    tsm::batched::Item* d_items;
    unsigned* d_counter;
    unsigned* d_tickets;
    double* d_parts;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

using namespace tsm;
using namespace tsm::batched;

extern "C" {

void tsm_batched_destroy(tsm_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_inst);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_tickets);
    cudaFree(b->d_parts);
    free(b);
}

tsm_status tsm_batched_create(const tsm_batch_desc* d, int count, tsm_batch** out) {
    if (!out || !d || count < 1) return TSM_ERR_INVALID_VALUE;
    *out = nullptr;
    // validate every descriptor first
    for (int i = 0; i < count; ++i) {
        const tsm_batch_desc& x = d[i];
        tsm_status st = validate_common(x.dtype, x.M, x.N, x.K, x.alpha, x.beta);
        if (st != TSM_OK) return st;
        if (x.kind == TSM_KIND_TSMTTSM) {
            if (x.op != TSM_OP_T && x.op != TSM_OP_C) return TSM_ERR_INVALID_VALUE;
            if (x.lda < x.M || x.ldb < x.N || x.ldo < x.N) return TSM_ERR_INVALID_VALUE;
        } else if (x.kind == TSM_KIND_TSMM) {
            if (x.op != TSM_OP_N) return TSM_ERR_NOT_SUPPORTED;
            if (x.lda < x.M || x.ldb < x.N || x.ldo < x.N) return TSM_ERR_INVALID_VALUE;
        } else {
            return TSM_ERR_INVALID_VALUE;
        }
        if (!x.out || (x.K > 0 && (!x.A || !x.B))) return TSM_ERR_INVALID_VALUE;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSM_ERR_NO_DEVICE;
    const DeviceInfo& di = device_info();
    if (di.cc_major != 10 || di.cc_minor != 3) return TSM_ERR_NO_DEVICE;

    // shared memory: TSMM C staging, at least the reduction buffer
    size_t smem = kThreads * 2 * sizeof(double);
    for (int i = 0; i < count; ++i)
        if (d[i].kind == TSM_KIND_TSMM)
            smem = std::max(smem, (size_t)d[i].M * d[i].N * (d[i].dtype == TSM_C64 ? 2 : 1) * sizeof(double));
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TSM_ERR_LAUNCH;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched, kThreads, smem) != cudaSuccess || occ < 1)
        return TSM_ERR_LAUNCH;
    const int ctas = di.sm_count * occ;

    // instance table and work items
    std::vector<Inst> inst(count);
    double total = 0.0;
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) {
        const int c = d[i].dtype == TSM_C64 ? 2 : 1;
        work[i] = (double)d[i].K * d[i].M * d[i].N * c * c + 1.0;
        total += work[i];
    }
    std::vector<Item> items;
    int64_t part_doubles = 0;
    for (int i = 0; i < count; ++i) {
        const tsm_batch_desc& x = d[i];
        Inst& in = inst[i];
        memset(&in, 0, sizeof(in));
        in.kind = x.kind;
        in.cplx = x.dtype == TSM_C64;
        in.conj = (in.cplx && x.op == TSM_OP_C) ? 1 : 0;
        in.M = x.M;
        in.N = x.N;
        in.K = x.K;
        in.lda = x.lda;
        in.ldb = x.ldb;
        in.ldo = x.ldo;
        in.A = (const double*)x.A;
        in.B = (const double*)x.B;
        in.out = (double*)x.out;
        in.ar = x.alpha[0];
        in.ai = in.cplx ? x.alpha[1] : 0.0;
        in.br = x.beta[0];
        in.bi = in.cplx ? x.beta[1] : 0.0;
        in.beta_zero = x.beta[0] == 0.0 && (!in.cplx || x.beta[1] == 0.0);
        int code = x.config & 0xFF;
        if (x.kind == TSM_KIND_TSMTTSM) {
            if (!tile_ok(code, x.M, x.N, in.cplx)) code = default_tile(x.M, x.N, in.cplx);
        } else if (code < 1 || code > 4) {
            // power-of-two threads per row when they cover N exactly, else
            // any count (code 4)
            const int tpr = x.N >= 16 ? 16 : (x.N >= 8 ? 8 : 4);
            const int npt = (x.N + tpr - 1) / tpr;
            const int cap = tpr == 4 ? 16 : (tpr == 8 ? 8 : 4);  // results per thread of codes 1, 2, 3
            const bool exact = npt * tpr == x.N && npt <= cap && !(in.cplx && tpr == 4);  // complex code 1 is 8 x 8
            code = exact ? (tpr == 16 ? 3 : (tpr == 8 ? 2 : 1)) : 4;
        }
        in.code = code;
        if (x.kind == TSM_KIND_TSMM && code == 4) {
            int npt = 1;
            rt_tsmm_tpr(x.N, 4, &in.tpr, &npt);
        }
        int64_t rows;
        const int lg = (x.config >> 8) & 0xFF;
        if (lg >= 10 && lg <= 22) {
            rows = (int64_t)1 << lg;
        } else {
            // about kItemsPerCta items per CTA over the whole batch, each
            // instance cut in proportion to its work; rows per item the
            // nearest power of two (at least 4096), so an instance ends in a
            // shorter ragged item and the largest-first order finishes on
            // small items
            const double share = work[i] / total * ctas * kItemsPerCta;
            const double n = std::max(1.0, std::floor(share));
            const int l = (int)std::lround(std::log2(std::max((double)x.K / n, 1.0)));
            rows = (int64_t)1 << std::min(22, std::max(12, l));
        }
        const int64_t K = std::max<int64_t>(x.K, 1);
        const int n_items = (int)((K + rows - 1) / rows);
        in.n_items = n_items;
        in.part_off = part_doubles;
        if (x.kind == TSM_KIND_TSMTTSM) part_doubles += (int64_t)n_items * x.M * x.N * (in.cplx ? 2 : 1);
        for (int j = 0; j < n_items; ++j) {
            Item it;
            it.inst = i;
            it.idx = j;
            it.r0 = std::min<int64_t>((int64_t)j * rows, x.K);
            it.r1 = std::min<int64_t>((int64_t)(j + 1) * rows, x.K);
            items.push_back(it);
        }
    }
    // largest items first (list scheduling over the persistent CTAs)
    std::stable_sort(items.begin(), items.end(), [&](const Item& a, const Item& b) {
        const Inst& ia = inst[a.inst];
        const Inst& ib = inst[b.inst];
        const double ca = (double)(a.r1 - a.r0 + 1) * ia.M * ia.N * (ia.cplx ? 4 : 1);
        const double cb = (double)(b.r1 - b.r0 + 1) * ib.M * ib.N * (ib.cplx ? 4 : 1);
        return ca > cb;
    });

    tsm_batch* b = (tsm_batch*)calloc(1, sizeof(tsm_batch));
    if (!b) return TSM_ERR_ALLOC;
    b->n_items = (int)items.size();
    b->n_inst = count;
    b->ctas = ctas;
    b->smem = smem;
    bool ok = cudaMalloc(&b->d_inst, sizeof(Inst) * count) == cudaSuccess &&
              cudaMalloc(&b->d_items, sizeof(Item) * items.size()) == cudaSuccess &&
              cudaMalloc(&b->d_counter, sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc(&b->d_tickets, sizeof(unsigned) * count) == cudaSuccess &&
              cudaMalloc(&b->d_parts, sizeof(double) * std::max<int64_t>(part_doubles, 1)) == cudaSuccess;
    if (!ok) {
        tsm_batched_destroy(b);
        return TSM_ERR_ALLOC;
    }
    if (cudaMemcpy(b->d_inst, inst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_tickets, 0, sizeof(unsigned) * count) != cudaSuccess) {
        tsm_batched_destroy(b);
        return TSM_ERR_LAUNCH;
    }
    // capture {counter reset, persistent kernel} once
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        tsm_batched_destroy(b);
        return TSM_ERR_LAUNCH;
    }
    bool cap = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (cap) {
        cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), cs);
        k_batched<<<ctas, kThreads, smem, cs>>>(b->d_inst, b->d_items, b->n_items, b->d_counter, b->d_tickets,
                                                b->d_parts);
        cap = cudaStreamEndCapture(cs, &b->graph) == cudaSuccess && b->graph != nullptr;
    }
    cudaStreamDestroy(cs);
    if (!cap || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        tsm_batched_destroy(b);
        return TSM_ERR_LAUNCH;
    }
    *out = b;
    return TSM_OK;
}

tsm_status tsm_batched_run(tsm_batch* b, tsm_stream_t stream) {
    if (!b || !b->exec) return TSM_ERR_INVALID_VALUE;
    return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? TSM_OK : TSM_ERR_LAUNCH;
}

tsm_status tsm_batched_run_direct(tsm_batch* b, tsm_stream_t stream) {
    if (!b) return TSM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), s) != cudaSuccess) return TSM_ERR_LAUNCH;
    k_batched<<<b->ctas, kThreads, b->smem, s>>>(b->d_inst, b->d_items, b->n_items, b->d_counter, b->d_tickets,
                                                 b->d_parts);
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_LAUNCH;
}

tsm_status tsm_batched_info(const tsm_batch* b, int* items, int* ctas) {
    if (!b || !items || !ctas) return TSM_ERR_INVALID_VALUE;
    *items = b->n_items;
    *ctas = b->ctas;
    return TSM_OK;
}

}  // extern "C"
