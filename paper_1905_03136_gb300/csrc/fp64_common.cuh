// Device helpers shared by the hand-written and the generated FP64 kernels.
#pragma once

#include "tsm_internal.h"

namespace tsm {

// Sum of the G per-CTA partials of entry o (CC doubles each) over the CTA
// slice s, s + S, s + 2S, ... in that fixed order; 8 loads in flight.
template <int CC>
__device__ __forceinline__ void sum_partials(const double* ws, int MNc, int o, int G, int s, int S,
                                             double* out) {
    double acc[CC][8];
#pragma unroll
    for (int c = 0; c < CC; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[c][r] = 0.0;
    int b = s;
    for (; b + 7 * S < G; b += 8 * S)
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < CC; ++c) acc[c][r] += __ldcg(ws + (int64_t)(b + r * S) * MNc + o * CC + c);
    for (; b < G; b += S)
#pragma unroll
        for (int c = 0; c < CC; ++c) acc[c][0] += __ldcg(ws + (int64_t)b * MNc + o * CC + c);
#pragma unroll
    for (int c = 0; c < CC; ++c)
        out[c] = ((acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3])) +
                 ((acc[c][4] + acc[c][5]) + (acc[c][6] + acc[c][7]));
}

// Warp-level sum of V values per lane (V a power of two, 1 <= V <= 32) by
// recursive halving: at the step with lane offset o = 16, 8, ..., a lane
// keeps half of its remaining values (the upper half if its bit o is set)
// and adds its partner's copy of that half, so a step costs as many adds
// as values remain, V - 1 adds over the first log2(V) steps; the remaining
// steps add the single value across lanes (butterfly).  On return v[0] of
// lane l holds the warp total of value l >> (5 - log2 V), and all lanes with
// the same l >> (5 - log2 V) hold identical bits.  A plain butterfly per
// value would take 5 V adds; on a part whose FP64 pipe issues one warp
// instruction per 64 cycles per scheduler, the difference is the fixed cost
// of the in-CTA reduction.  Pairing is fixed, so results repeat bit for bit.
template <int V>
__device__ __forceinline__ void warp_reduce_scatter(double* v, int lane) {
    static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
    int n = V;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
        if (n > 1) {
            const int h = n >> 1;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i >= h) break;
                const double send = up ? v[i] : v[h + i];
                const double keep = up ? v[h + i] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
            n = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  A
// product kernel waits for the previous launch on its stream to complete,
// with its writes visible (pdl_wait), before it writes global memory -- its
// partials, C, or B -- so its own completion implies that of every earlier
// launch.  A TSMTTSM lets the next launch be scheduled (pdl_trigger) once
// its main loop is done: the next product's CTAs then start streaming while
// this one reduces across CTAs, but two products never stream at the same
// time.  A TSMM triggers only by exiting.  A launch that waits at its start
// is a barrier: the launches after it can only overlap it and one another.
// A TSMTTSM reads its inputs before waiting only when the host found that
// no product launched since the last barrier wrote them.  Without the
// launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void tsmttsm_begin(const TsmttsmArgs& a) {
    if (!a.early) pdl_wait();
}

// TSMM's main loop writes B, so it always waits first (a barrier).
__device__ __forceinline__ void tsmm_begin(const TsmmArgs&) { pdl_wait(); }

constexpr int log2_pow2(int v) { return v <= 1 ? 0 : 1 + log2_pow2(v >> 1); }
constexpr int next_pow2(int v) { return v <= 1 ? 1 : 2 * next_pow2((v + 1) >> 1); }

// Epilogue of one entry o = m * N + n of C: C[m][n] = alpha * v + beta *
// C[m][n] (C not read when beta == 0).
template <int CC>
__device__ __forceinline__ void tsmttsm_store_entry(const TsmttsmArgs& a, int o, const double* v) {
    const int m = o / a.N, n = o - m * a.N;
    double* out = a.C + ((int64_t)m * a.ldc + n) * CC;
    if (CC == 1) {
        double r = a.alpha_r * v[0];
        if (!a.beta_zero) r = fma(a.beta_r, out[0], r);
        out[0] = r;
    } else {
        double rr = a.alpha_r * v[0] - a.alpha_i * v[CC - 1];
        double ri = a.alpha_r * v[CC - 1] + a.alpha_i * v[0];
        if (!a.beta_zero) {
            const double orr = out[0], oi = out[CC - 1];
            rr += a.beta_r * orr - a.beta_i * oi;
            ri += a.beta_r * oi + a.beta_i * orr;
        }
        out[0] = rr;
        out[CC - 1] = ri;
    }
}

// Cross-CTA step of the TSMTTSM reduction, called by every thread of every
// CTA once its M x N partial is in the workspace (a.ws + blockIdx.x * M*N*CC):
// the last CTA to take the ticket sums all partials (S threads share each
// entry, thread s taking CTAs s, s + S, ... in order; the S slice sums are
// combined by a pairwise tree with a fixed pairing), stores alpha * sum +
// beta * C (C not read when beta == 0) and resets the ticket for the next
// launch.  `red` is shared
// memory of at least kBlock * CC doubles, free for reuse.  With
// a.final_pass set the CTAs stop after writing their partials and the host
// launches the final kernel instead (many partials: see kFinalThreshold).
template <int CC>
__device__ __forceinline__ void tsmttsm_cross_cta(const TsmttsmArgs& a, double* red) {
    if (a.final_pass) return;  // the partials are summed by the final kernel
    __shared__ unsigned s_last;
    const int M = a.M, N = a.N;
    const int t = threadIdx.x;
    const int MNc = M * N * CC;
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int MN = M * N;
    const int G = gridDim.x;
    // S threads per entry when there are fewer entries than threads.
    int S = 1;
    while (S * 2 * MN <= (int)blockDim.x && S * 2 <= G) S *= 2;
    for (int base = 0; base < MN * S; base += blockDim.x) {
        const int w = base + t;
        double v[CC];
        const bool mine = w < MN * S;
        if (mine) sum_partials<CC>(a.ws, MNc, w / S, G, w % S, S, v);
        if (S > 1) {
            // slice sums of one entry are adjacent threads: pairwise tree
            // with a fixed pairing (slice s absorbs slice s + h).  A serial
            // chain of S - 1 dependent adds would cost S - 1 full FP64
            // issue slots of this part's slow FP64 pipe.
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
        tsmttsm_store_entry<CC>(a, w / S, v);
    }
    if (t == 0) *a.ticket = 0u;
}

// Deterministic two-level reduction of TSMTTSM partial tiles (replaces the
// atomics of Sec. 3.2).  Thread (lane, p) holds acc[(i * TN + j) * CC + c] for
// C[pm + i*PM][pn + j*PN] with pm = p % PM, pn = p / PM.
//   1. the L lanes of each tile entry are summed through shared memory by a
//      pairwise tree with a fixed pairing (lane l absorbs lane l + h), one
//      tile entry at a time, into this CTA's M x N partial in the workspace;
//   2. the last CTA to take the ticket sums all partials: S threads share
//      each entry, thread s taking CTAs s, s + S, ... in order, and the S
//      slice sums are added in slice order; then alpha * sum + beta * C (C
//      not read when beta == 0) is stored and the ticket reset for the next
//      launch.  With many partials (a.final_pass) the CTAs stop after step
//      1 and the host launches the final kernel for step 2.
// (The narrow kernels, whose few entries put up to 256 slices on one
// entry, use tsmttsm_cross_cta instead, with a tree over the slices.)
// Every order above depends only on (G, M, N, tile), so results repeat bit
// for bit.
// Kernels with a tile chosen at launch pass its size (tm <= TM, tn <= TN;
// warp-uniform, so skipped entries cost nothing).  BLK is the kernel's CTA
// size (L * P <= BLK).
template <int TM, int TN, int CC, int BLK = kBlock>
__device__ __forceinline__ void tsmttsm_finish(const TsmttsmArgs& a, const double* acc, int PM, int PN,
                                               int L, int lane, int p, bool active, int tm = TM, int tn = TN) {
    __shared__ double red[BLK * CC];
    __shared__ unsigned s_last;
    const int M = a.M, N = a.N;
    const int P = PM * PN;
    const int t = threadIdx.x;
    const int MNc = M * N * CC;
    double* part = a.ws + (int64_t)blockIdx.x * MNc;
    pdl_trigger();  // the main loop is done
    pdl_wait();     // the previous launch on the stream may still use the workspace
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
#pragma unroll
            for (int c = 0; c < CC; ++c) {
                if (i >= tm || j >= tn) continue;
                if (active) red[lane * P + p] = acc[(i * TN + j) * CC + c];
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

    if (a.final_pass) return;  // the partials are summed by the final kernel
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int MN = M * N;
    const int G = gridDim.x;
    // S threads per entry when there are fewer entries than threads.
    int S = 1;
    while (S * 2 * MN <= (int)blockDim.x && S * 2 <= G) S *= 2;
    for (int base = 0; base < MN * S; base += blockDim.x) {
        const int w = base + t;
        double v[CC];
        const bool mine = w < MN * S;
        if (mine) sum_partials<CC>(a.ws, MNc, w / S, G, w % S, S, v);
        if (S > 1) {
            // slice sums of one entry are adjacent threads: combine in order
#pragma unroll
            for (int c = 0; c < CC; ++c) red[t * CC + c] = mine ? v[c] : 0.0;
            __syncthreads();
            if (mine && (w % S) == 0)
                for (int s = 1; s < S; ++s)
#pragma unroll
                    for (int c = 0; c < CC; ++c) v[c] += red[(t + s) * CC + c];
            __syncthreads();
        }
        if (!mine || (w % S) != 0) continue;
        const int o = w / S;
        const int m = o / N, n = o - m * N;
        double* out = a.C + ((int64_t)m * a.ldc + n) * CC;
        if (CC == 1) {
            double r = a.alpha_r * v[0];
            if (!a.beta_zero) r = fma(a.beta_r, out[0], r);
            out[0] = r;
        } else {
            double rr = a.alpha_r * v[0] - a.alpha_i * v[CC - 1];
            double ri = a.alpha_r * v[CC - 1] + a.alpha_i * v[0];
            if (!a.beta_zero) {
                const double orr = out[0], oi = out[CC - 1];
                rr += a.beta_r * orr - a.beta_i * oi;
                ri += a.beta_r * oi + a.beta_i * orr;
            }
            out[0] = rr;
            out[CC - 1] = ri;
        }
    }
    if (t == 0) *a.ticket = 0u;
}

// Starting value of a TSMM accumulator for B[row][n] whose old value (or,
// oi) was loaded earlier.  GEN = false serves beta == 0 (start at 0) and
// beta == 1 (start at the old value itself): selects only, no FP64
// operation.  GEN = true serves any other beta (start at beta * old).  The
// beta term thus opens the FMA chain instead of costing an FP64 operation
// after it, and the two cases are separate kernel instantiations: with one
// code path for all betas the compiler would run the beta * old multiply
// for beta == 1 too (if-converted), an extra FP64 operation per output on
// the pipe that bounds these kernels.  For real data (CC == 1) xi is not
// written: callers may pass xr's variable.
template <int CC, bool GEN>
__device__ __forceinline__ void tsmm_acc_init(const TsmmArgs& a, double orr, double oi, double& xr, double& xi) {
    if (!GEN) {
        xr = a.beta_zero ? 0.0 : orr;
        if (CC == 2) xi = a.beta_zero ? 0.0 : oi;
    } else if (CC == 1) {
        xr = a.beta_r * orr;
    } else {
        const double nr = fma(a.beta_r, orr, -a.beta_i * oi);
        const double ni = fma(a.beta_r, oi, a.beta_i * orr);
        xr = nr;
        xi = ni;
    }
}

// Single-instantiation form of tsmm_acc_init, for the kernels that are not
// split by beta (the narrow kernels and the generated ones with more than
// 8 threads per row): the general-beta products are volatile asm so that
// the compiler keeps the branch (if-converted, the multiply would run for
// beta == 1 as well).  Measured side by side, the split made those kernels
// slower (their beta = 0 path by up to 60 %), and this form keeps beta = 1
// free of FP64 multiplies without it.
__device__ __forceinline__ double dmul_kept(double x, double y) {
    double r;
    asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(x), "d"(y));
    return r;
}
__device__ __forceinline__ double dfma_kept(double x, double y, double z) {
    double r;
    asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(x), "d"(y), "d"(z));
    return r;
}

template <int CC>
__device__ __forceinline__ void tsmm_acc_init_kept(const TsmmArgs& a, double orr, double oi, double& xr, double& xi) {
    if (a.beta_zero) {
        xr = 0.0;
        if (CC == 2) xi = 0.0;
    } else if (a.beta_one) {
        xr = orr;
        if (CC == 2) xi = oi;
    } else if (CC == 1) {
        xr = dmul_kept(a.beta_r, orr);
    } else {
        const double nr = dfma_kept(a.beta_r, orr, -dmul_kept(a.beta_i, oi));
        const double ni = dfma_kept(a.beta_r, oi, dmul_kept(a.beta_i, orr));
        xr = nr;
        xi = ni;
    }
}

// Host side: a beta other than 0 and 1 takes the instantiation that scales
// the old B values (GEN = true above).
inline bool tsmm_general_beta(const TsmmArgs& a) { return !a.beta_zero && !a.beta_one; }

// TSMM output store of a finished accumulator (beta already folded in).
template <int CC>
__device__ __forceinline__ void tsmm_store_plain(double* out, int n, double vr, double vi) {
    if (CC == 1) {
        out[n] = vr;
    } else {
        out[n * 2] = vr;
        out[n * 2 + 1] = vi;
    }
}

// Stages alpha * C (M x N) into shared memory for TSMM (Sec. 4.2).
template <int CC>
__device__ __forceinline__ void tsmm_stage_c(const TsmmArgs& a, double* cs) {
    const int M = a.M, N = a.N;
    for (int o = threadIdx.x; o < M * N; o += blockDim.x) {
        const int m = o / N, n = o - m * N;
        const double* src = a.Cm + ((int64_t)m * a.ldc + n) * CC;
        if (CC == 1) {
            cs[o] = a.alpha_r * src[0];
        } else {
            const double cr = src[0], ci = src[CC - 1];
            cs[o * CC] = a.alpha_r * cr - a.alpha_i * ci;
            cs[o * CC + CC - 1] = a.alpha_r * ci + a.alpha_i * cr;
        }
    }
    __syncthreads();
}

}  // namespace tsm
