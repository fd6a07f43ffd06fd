// Device helpers shared by the hand-written and the generated FP64 kernels.
#pragma once

#include "tsm_internal.h"

namespace tsm {

// Deterministic two-level reduction of TSMTTSM partial tiles (replaces the
// atomics of Sec. 3.2).  Thread (lane, p) holds acc[(i * TN + j) * CC + c] for
// C[pm + i*PM][pn + j*PN] with pm = p % PM, pn = p / PM.
//   1. lanes are summed through shared memory in lane order, one tile entry
//      at a time, into this CTA's M x N partial in the workspace;
//   2. the last CTA to take the ticket sums all partials in CTA order (four
//      interleaved accumulators, combined pairwise), applies
//      alpha * sum + beta * C (C not read when beta == 0) and resets the
//      ticket for the next launch.
template <int TM, int TN, int CC>
__device__ __forceinline__ void tsmttsm_finish(const TsmttsmArgs& a, const double* acc, int PM, int PN,
                                               int L, int lane, int p, bool active) {
    __shared__ double red[kBlock];
    __shared__ unsigned s_last;
    const int M = a.M, N = a.N;
    const int P = PM * PN;
    const int t = threadIdx.x;
    const int MNc = M * N * CC;
    double* part = a.ws + (int64_t)blockIdx.x * MNc;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
#pragma unroll
            for (int c = 0; c < CC; ++c) {
                if (active) red[lane * P + p] = acc[(i * TN + j) * CC + c];
                __syncthreads();
                if (t < P) {
                    const int m = (t % PM) + i * PM, n = (t / PM) + j * PN;
                    if (m < M && n < N) {
                        double s = 0.0;
                        for (int l = 0; l < L; ++l) s += red[l * P + t];
                        part[(m * N + n) * CC + c] = s;
                    }
                }
                __syncthreads();
            }

    __threadfence();
    __syncthreads();
    if (t == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int MN = M * N;
    const int G = gridDim.x;
    for (int o = t; o < MN; o += blockDim.x) {
        double s[CC][4];
#pragma unroll
        for (int c = 0; c < CC; ++c)
#pragma unroll
            for (int r = 0; r < 4; ++r) s[c][r] = 0.0;
        int b = 0;
        for (; b + 3 < G; b += 4)
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < CC; ++c) s[c][r] += __ldcg(a.ws + (int64_t)(b + r) * MNc + o * CC + c);
        for (; b < G; ++b)
#pragma unroll
            for (int c = 0; c < CC; ++c) s[c][0] += __ldcg(a.ws + (int64_t)b * MNc + o * CC + c);
        double v[CC];
#pragma unroll
        for (int c = 0; c < CC; ++c) v[c] = (s[c][0] + s[c][1]) + (s[c][2] + s[c][3]);
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

// TSMM output store: B[row][n] = acc (+ beta * B[row][n] unless beta == 0).
template <int CC>
__device__ __forceinline__ void tsmm_store(const TsmmArgs& a, double* out, int n, double vr, double vi) {
    if (CC == 1) {
        if (!a.beta_zero) vr = fma(a.beta_r, out[n], vr);
        out[n] = vr;
    } else {
        if (!a.beta_zero) {
            const double orr = out[n * 2], oi = out[n * 2 + 1];
            vr += a.beta_r * orr - a.beta_i * oi;
            vi += a.beta_r * oi + a.beta_i * orr;
        }
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
