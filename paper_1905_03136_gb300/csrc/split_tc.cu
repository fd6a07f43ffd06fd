// Split-precision TSMTTSM on the 5th-generation tensor cores (tcgen05).
//
// G = X^T Y for real tall & skinny X (K x P) and Y (K x Q) in binary64 --
// complex A^T B / A^H B are the real product of the interleaved (re, im)
// columns, recombined at the end -- computed with error-free splitting after
// Ozaki, Ogita, Oishi, Rump (Numer. Algorithms 59, 2012):
//
//   x = 2^e * sum_s alpha_s * 2^(-7 - 8s),  s = 0..5, alpha_s integer, |alpha_s| <= 128
//
// where e is a running maximum exponent of x's column (|x| < 2^e), so every
// alpha_s is exact in fp16 (11-bit significand).  Then, per accumulation tile of at most 256
// rows in which no column exponent changes,
//
//   sum_k x_kp y_kq = 2^(e_p + e_q - 14) * sum_d 2^(-8d) P_d[p][q],
//   P_d = sum_k sum_{s+t=d} alpha_s beta_t,  d = 0..5 (pairs with s+t > 5 dropped),
//
// and each P_d is a sum of at most 6 * 256 products of magnitude <= 2^14:
// exact in FP32 for d <= 3 (<= 2^24), and within a few FP32 units for
// d = 4, 5 whose weight is below 2^-46.  The tensor cores form all P_d in
// tensor memory; the epilogue converts them to one exact 64-bit integer
// W = sum_d P_d 2^(8(5-d)) per entry and accumulates W * 2^(e_p+e_q-54) in
// binary64.  Partials of all CTAs are reduced in a fixed order.
//
// CTA organisation (one CTA per SM, persistent over a contiguous K range and
// a chunk of Y's columns):
//   warps 0-15  converters: stage upcoming 16-row steps of X and Y from
//               global memory into a per-thread cp.async ring several steps
//               ahead (loads of later steps are in flight while step s is
//               converted: the paper's leap frogging, Sec. 3.1, made deep),
//               update the running column exponents, and write the six fp16
//               slices into shared memory in the canonical K-major
//               core-matrix layout of the MMA operands; one unit of work is
//               4 rows of one column;
//   warp 16     allocates tensor memory and issues tcgen05.mma (one thread);
//   warps 17-20 epilogue: drain tensor memory after each tile (tcgen05.ld),
//               recombine, accumulate in binary64 in shared memory.
// MMA operand A (M = 128 rows): X slices, two slices per 128-row block when
// P <= 64 ("stacked"), one slice per block when 64 < P <= 128.  Operand B
// (N rows): the six Y slices stacked, Qp rows each.  Accumulator column
// block j holds the slice pair(s) whose weight index is d = j (rows of the
// second stacked slice: d = j + 1).
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the
// kernel records an error word, stops issuing work, drains its own MMAs,
// frees tensor memory and exits; the combine kernel then writes NaN.
#include <cstdint>
#include <cstdio>

#include <cuda_fp16.h>

#include "tsm_internal.h"
#include "tsm_split.h"

namespace tsm {
namespace split {

constexpr int KSTEP = 16;           // rows per MMA (16-bit inputs: K = 16)
constexpr int TILE_STEPS = 16;      // steps per exact accumulation tile (256 rows)
constexpr int NSLICE = 6;           // 8-bit slices per input
constexpr int NDIG = 2;             // digit stages (converters -> MMA)
constexpr int NST_MAX = 8;          // FP64 staging stages (cp.async ring, per thread)
constexpr int NEXP = 4;             // exponent snapshot ring (converters -> epilogue)
constexpr int MAX_CONV_WARPS = 16;  // converters: a per-shape multiple of 32 threads
constexpr int NCONV_MAX = MAX_CONV_WARPS * 32;
constexpr int NEPI_WARPS = 4;
constexpr int NTHREADS_MAX = (MAX_CONV_WARPS + 1 + NEPI_WARPS) * 32;  // 672
constexpr int TMEM_COLS = 512;
constexpr int E_NONE = -4000;       // running exponent before any nonzero value
constexpr long long kDefaultTimeout = 4000000000ll;  // SM cycles (~2 s)

struct Params {
    const double* X;
    int64_t ldx;  // doubles
    const double* Y;
    int64_t ldy;
    int P, Q;     // real column counts of X and Y
    int64_t K;
    int n_kr, n_qc;
    int q0[2], qw[2];
    int64_t steps_per_kr;
    int stacked;  // P <= 64
    int Qp;       // padded chunk width (multiple of 16)
    int nconv;    // converter threads (multiple of 32, <= NCONV_MAX); MMA warp and 4 epilogue warps follow
    double* ws;     // [n_kr][P][Q]
    double* flush;  // [CTA][Qp][128]: binary64 totals of the epilogue lanes
    int* err;
    long long timeout;
};

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and the error word set) if the phase did not complete
// within `timeout` SM cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long timeout, int* err,
                                          int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 16;  // back off so waiting warps leave issue slots to working ones
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > timeout) {
            atomicCAS(err, 0, code);
            return false;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes (128 contiguous bytes); `lbo` is the byte
// distance between core matrices adjacent along K, `sbo` between core
// matrices adjacent along M/N.  Bits 46-48 hold the fixed value 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D = F32, A = B = F16 (format code 0),
// both K-major, M = 128, N as given.
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ shared layout

struct Layout {
    int nrb;            // 128-row blocks of operand A per step
    int units;          // (column, 4-row group) units per step: 4 * (P + Qw)
    int nst;            // FP64 staging stages
    uint32_t a_bytes;   // operand A bytes per step
    uint32_t b_bytes;   // operand B bytes per step
    uint32_t stage;     // digit stage bytes (1024-aligned)
    uint32_t dig_off;   // offset of digit stage 0
    uint32_t acc_off;   // binary64 accumulators [Qp][128]
    uint32_t exp_off;   // running exponents [P + Qp] then snapshots [NEXP][P + Qp]
    uint32_t misc_off;  // barriers, flags, tmem slot
    uint32_t stg_off;   // FP64 staging ring: nst x [4 rows][units] doubles
    uint32_t stg_bytes; // bytes per staging stage
    uint32_t total;
};

constexpr uint32_t kSmemBudget = 227u * 1024u;

__host__ __device__ inline Layout make_layout(int P, int Qp, int Qw, int stacked) {
    Layout L;
    L.nrb = stacked ? 3 : 6;
    L.units = 4 * (P + Qw);
    L.a_bytes = (uint32_t)L.nrb * 4096u;
    L.b_bytes = (uint32_t)NSLICE * Qp * 32u;
    L.stage = ((L.a_bytes + L.b_bytes) + 1023u) & ~1023u;
    L.dig_off = 0;
    L.acc_off = L.dig_off + NDIG * L.stage;
    const uint32_t ne = (uint32_t)(P + Qp);
    L.exp_off = L.acc_off + (uint32_t)Qp * 128u * 8u;
    L.misc_off = (L.exp_off + (1u + NEXP) * ne * 4u + 127u) & ~127u;
    L.stg_off = (L.misc_off + 512u + 127u) & ~127u;
    L.stg_bytes = (uint32_t)L.units * 32u;
    // as many staging stages as fit (at least 2), up to NST_MAX
    int nst = 2;
    const int opts[4] = {8, 6, 4, 3};
    for (int i = 0; i < 4; ++i)
        if (L.stg_off + (uint32_t)opts[i] * L.stg_bytes <= kSmemBudget) {
            nst = opts[i];
            break;
        }
    L.nst = nst;
    L.total = L.stg_off + (uint32_t)nst * L.stg_bytes;
    if (L.total < 120u * 1024u) L.total = 120u * 1024u;  // one CTA per SM (tensor memory is taken whole)
    return L;
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most `pending` of this thread's groups are in flight.
__device__ __forceinline__ void cp_async_wait(int pending) {
    switch (pending) {
        case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
        case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
    }
}

// misc area: byte offsets of the barriers and flags
enum {
    M_DIG_FULL = 0,     // NDIG x 8
    M_DIG_EMPTY = 32,   // NDIG x 8
    M_EXP_EMPTY = 64,   // NEXP x 8
    M_TILE_FULL = 96,
    M_TMEM_EMPTY = 104,
    M_MMA_DONE = 112,
    M_TMEM_SLOT = 128,
    M_META = 136,       // NDIG ints: bit0 new tile, bits 1..: exponent slot
    M_BRK = 160,        // 2 ints
    M_ABORT = 168,
    M_TILE_INFO = 172,  // slot | last << 8
    M_CONV_FAIL = 176,
};

// ------------------------------------------------------------ digit maths

// |x| as a fixed-point integer with 47 bits below 2^e (truncated), plus the
// five low bytes biased by 0x80 so that they read back as balanced digits:
// returns Y = X + 0x8080808080 where X = floor(|x| 2^(47-e)) < 2^47.  The
// six base-256 digits of X = sum_s d_s 2^(40-8s) are d_0 = byte 5 of Y in
// [0, 128] and d_s = byte (5-s) of Y - 128 in [-128, 127] for s >= 1.
// Requires |x| < 2^e; subnormals are exact (no implicit bit); values below
// the column's range give 0 (the shift is clamped to 63).
__device__ __forceinline__ unsigned long long fixed47(double x, int e, uint32_t* sign) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(bits >> 32);
    *sign = hi & 0x80000000u;
    const int ef = (int)((hi >> 20) & 0x7FFu);
    const uint32_t mhi = (hi & 0xFFFFFu) | (ef ? 0x100000u : 0u);
    const unsigned long long mant = ((unsigned long long)mhi << 32) | (uint32_t)bits;
    const int sh = min(e + 1028 - max(ef, 1), 63);
    return (mant >> sh) + 0x8080808080ull;
}

// The six fp16 slices of two values a (row r) and b (row r + 1) of one
// column, packed per slice as (a, b) in one 32-bit word, sign applied.  A
// digit byte placed under the fp16 exponent of 1024 (0x64XX) is 1024 + byte
// exactly; one packed subtraction removes 1024 (+ 128) from both halves.
__device__ __forceinline__ void split_pair(double xa, double xb, int e, uint32_t* w) {
    uint32_t sa, sb;
    const unsigned long long ya = fixed47(xa, e, &sa), yb = fixed47(xb, e, &sb);
    const uint32_t alo = (uint32_t)ya, ahi = (uint32_t)(ya >> 32);
    const uint32_t blo = (uint32_t)yb, bhi = (uint32_t)(yb >> 32);
    const uint32_t sg = (sa >> 16) | sb;
    const __half2 top = __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400));  // 1024
    const __half2 low = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));  // 1152
    auto make = [&](uint32_t x, uint32_t y, uint32_t sel, __half2 bias) {
        uint32_t u = (__byte_perm(x, y, sel) & 0x00FF00FFu) | 0x64006400u;
        __half2 h = __hsub2(*reinterpret_cast<__half2*>(&u), bias);
        return *reinterpret_cast<uint32_t*>(&h) ^ sg;
    };
    w[0] = make(ahi, bhi, 0x0501, top);  // byte 5
    w[1] = make(ahi, bhi, 0x0400, low);  // byte 4
    w[2] = make(alo, blo, 0x0703, low);  // byte 3
    w[3] = make(alo, blo, 0x0602, low);  // byte 2
    w[4] = make(alo, blo, 0x0501, low);  // byte 1
    w[5] = make(alo, blo, 0x0400, low);  // byte 0
}

// Exponent from the largest magnitude high word of a column: |x| < 2^e for
// every x of the column (zero and subnormal columns give the subnormal bound).
__device__ __forceinline__ int exp_from_hi(uint32_t hmax) {
    const int ef = (int)(hmax >> 20);
    return (ef > 0 ? ef : 1) - 1022;
}

// Byte offset of element (row r, k-group g) inside a K-major operand block
// (core matrices of 8 rows x 16 bytes; LBO = 128, SBO = 256).
__device__ __forceinline__ uint32_t kmajor_off(int r, int g) {
    return (uint32_t)((r >> 3) * 256 + g * 128 + (r & 7) * 16);
}

// ------------------------------------------------------------ the kernel

__global__ void __launch_bounds__(NTHREADS_MAX, 1) k_split(const Params prm) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int P = prm.P;
    const int kr = blockIdx.x / prm.n_qc, qc = blockIdx.x - kr * prm.n_qc;
    // (selects, not an indexed load: indexing the parameter arrays would
    // copy the whole parameter block to local memory)
    const int q0 = qc ? prm.q0[1] : prm.q0[0];
    const int Qw = qc ? prm.qw[1] : prm.qw[0];
    const int Qp = prm.Qp;
    const double* __restrict__ Xg = prm.X;
    const double* __restrict__ Yg = prm.Y;
    const int64_t ldx = prm.ldx, ldy = prm.ldy, Ktot = prm.K;
    const int stacked = prm.stacked;
    const Layout L = make_layout(P, Qp, Qw, stacked);
    const int NE = P + Qp;
    unsigned char* dig = smem + L.dig_off;
    double* acc = reinterpret_cast<double*>(smem + L.acc_off);  // epilogue integer sums (64-bit)
    int* e_run = reinterpret_cast<int*>(smem + L.exp_off);
    int* e_snap = e_run + NE;
    unsigned char* misc = smem + L.misc_off;
    const uint32_t misc_a = smem_addr(misc);
    auto bar = [&](int off) { return misc_a + (uint32_t)off; };
    volatile int* meta = reinterpret_cast<volatile int*>(misc + M_META);
    volatile int* brk = reinterpret_cast<volatile int*>(misc + M_BRK);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + M_ABORT);
    volatile int* tile_info = reinterpret_cast<volatile int*>(misc + M_TILE_INFO);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long tmo = prm.timeout;
    const int NCONV = prm.nconv, NCONV_WARPS = NCONV / 32;
    const int MMA_WARP = NCONV_WARPS, EPI_WARP0 = NCONV_WARPS + 1;
    const int NTHREADS = blockDim.x;

    // K range of this CTA, in 16-row steps
    const int64_t steps_total = (prm.K + KSTEP - 1) / KSTEP;
    const int64_t s_begin = (int64_t)kr * prm.steps_per_kr;
    int64_t s_end = s_begin + prm.steps_per_kr;
    if (s_end > steps_total) s_end = steps_total;
    const int64_t nsteps = s_end > s_begin ? s_end - s_begin : 0;

    // ---- set-up: zero digit stages, accumulators, exponents; init barriers
    for (uint32_t i = threadIdx.x * 16u; i < L.misc_off; i += NTHREADS * 16u)  // not the staging ring
        *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < NE; i += NTHREADS) e_run[i] = E_NONE;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NDIG; ++i) {
            mbar_init(bar(M_DIG_FULL + 8 * i), NCONV_WARPS);
            mbar_init(bar(M_DIG_EMPTY + 8 * i), 1);
        }
        for (int i = 0; i < NEXP; ++i) mbar_init(bar(M_EXP_EMPTY + 8 * i), NEPI_WARPS);
        mbar_init(bar(M_TILE_FULL), 1);
        mbar_init(bar(M_TMEM_EMPTY), NEPI_WARPS);
        mbar_init(bar(M_MMA_DONE), 1);
        brk[0] = brk[1] = 0;
        *abort_flag = 0;
        fence_mbar_init();
    }
    fence_proxy_async();
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         bar(M_TMEM_SLOT)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(misc + M_TMEM_SLOT);

    if (warp < NCONV_WARPS) {
        // ================================================= converters
        const int ct = threadIdx.x;  // 0..255
        const int units = L.units;
        const int per = (units + NCONV - 1) / NCONV;  // <= 2 by the host's choice of NCONV
        const int nst = L.nst;
        const uint32_t stg_a = smem_addr(smem + L.stg_off);
        double cur[2][4];
        // unit u: column c = u / 4, rows 8g + 4h .. 8g + 4h + 3 of the step
        // with g = (u / 2) % 2, h = u % 2.  Stage element (row r of 4, unit
        // u) of ring slot `slot` sits at stg_off + slot * stg_bytes +
        // (r * units + u) * 8: a thread reads back exactly what it copied, so
        // no barrier guards the ring
        auto issue_step = [&](int64_t s) {
            if (s < nsteps) {
                const int64_t row0 = (s_begin + s) * KSTEP;
                const uint32_t base = stg_a + (uint32_t)(s % nst) * L.stg_bytes;
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    const int u = ct + it * NCONV;
                    if (!(it < per && u < units)) continue;
                    const int c = u >> 2, rb = (u & 3) * 4;
                    const double* col;
                    int64_t ld;
                    if (c < P) {
                        col = Xg + c;
                        ld = ldx;
                    } else {
                        col = Yg + q0 + (c - P);
                        ld = ldy;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int64_t k = row0 + rb + r;
                        const bool ok = k < Ktot;
                        cp_async8(base + (uint32_t)((r * units + u) * 8), col + (ok ? k : 0) * ld, ok);
                    }
                }
            }
            cp_async_commit();  // one group per step, empty or not
        };
        auto read_step = [&](int64_t s) {
            const double* base = reinterpret_cast<const double*>(smem + L.stg_off + (uint32_t)(s % nst) * L.stg_bytes);
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int u = ct + it * NCONV;
                const bool valid = it < per && u < units;
#pragma unroll
                for (int r = 0; r < 4; ++r) cur[it][r] = valid ? base[r * units + u] : 0.0;
            }
        };
        for (int i = 0; i < nst - 1; ++i) issue_step(i);
        int64_t tile = -1;
        int steps_in_tile = TILE_STEPS;
        int slot = 0;
        for (int64_t s = 0; s < nsteps; ++s) {
            issue_step(s + nst - 1);
            cp_async_wait(nst - 1);
            read_step(s);
            // -- phase 1: column exponents of this step, running maxima
            if (ct == 0) brk[(s + 1) & 1] = 0;  // read by everyone before the previous barrier
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                uint32_t hm = 0;
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(cur[it][r]) >> 32) & 0x7FFFFFFFu);
                hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, 1));  // the four units of a column
                hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, 2));  // are adjacent lanes
                const int em = exp_from_hi(hm);
                const int u = ct + it * NCONV;
                if (it < per && u < units && (u & 3) == 0) {
                    const int c = u >> 2;
                    if (em > e_run[c]) {
                        e_run[c] = em;
                        brk[s & 1] = 1;
                    }
                }
            }
            named_sync(1, NCONV);
            if (*abort_flag) break;  // uniform: set before this barrier by a failed warp
            const bool expchg = brk[s & 1] != 0;  // a column exponent grew: new scale
            const bool new_tile = expchg || steps_in_tile >= TILE_STEPS;
            // waits are taken by lane 0 and broadcast, so failure is warp-uniform
            bool ok = true;
            if (new_tile) {
                ++tile;
                steps_in_tile = 0;
                slot = (int)(tile % NEXP);
                int w_ok = 1;
                if (lane == 0)
                    w_ok = mbar_wait(bar(M_EXP_EMPTY + 8 * slot), (uint32_t)(((tile / NEXP) & 1) ^ 1), tmo,
                                     prm.err, 1);
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                if (ok)
                    for (int i = ct; i < NE; i += NCONV) e_snap[slot * NE + i] = e_run[i];
            }
            ++steps_in_tile;
            const int d = (int)(s % NDIG);
            if (ok) {
                int w_ok = 1;
                if (lane == 0)
                    w_ok = mbar_wait(bar(M_DIG_EMPTY + 8 * d), (uint32_t)(((s / NDIG) & 1) ^ 1), tmo, prm.err, 2);
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
            }
            if (!ok) {
                *abort_flag = 1;  // the others stop at the next barrier
                continue;
            }
            // -- phase 2: six fp16 slices of every value into the digit stage
            unsigned char* stage = dig + d * L.stage;
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int u = ct + it * NCONV;
                if (!(it < per && u < units)) continue;
                const int c = u >> 2, g = (u >> 1) & 1, hb = (u & 1) * 8;
                const int e = e_run[c];
                uint32_t w[NSLICE][2];
#pragma unroll
                for (int r = 0; r < 4; r += 2) {
                    uint32_t wp[NSLICE];
                    split_pair(cur[it][r], cur[it][r + 1], e, wp);
#pragma unroll
                    for (int sl = 0; sl < NSLICE; ++sl) w[sl][r >> 1] = wp[sl];
                }
                if (c < P) {
                    // operand A: slice sl in block (stacked ? sl/2 : sl), row (stacked ? (sl&1)*64 : 0) + c
#pragma unroll
                    for (int sl = 0; sl < NSLICE; ++sl) {
                        const int blk = stacked ? (sl >> 1) : sl;
                        const int row = (stacked ? (sl & 1) * 64 : 0) + c;
                        *reinterpret_cast<uint2*>(stage + blk * 4096 + kmajor_off(row, g) + hb) =
                            make_uint2(w[sl][0], w[sl][1]);
                    }
                } else {
                    const int q = c - P;
#pragma unroll
                    for (int sl = 0; sl < NSLICE; ++sl)
                        *reinterpret_cast<uint2*>(stage + L.a_bytes + kmajor_off(sl * Qp + q, g) + hb) =
                            make_uint2(w[sl][0], w[sl][1]);
                }
            }
            if (ct == 0) meta[d] = (new_tile ? 1 : 0) | (expchg ? 2 : 0) | (slot << 2);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(M_DIG_FULL + 8 * d));
        }
        cp_async_wait(0);  // no copy may land after the CTA exits
    } else if (warp == MMA_WARP) {
        // ================================================= MMA issuer
        if (lane == 0) {
            int64_t tile = -1;
            int cur_slot = 0, cur_chg = 0;
            bool failed = false;
            uint32_t mma_phase = 0;
            const uint32_t dig_a = smem_addr(dig);
            for (int64_t s = 0; s < nsteps && !failed; ++s) {
                const int d = (int)(s % NDIG);
                if (!mbar_wait(bar(M_DIG_FULL + 8 * d), (uint32_t)((s / NDIG) & 1), tmo, prm.err, 3)) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const int m = meta[d];
                const bool new_tile = (m & 1) != 0;
                if (new_tile) {
                    if (tile >= 0) {
                        // hand the finished tile to the epilogue
                        mma_commit(bar(M_MMA_DONE));
                        if (!mbar_wait(bar(M_MMA_DONE), mma_phase, tmo, prm.err, 4)) {
                            failed = true;
                            break;
                        }
                        mma_phase ^= 1;
                        *tile_info = cur_slot | (cur_chg << 10);
                        tc_fence_before();
                        mbar_arrive(bar(M_TILE_FULL));
                        if (!mbar_wait(bar(M_TMEM_EMPTY), (uint32_t)(tile & 1), tmo, prm.err, 5)) {
                            failed = true;
                            break;
                        }
                        tc_fence_after();
                    }
                    ++tile;
                    cur_slot = m >> 2;
                    cur_chg = (m >> 1) & 1;
                }
                const uint32_t sa = dig_a + (uint32_t)d * L.stage;
                const uint32_t sb = sa + L.a_bytes;
                const int maxs = 256 / Qp;  // slices per MMA (N <= 256)
                // first MMA per accumulator block overwrites when the tile starts:
                // row block 0 covers every block j = 0..5, so it goes first.
                for (int rb = 0; rb < L.nrb; ++rb) {
                    const int s_a = stacked ? 2 * rb : rb;  // first slice index of this row block
                    const int nt = NSLICE - s_a;            // slices t with s_a + t <= 5
                    for (int t0 = 0; t0 < nt; t0 += maxs) {
                        const int cnt = min(maxs, nt - t0);
                        const uint64_t ad = smem_desc(sa + rb * 4096, 128, 256);
                        const uint64_t bd = smem_desc(sb + (uint32_t)(t0 * Qp * 32), 128, 256);
                        const uint32_t dcol = (uint32_t)((s_a + t0) * Qp);
                        mma_f16(tmem + dcol, ad, bd, instr_desc(cnt * Qp), (rb == 0 && new_tile) ? 0u : 1u);
                    }
                }
                mma_commit(bar(M_DIG_EMPTY + 8 * d));
            }
            // last tile (or drain after a failure)
            mma_commit(bar(M_MMA_DONE));
            const bool drained = mbar_wait(bar(M_MMA_DONE), mma_phase, kDefaultTimeout, prm.err, 6);
            if (!failed && drained && tile >= 0) {
                *tile_info = cur_slot | (1 << 8) | (cur_chg << 10);
                tc_fence_before();
                mbar_arrive(bar(M_TILE_FULL));
            } else if (tile < 0 && !failed) {
                *tile_info = 1 << 9;  // empty range: nothing to drain
                mbar_arrive(bar(M_TILE_FULL));
            }
        }
        __syncwarp();
    } else {
        // ================================================= epilogue
        // Per (lane, column): an exact 64-bit integer sum of the tiles' W in
        // shared memory, at the scale of the current column exponents.  It
        // moves to binary64 (`flush`, this thread's own entries in global
        // memory) only when an exponent grows, when the integer sum would
        // overflow, and at the end -- not once per tile.
        const int ew = warp - EPI_WARP0;
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;  // TMEM lane = accumulator row
        const int p = stacked ? (row & 63) : row;
        const int half = stacked ? (row >> 6) : 0;
        const bool prow = p < P;
        long long* iacc = reinterpret_cast<long long*>(acc);
        double* flush = prm.flush + (int64_t)blockIdx.x * Qp * 128;
        for (int q = 0; q < Qp; ++q) flush[q * 128 + row] = 0.0;
        auto scaled = [](long long a, int E) {
            return (E >= -1022 && E <= 1023) ? (double)a * __longlong_as_double((long long)(E + 1023) << 52)
                                             : scalbn((double)a, E);
        };
        auto flush_all = [&](const int* exs) {
            if (!prow) return;
            const int epf = exs[p];
            for (int q = 0; q < Qw; ++q) {
                const long long a = iacc[q * 128 + row];
                if (a == 0) continue;
                iacc[q * 128 + row] = 0;
                flush[q * 128 + row] += scaled(a, epf + exs[P + q] - 54);
            }
        };
        int prev_slot = -1;
        for (int64_t tile = 0;; ++tile) {
            if (!mbar_wait(bar(M_TILE_FULL), (uint32_t)(tile & 1), tmo, prm.err, 7)) break;
            tc_fence_after();
            const int info = *tile_info;
            if (info & (1 << 9)) break;
            const int slot = info & 0xFF;
            const bool chg = (info >> 10) & 1;
            if (prev_slot >= 0) {
                if (chg) flush_all(e_snap + prev_slot * NE);  // sums so far carry the old scale
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(M_EXP_EMPTY + 8 * prev_slot));
            }
            const int* ex = e_snap + slot * NE;
            const int ep = prow ? ex[p] : 0;
            for (int qb = 0; qb < Qp; qb += 8) {
                uint32_t v[NSLICE][8];
#pragma unroll
                for (int j = 0; j < NSLICE; ++j)
                    tmem_ld8(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(j * Qp + qb), v[j]);
                tmem_wait_ld();
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int q = qb + qq;
                    if (!prow || q >= Qw) continue;
                    long long W = 0;
#pragma unroll
                    for (int j = 0; j < NSLICE; ++j) {
                        const int dd = j + half;
                        if (dd < NSLICE)
                            W += (long long)__float2int_rn(__uint_as_float(v[j][qq])) << (8 * (NSLICE - 1 - dd));
                    }
                    if (W == 0) continue;
                    long long* ap = &iacc[q * 128 + row];
                    const long long a = *ap;
                    long long sum = (long long)((unsigned long long)a + (unsigned long long)W);
                    if (((a ^ sum) & (W ^ sum)) < 0) {  // would overflow: move a to binary64
                        flush[q * 128 + row] += scaled(a, ep + ex[P + q] - 54);
                        sum = W;
                    }
                    *ap = sum;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(M_TMEM_EMPTY));
            prev_slot = slot;
            if (info & (1 << 8)) {
                flush_all(ex);
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(M_EXP_EMPTY + 8 * slot));
                break;
            }
        }
        (void)ew;
    }

    __syncthreads();
    // CTA partial: G[p][q0 + q] for this K range
    double* out = prm.ws + (int64_t)kr * P * prm.Q;
    const double* fl = prm.flush + (int64_t)blockIdx.x * Qp * 128;
    for (int i = threadIdx.x; i < P * Qw; i += NTHREADS) {
        const int pp = i / Qw, q = i - pp * Qw;
        double v = fl[q * 128 + pp];
        if (stacked) v += fl[q * 128 + 64 + pp];
        out[(int64_t)pp * prm.Q + q0 + q] = v;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Sums the per-range partials in range order and applies alpha / beta; for
// complex data G holds the real products of interleaved columns:
// A^T B = (RR - II) + i (RI + IR), A^H B = (RR + II) + i (RI - IR).
__global__ void k_split_combine(const double* ws, int n_kr, int P, int Q, int M, int N, int cplx, int conj,
                                double ar, double ai, double br, double bi, int beta_zero, double* C,
                                int64_t ldc, const int* err) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= M * N) return;
    const int m = o / N, n = o - m * N;
    const bool bad = *err != 0;
    auto G = [&](int p, int q) {
        double s = 0.0;
        for (int r = 0; r < n_kr; ++r) s += ws[(int64_t)r * P * Q + (int64_t)p * Q + q];
        return s;
    };
    if (!cplx) {
        double v = ar * G(m, n);
        double* out = C + (int64_t)m * ldc + n;
        if (!beta_zero) v = fma(br, *out, v);
        *out = bad ? __longlong_as_double(0x7ff8000000000000ll) : v;
    } else {
        const double rr = G(2 * m, 2 * n), ii = G(2 * m + 1, 2 * n + 1);
        const double ri = G(2 * m, 2 * n + 1), ir = G(2 * m + 1, 2 * n);
        const double gr = conj ? rr + ii : rr - ii;
        const double gi = conj ? ri - ir : ri + ir;
        double vr = ar * gr - ai * gi, vi = ar * gi + ai * gr;
        double* out = C + ((int64_t)m * ldc + n) * 2;
        if (!beta_zero) {
            const double orr = out[0], oi = out[1];
            vr += br * orr - bi * oi;
            vi += br * oi + bi * orr;
        }
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        out[0] = bad ? nan : vr;
        out[1] = bad ? nan : vi;
    }
}

long long g_timeout = kDefaultTimeout;

}  // namespace split

tsm_status validate_common(int dtype, int M, int N, int64_t K, const double* alpha, const double* beta);

}  // namespace tsm

using namespace tsm;

extern "C" tsm_status tsm_tsmttsm_split(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K,
                                        const double* alpha, const void* A, int64_t lda, const void* B,
                                        int64_t ldb, const double* beta, void* C, int64_t ldc,
                                        tsm_stream_t stream) {
    tsm_status st = validate_common(dtype, M, N, K, alpha, beta);
    if (st != TSM_OK) return st;
    if (opA != TSM_OP_T && opA != TSM_OP_C) return TSM_ERR_INVALID_VALUE;
    if (lda < M || ldb < N || ldc < N || !C) return TSM_ERR_INVALID_VALUE;
    const int cplx = dtype == TSM_C64;
    const bool alpha0 = alpha[0] == 0.0 && (!cplx || alpha[1] == 0.0);
    if (K > 0 && !alpha0 && (!A || !B)) return TSM_ERR_INVALID_VALUE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSM_ERR_NO_DEVICE;
    const DeviceInfo& di = device_info();
    if (di.cc_major != 10 || di.cc_minor != 3) return TSM_ERR_NO_DEVICE;
    const int beta_zero = beta[0] == 0.0 && (!cplx || beta[1] == 0.0);
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0 || alpha0) {
        return launch_scale_small((double*)C, M, N, ldc, cplx, beta[0], cplx ? beta[1] : 0.0, beta_zero, s) ==
                       cudaSuccess
                   ? TSM_OK
                   : TSM_ERR_LAUNCH;
    }
    const int c = cplx ? 2 : 1;
    const int P = M * c, Q = N * c;
    const int64_t ldx = lda * c, ldy = ldb * c;
    split::Params prm;
    prm.X = (const double*)A;
    prm.ldx = ldx;
    prm.Y = (const double*)B;
    prm.ldy = ldy;
    prm.P = P;
    prm.Q = Q;
    prm.K = K;
    prm.stacked = P <= 64 ? 1 : 0;
    // Y column chunks: one if 6 slices of it fit tensor memory, else two
    // chunks split on an even column
    if (Q <= 80) {
        prm.n_qc = 1;
        prm.q0[0] = 0;
        prm.qw[0] = Q;
        prm.q0[1] = 0;
        prm.qw[1] = 0;
    } else {
        int q1 = ((Q / 2) + 1) & ~1;
        prm.n_qc = 2;
        prm.q0[0] = 0;
        prm.qw[0] = q1;
        prm.q0[1] = q1;
        prm.qw[1] = Q - q1;
    }
    int qmax = prm.qw[0] > prm.qw[1] ? prm.qw[0] : prm.qw[1];
    prm.Qp = (qmax + 15) & ~15;
    const int64_t steps = (K + split::KSTEP - 1) / split::KSTEP;
    int n_kr = di.sm_count / prm.n_qc;
    if (n_kr < 1) n_kr = 1;
    if ((int64_t)n_kr > steps) n_kr = (int)steps;
    prm.steps_per_kr = (steps + n_kr - 1) / n_kr;
    n_kr = (int)((steps + prm.steps_per_kr - 1) / prm.steps_per_kr);
    prm.n_kr = n_kr;
    prm.timeout = split::g_timeout;

    Workspace* ws = nullptr;
    const size_t part = (size_t)n_kr * P * Q * sizeof(double);
    const size_t flush = (size_t)n_kr * prm.n_qc * prm.Qp * 128 * sizeof(double);
    if ((st = workspace_get(s, part + flush + 256, 1, &ws)) != TSM_OK) return st;
    prm.ws = ws->partials;
    prm.flush = ws->partials + (size_t)n_kr * P * Q;
    prm.err = reinterpret_cast<int*>(ws->tickets) + 32;  // error word of this stream
    const split::Layout L = split::make_layout(P, prm.Qp, qmax, prm.stacked);
    // converters: the fewest rounds of units, spread evenly over a multiple
    // of 32 threads
    {
        const int units = L.units;
        const int rounds = (units + split::NCONV_MAX - 1) / split::NCONV_MAX;
        int nconv = (units + rounds - 1) / rounds;
        nconv = (nconv + 31) & ~31;
        if (nconv > split::NCONV_MAX) nconv = split::NCONV_MAX;
        prm.nconv = nconv;
    }
    if (L.total > di.smem_optin) return TSM_ERR_NOT_SUPPORTED;
    if (cudaFuncSetAttribute(split::k_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) !=
        cudaSuccess)
        return TSM_ERR_LAUNCH;
    if (cudaMemsetAsync(prm.err, 0, sizeof(int), s) != cudaSuccess) return TSM_ERR_LAUNCH;
    split::k_split<<<n_kr * prm.n_qc, prm.nconv + (1 + split::NEPI_WARPS) * 32, L.total, s>>>(prm);
    if (cudaGetLastError() != cudaSuccess) return TSM_ERR_LAUNCH;
    const int outs = M * N;
    split::k_split_combine<<<(outs + 127) / 128, 128, 0, s>>>(
        ws->partials, n_kr, P, Q, M, N, cplx, (cplx && opA == TSM_OP_C) ? 1 : 0, alpha[0], cplx ? alpha[1] : 0.0,
        beta[0], cplx ? beta[1] : 0.0, beta_zero, (double*)C, ldc, prm.err);
    if (cudaGetLastError() != cudaSuccess) return TSM_ERR_LAUNCH;
    return TSM_OK;
}

extern "C" tsm_status tsm_split_status(tsm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    Workspace* ws = nullptr;
    tsm_status st = workspace_get(s, 256, 1, &ws);
    if (st != TSM_OK) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TSM_ERR_LAUNCH;
    int err = 0;
    int* p = reinterpret_cast<int*>(ws->tickets) + 32;
    if (cudaMemcpy(&err, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TSM_ERR_LAUNCH;
    if (err) {
        const int zero = 0;
        if (cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return TSM_ERR_LAUNCH;
        return TSM_ERR_TIMEOUT;
    }
    return TSM_OK;
}

extern "C" tsm_status tsm_split_set_timeout(int64_t timeout_cycles) {
    split::g_timeout = timeout_cycles > 0 ? (long long)timeout_cycles : split::kDefaultTimeout;
    return TSM_OK;
}
