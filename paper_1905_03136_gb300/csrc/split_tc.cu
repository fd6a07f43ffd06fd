// Split-precision TSMTTSM on the 5th-generation tensor cores (tcgen05).
//
// G = X^T Y for real tall & skinny X (K x P) and Y (K x Q) in binary64 --
// complex A^T B / A^H B are the real product of the interleaved (re, im)
// columns, recombined at the end -- computed with error-free splitting after
// Ozaki, Ogita, Oishi, Rump (Numer. Algorithms 59, 2012), shown here for
// S = 6 slices (the kernel is templated on S in [4, 6]):
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
// W = sum_d P_d 2^(8(5-d)) per entry and sums W exactly in 64-bit integers
// across tiles, moving the sum to binary64 only when a column exponent
// grows, when it would overflow, and at the end.  Partials of all CTAs are
// reduced in a fixed order.
//
// CTA organisation (one to four CTAs per SM, as tensor memory and shared
// memory allow; each persistent over a contiguous K range and a chunk of Y's
// columns):
//   converter warps  each thread owns one fixed "unit" (8 rows of one
//                    column in every 16-row step) and keeps the global
//                    loads of its next step in flight in registers (the
//                    paper's leap frogging, Sec. 3.1); it keeps its column's
//                    running exponent in a register and writes the S fp16
//                    slices of its 8 values, 16 bytes per slice, into a ring
//                    of digit stages in the canonical K-major core-matrix
//                    layout of the MMA operands.  The warps do not
//                    synchronise with one another: a warp whose column
//                    exponent grew stamps the stage with the step index;
//   MMA warp         allocates tensor memory; lane 0 issues tcgen05.mma and
//                    decides the tile boundaries (a stamped stage, or 16
//                    steps); the warp copies the tile's exponents for the
//                    epilogue;
//   epilogue warps   8 (two per tensor-memory lane quarter, each on half
//                    of the columns) or, with several CTAs per SM, 4:
//                    drain tensor memory after each tile (tcgen05.ld) and
//                    accumulate.
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

#include <type_traits>

#include "tsm_internal.h"
#include "tsm_split.h"

namespace tsm {
namespace split {

constexpr int KSTEP = 16;           // rows per MMA (16-bit inputs: K = 16)
constexpr int TILE_STEPS = 16;      // steps per exact accumulation tile (256 rows)
constexpr int NSLICE_MAX = 6;       // 8-bit slices per input: S in [4, 6], a template parameter
constexpr int NDIG_MAX = 6;         // digit stages (converters -> MMA): as many as fit, up to this
constexpr int NEXP = 4;             // exponent snapshot ring (MMA warp -> epilogue)
constexpr int MAX_MMAS = 9;         // MMAs per step (six slices of X against the Y slices, N <= 256 each)
constexpr int NEPI_MAX = 8;         // epilogue warps: 8 (two per lane quarter) or 4
constexpr int TMEM_COLS_MAX = 512;
constexpr int E_NONE = -4000;       // running exponent before any nonzero value
constexpr long long kDefaultTimeout = 4000000000ll;  // SM cycles (~2 s)

// Converter configuration: each converter thread owns one unit of R rows
// (4 or 8) of one column in every 16-row step, with the loads of DEPTH
// further steps in flight (DEPTH + 1 register sets).  R = 4 gives four
// units per column (more threads, for products of at most 128 columns);
// R = 8 gives two, stored as whole 16-byte core-matrix rows (wider
// products, up to 208 columns P + Qw per CTA).  The CTA size bounds the
// registers per thread.
template <int R>
struct Conv;
template <>
struct Conv<4> {
    static constexpr int MAX_THREADS = 512, DEPTH = 2;
};
template <>
struct Conv<8> {
    static constexpr int MAX_THREADS = 416, DEPTH = 1;
};
template <int R>
constexpr int block_threads() {
    return Conv<R>::MAX_THREADS + (1 + NEPI_MAX) * 32;
}
// converter threads a CTA needs for `cols` columns with R-row units
__host__ __device__ constexpr int conv_threads(int cols, int R) { return 32 * (((16 / R) * cols + 31) / 32); }

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
    int nconv;    // converter threads (multiple of 32); the MMA warp and the epilogue warps follow
    int nepi;     // epilogue warps: 4 (each on all columns) or 8 (two per lane quarter, half the columns each)
    int tmem_cols;  // tensor-memory columns allocated: a power of two >= 6 * Qp
    int smem_budget;  // bytes of shared memory the layout may use (several CTAs per SM share 228 KB)
    int smem_floor;   // minimum dynamic shared memory: keeps more CTAs than planned off an SM
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
// Bounded wait: false if the phase did not complete within `timeout` SM
// cycles (the error word is then set to `code`), or if another warp raised
// the CTA's abort flag meanwhile (`abort_flag` may be null: wait regardless).
// mbarrier.try_wait itself suspends the warp until the phase completes or a
// hardware time limit passes, so the loop wakes as soon as the barrier
// flips; only waits longer than 2^16 cycles (never in steady state) add a
// sleep to leave issue slots to the working warps.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long timeout, int* err,
                                          int code, const volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        const long long dt = clock64() - t0;
        if (dt > timeout) {
            atomicCAS(err, 0, code);
            return false;
        }
        if (dt > 65536) __nanosleep(256);
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
// One lane of a converged warp (the same lane every time: the lowest).
__device__ __forceinline__ bool elect_one() {
    uint32_t pred = 0;
    asm volatile("{\n.reg .pred P;\nelect.sync _|P, 0xffffffff;\nselp.u32 %0, 1, 0, P;\n}\n" : "=r"(pred));
    return pred != 0;
}

// ------------------------------------------------------------ shared layout

struct Layout {
    int nrb;            // 128-row blocks of operand A per step
    int ndig;           // digit stages
    int ne;             // exponent entries: P + Qp
    uint32_t a_bytes;   // operand A bytes per step
    uint32_t b_bytes;   // operand B bytes per step
    uint32_t stage;     // digit stage bytes (1024-aligned)
    uint32_t dig_off;   // offset of digit stage 0
    uint32_t acc_off;   // 64-bit integer accumulators [Qp][128]
    uint32_t exps_off;  // per-stage column exponents [ndig][ne]
    uint32_t snap_off;  // per-tile exponent snapshots [NEXP][ne]
    uint32_t misc_off;  // barriers, flags, tmem slot
    uint32_t total;
};

constexpr uint32_t kSmemBudget = 227u * 1024u;  // one CTA per SM
constexpr uint32_t kSmemPerSM = 228u * 1024u;   // shared by the CTAs of an SM, 1 KB reserved per CTA
constexpr uint32_t kMiscBytes = 256u;

__host__ __device__ inline Layout make_layout(int P, int Qp, int Qw, int stacked, uint32_t budget,
                                              uint32_t floor_bytes, int S) {
    Layout L;
    L.nrb = stacked ? (S + 1) / 2 : S;
    L.ne = P + Qp;
    L.a_bytes = (uint32_t)L.nrb * 4096u;
    L.b_bytes = (uint32_t)S * Qp * 32u;
    L.stage = ((L.a_bytes + L.b_bytes) + 1023u) & ~1023u;
    const uint32_t acc = (uint32_t)Qp * 128u * 8u;
    const uint32_t exps = (uint32_t)L.ne * 4u;
    const uint32_t fixed = acc + NEXP * exps + kMiscBytes + 256u;  // + alignment slack
    int ndig = budget > fixed ? (int)((budget - fixed) / (L.stage + exps)) : 0;
    if (ndig > NDIG_MAX) ndig = NDIG_MAX;
    L.ndig = ndig;  // the host rejects fewer than 2
    L.dig_off = 0;
    L.acc_off = L.dig_off + (uint32_t)ndig * L.stage;
    L.exps_off = L.acc_off + acc;
    L.snap_off = L.exps_off + (uint32_t)ndig * exps;
    L.misc_off = (L.snap_off + NEXP * exps + 127u) & ~127u;
    L.total = L.misc_off + kMiscBytes;
    if (L.total < floor_bytes) L.total = floor_bytes;  // no more CTAs per SM than tensor memory was split for
    return L;
}

// misc area: byte offsets of the barriers and flags
enum {
    M_DIG_FULL = 0,     // NDIG_MAX x 8
    M_DIG_EMPTY = 48,   // NDIG_MAX x 8
    M_EXP_EMPTY = 96,   // NEXP x 8
    M_TILE_FULL = 128,
    M_TMEM_EMPTY = 136,
    M_MMA_DONE = 144,
    M_TMEM_SLOT = 152,
    M_CHG = 160,        // NDIG_MAX ints: last step whose conversion grew a column exponent
    M_ABORT = 184,
    M_TILE_INFO = 188,  // slot | last << 8 | empty << 9 | exponents changed << 10
};
static_assert(M_TILE_INFO + 4 <= (int)kMiscBytes, "misc area");

// ------------------------------------------------------------ digit maths

// |x| as a fixed-point integer with 8S - 1 bits below 2^e (truncated), plus
// the S - 1 low bytes biased by 0x80 so that they read back as balanced
// digits: returns Y = X + 0x80...80 where X = floor(|x| 2^(8S-1-e)) <
// 2^(8S-1).  The S base-256 digits of X = sum_s d_s 2^(8(S-1-s)) are
// d_0 = byte S-1 of Y in [0, 128] and d_s = byte (S-1-s) of Y - 128 in
// [-128, 127] for s >= 1.  Requires |x| < 2^e; subnormals are exact (no
// implicit bit); values below the column's range give 0 (the shift is
// clamped to 63).
template <int S>
__device__ __forceinline__ unsigned long long fixed_digits(double x, int e, uint32_t* sign) {
    constexpr unsigned long long kBias = ((1ull << (8 * (S - 1))) - 1) / 255 * 0x80;  // 0x80 in S-1 bytes
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(bits >> 32);
    *sign = hi & 0x80000000u;
    const int ef = (int)((hi >> 20) & 0x7FFu);
    const uint32_t mhi = (hi & 0xFFFFFu) | (ef ? 0x100000u : 0u);
    const unsigned long long mant = ((unsigned long long)mhi << 32) | (uint32_t)bits;
    const int sh = min(e + 1076 - 8 * S - max(ef, 1), 63);
    return (mant >> sh) + kBias;
}

// fixed_digits for columns whose running exponent e exceeds -960, with the
// shift base Eb = e + 1076 - 8S precomputed per column: the implicit bit is
// set unconditionally, which changes nothing here, since a zero or
// subnormal x (exponent field 0) then shifts by at least 63 and gives 0, as
// its exact value (|x| < 2^-1022, so |x| 2^(8S-1-e) < 2^-15) does.
template <int S>
__device__ __forceinline__ unsigned long long fixed_digits_fast(double x, int Eb, uint32_t* sign) {
    constexpr unsigned long long kBias = ((1ull << (8 * (S - 1))) - 1) / 255 * 0x80;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(bits >> 32);
    *sign = hi & 0x80000000u;
    const int ef = (int)((hi >> 20) & 0x7FFu);
    const uint32_t mhi = (hi & 0xFFFFFu) | 0x100000u;
    const unsigned long long mant = ((unsigned long long)mhi << 32) | (uint32_t)bits;
    return (mant >> min(Eb - ef, 63)) + kBias;
}

// The S fp16 slices of two values a (row r) and b (row r + 1) of one
// column, packed per slice as (a, b) in one 32-bit word, sign applied.  A
// digit byte placed under the fp16 exponent of 1024 (0x64XX) is 1024 + byte
// exactly.  Byte permutes gather the digit bytes of both values two slices at
// a time and place them under 0x64; one packed fused multiply-add then forms
// sign * (1024 + byte) - sign * bias, bias = 1024 for the top digit and 1152
// (1024 + 128) for the balanced low digits: exact, since every result is a
// small integer.  Slice s is byte S - 1 - s of Y.
// FAST: `e` is the shift base of fixed_digits_fast instead of the exponent.
template <int S, bool FAST>
__device__ __forceinline__ void split_pair(double xa, double xb, int e, uint32_t* w) {
    uint32_t sa, sb;
    const unsigned long long ya = FAST ? fixed_digits_fast<S>(xa, e, &sa) : fixed_digits<S>(xa, e, &sa);
    const unsigned long long yb = FAST ? fixed_digits_fast<S>(xb, e, &sb) : fixed_digits<S>(xb, e, &sb);
    const uint32_t alo = (uint32_t)ya, ahi = (uint32_t)(ya >> 32);
    const uint32_t blo = (uint32_t)yb, bhi = (uint32_t)(yb >> 32);
    const uint32_t sg = (sa >> 16) | sb;       // sign of a in bit 15, of b in bit 31
    const uint32_t k64 = 0x64646464u;
    const uint32_t mul = 0x3C003C00u | sg;     // (+-1.0, +-1.0)
    const uint32_t c_top = 0xE400E400u ^ sg;   // -1024 * sign
    const uint32_t c_low = 0xE480E480u ^ sg;   // -1152 * sign
    // [b5 a5 b4 a4], [b3 a3 b2 a2], [b1 a1 b0 a0] (byte n of Y written an, bn)
    const uint32_t m45 = __byte_perm(ahi, bhi, 0x5140);
    const uint32_t m23 = __byte_perm(alo, blo, 0x7362);
    const uint32_t m01 = __byte_perm(alo, blo, 0x5140);
    auto fin = [&](uint32_t pair, uint32_t sel, uint32_t add) {
        uint32_t u = __byte_perm(pair, k64, sel);  // [0x64 b 0x64 a]
        __half2 h = __hfma2(*reinterpret_cast<__half2*>(&u), *reinterpret_cast<const __half2*>(&mul),
                            *reinterpret_cast<const __half2*>(&add));
        return *reinterpret_cast<uint32_t*>(&h);
    };
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int y = S - 1 - sl;  // byte of Y
        const uint32_t pair = y >= 4 ? m45 : (y >= 2 ? m23 : m01);
        w[sl] = fin(pair, (y & 1) ? 0x4342u : 0x4140u, sl == 0 ? c_top : c_low);
    }
}

// W = sum_d P_d 2^(8(S-1-d)) for accumulator entry qq of the S blocks v[j]
// (tensor-memory words, FP32 integers): block j holds weight d = j + H (rows
// of the second stacked slice: H = 1; their d = S block is dropped).  The
// terms shifted by 32 or more bits (P_0 2^8 + P_1 for S = 6, P_0 for S = 5)
// are summed in 32 bits (|P_0| <= 2^22, |P_1| <= 2^23), the rest are exact
// 64-bit multiply-adds.
template <int H, int S>
__device__ __forceinline__ long long combine_w(const uint32_t (&v)[S][8], int qq) {
    int pd[S];
#pragma unroll
    for (int d = 0; d < S; ++d) pd[d] = d >= H ? __float2int_rn(__uint_as_float(v[d - H][qq])) : 0;
    long long lo = 0;
    int hi = 0;
#pragma unroll
    for (int d = 0; d < S; ++d) {
        const int sh = 8 * (S - 1 - d);
        if (sh >= 32)
            hi += pd[d] * (1 << (sh - 32));
        else
            lo += (long long)pd[d] * (1ll << sh);
    }
    return (long long)((unsigned long long)lo + ((unsigned long long)(unsigned int)hi << 32));
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

template <int R, int S>
__global__ void __launch_bounds__(block_threads<R>(), 1) k_split(const Params prm) {
    constexpr int PER = 1;  // units per converter thread
    constexpr int DEPTH = Conv<R>::DEPTH;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int P = prm.P;
    const int kr = blockIdx.x / prm.n_qc, qc = blockIdx.x - kr * prm.n_qc;
    // (selects, not an indexed load: indexing the parameter arrays would
    // copy the whole parameter block to local memory)
    const int q0 = qc ? prm.q0[1] : prm.q0[0];
    const int Qw = qc ? prm.qw[1] : prm.qw[0];
    const int Qp = prm.Qp;
    const int64_t Ktot = prm.K;
    const int stacked = prm.stacked;
    const Layout L = make_layout(P, Qp, Qw, stacked, (uint32_t)prm.smem_budget, (uint32_t)prm.smem_floor, S);
    const int NE = L.ne, ndig = L.ndig;
    unsigned char* dig = smem + L.dig_off;
    long long* iacc = reinterpret_cast<long long*>(smem + L.acc_off);
    int* exps = reinterpret_cast<int*>(smem + L.exps_off);
    int* snap = reinterpret_cast<int*>(smem + L.snap_off);
    unsigned char* misc = smem + L.misc_off;
    const uint32_t misc_a = smem_addr(misc);
    auto bar = [&](int off) { return misc_a + (uint32_t)off; };
    volatile int* chg_step = reinterpret_cast<volatile int*>(misc + M_CHG);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + M_ABORT);
    volatile int* tile_info = reinterpret_cast<volatile int*>(misc + M_TILE_INFO);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long tmo = prm.timeout;
    const int NCONV = prm.nconv, NCONV_WARPS = NCONV / 32;
    const int MMA_WARP = NCONV_WARPS, EPI_WARP0 = NCONV_WARPS + 1;
    const int NTHREADS = blockDim.x;

    // K range of this CTA, in 16-row steps
    const int64_t steps_total = (Ktot + KSTEP - 1) / KSTEP;
    const int64_t s_begin = (int64_t)kr * prm.steps_per_kr;
    int64_t s_end = s_begin + prm.steps_per_kr;
    if (s_end > steps_total) s_end = steps_total;
    const int64_t nsteps = s_end > s_begin ? s_end - s_begin : 0;

    // ---- set-up: zero everything up to the barriers; init barriers
    for (uint32_t i = threadIdx.x * 16u; i < L.misc_off + kMiscBytes; i += NTHREADS * 16u)
        *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < ndig; ++i) {
            mbar_init(bar(M_DIG_FULL + 8 * i), NCONV_WARPS);
            mbar_init(bar(M_DIG_EMPTY + 8 * i), 1);
            chg_step[i] = -1;
        }
        for (int i = 0; i < NEXP; ++i) mbar_init(bar(M_EXP_EMPTY + 8 * i), prm.nepi);
        mbar_init(bar(M_TILE_FULL), 1);
        mbar_init(bar(M_TMEM_EMPTY), prm.nepi);
        mbar_init(bar(M_MMA_DONE), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    fence_proxy_async();
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         bar(M_TMEM_SLOT)),
                     "r"(prm.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(misc + M_TMEM_SLOT);

    if (warp < NCONV_WARPS) {
        // ================================================= converters
        // Unit u = threadIdx.x of every step.  R = 8: rows 8g .. 8g + 7 of
        // the step (g = (u / 16) % 2) of column slot c = 16 (u / 32) + u % 16;
        // its 8 digits of one slice are the 16 contiguous bytes of one
        // K-major core-matrix row, written with a single 16-byte store, and
        // a warp's store covers 512 contiguous bytes (four core matrices);
        // the two units of a column are lanes l and l ^ 16.  R = 4: rows
        // 8g + 4h .. + 3 (h = u % 2) of slot c = 8 (u / 32) + (u / 2) % 8,
        // 8-byte stores, a half-warp writing one 128-byte core row; the four
        // units of a column are lanes l, l ^ 1, l ^ 16, l ^ 17.  No bank
        // conflicts either way.  Slots [0, P) are X's columns, [P, P + Qw)
        // this chunk's Y columns; the rest are idle.
        const int ct = threadIdx.x;
        bool valid[PER];
        const char* src[PER];   // column base
        int64_t ldb[PER];       // row stride in bytes
        int rq[PER];            // first row of the unit within a step
        uint32_t off0[PER], dsl[PER];  // stage offset of slice 0 and the per-slice stride
        int e[PER];
        int col[PER];           // exponent index: X columns, then Y columns
        bool owner[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int u = ct + i * NCONV;
            const int slot = R == 8 ? 16 * (u >> 5) + (u & 15) : 8 * (u >> 5) + ((u >> 1) & 7);
            const int g = (u >> 4) & 1, hb = R == 8 ? 0 : (u & 1);
            const bool is_x = slot < P, is_y = slot >= P && slot < P + Qw;
            valid[i] = is_x || is_y;
            const int c = valid[i] ? slot : 0;  // X columns, then Y columns
            rq[i] = 8 * g + 4 * hb;
            owner[i] = valid[i] && g == 0 && hb == 0;
            col[i] = c;
            e[i] = E_NONE;
            if (c < P) {
                src[i] = reinterpret_cast<const char*>(prm.X + c);
                ldb[i] = prm.ldx * 8;
                // slice s in operand-A block (stacked ? s / 2 : s), row (stacked ? (s % 2) * 64 : 0) + c
                off0[i] = kmajor_off(c, g) + 8 * hb;
                dsl[i] = stacked ? 2048u : 4096u;
            } else {
                src[i] = reinterpret_cast<const char*>(prm.Y + q0 + (c - P));
                ldb[i] = prm.ldy * 8;
                off0[i] = L.a_bytes + kmajor_off(c - P, g) + 8 * hb;
                dsl[i] = (uint32_t)Qp * 32u;
            }
        }
        // loads of step s (zero beyond this CTA's steps and beyond row K);
        // whole steps inside the matrix skip the per-row bounds checks
        auto load_step = [&](double(&v)[PER][R], int64_t s) {
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int64_t k = (s_begin + s) * KSTEP + rq[i];
                const bool live = valid[i] && s < nsteps;
                const int64_t left = live ? Ktot - k : 0;
                const char* p = src[i] + (live ? k : 0) * ldb[i];
                if (left >= R) {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[i][r] = __ldg(reinterpret_cast<const double*>(p + r * ldb[i]));
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        v[i][r] = left > r ? __ldg(reinterpret_cast<const double*>(p + r * ldb[i])) : 0.0;
                }
            }
        };
        int d = 0;
        uint32_t phase = 0;
        bool fast = false;  // every valid column's exponent above -960 (set when one grows)
        // converts step s from registers into digit stage d; false: stop
        auto convert_step = [&](const double(&v)[PER][R], int64_t s) -> bool {
            // -- running column exponents (registers; the lanes of a column agree)
            bool grew = false;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                uint32_t hm = 0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    hm = max(hm, (uint32_t)((unsigned long long)__double_as_longlong(v[i][r]) >> 32) & 0x7FFFFFFFu);
                if (R == 4) hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, 1));
                hm = max(hm, __shfl_xor_sync(0xffffffffu, hm, 16));
                const int em = exp_from_hi(hm);
                if (valid[i] && em > e[i]) {
                    e[i] = em;
                    grew = true;
                }
            }
            grew = __any_sync(0xffffffffu, grew);
            if (grew) {
                bool tiny = false;
#pragma unroll
                for (int i = 0; i < PER; ++i) tiny |= valid[i] && e[i] <= -960;
                fast = !__any_sync(0xffffffffu, tiny);
            }
            // -- the stage must be free (waited by lane 0, broadcast: warp-uniform)
            int w_ok = 1;
            if (lane == 0)
                w_ok = mbar_wait(bar(M_DIG_EMPTY + 8 * d), phase ^ 1u, tmo, prm.err, 2, abort_flag);
            if (!__shfl_sync(0xffffffffu, w_ok, 0)) {
                *abort_flag = 1;
                return false;
            }
            if (grew && lane == 0) chg_step[d] = (int)s;
            int* ex = exps + d * NE;
            unsigned char* stage = dig + d * L.stage;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                if (!valid[i]) continue;
                if (owner[i]) ex[col[i]] = e[i];
                uint32_t w[S][R / 2];
                if (fast) {  // warp-uniform
                    const int eb = e[i] + 1076 - 8 * S;
#pragma unroll
                    for (int r = 0; r < R; r += 2) {
                        uint32_t wp[S];
                        split_pair<S, true>(v[i][r], v[i][r + 1], eb, wp);
#pragma unroll
                        for (int sl = 0; sl < S; ++sl) w[sl][r >> 1] = wp[sl];
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < R; r += 2) {
                        uint32_t wp[S];
                        split_pair<S, false>(v[i][r], v[i][r + 1], e[i], wp);
#pragma unroll
                        for (int sl = 0; sl < S; ++sl) w[sl][r >> 1] = wp[sl];
                    }
                }
#pragma unroll
                for (int sl = 0; sl < S; ++sl) {
                    if (R == 8)
                        *reinterpret_cast<uint4*>(stage + off0[i] + sl * dsl[i]) =
                            make_uint4(w[sl][0], w[sl][1], w[sl][R == 8 ? 2 : 0], w[sl][R == 8 ? 3 : 1]);
                    else
                        *reinterpret_cast<uint2*>(stage + off0[i] + sl * dsl[i]) = make_uint2(w[sl][0], w[sl][1]);
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(M_DIG_FULL + 8 * d));
            if (++d == ndig) {
                d = 0;
                phase ^= 1u;
            }
            return true;
        };
        // DEPTH + 1 register sets in rotation: while step s is converted,
        // the loads of steps s + 1 .. s + DEPTH are in flight
        double buf[DEPTH + 1][PER][R];
#pragma unroll
        for (int j = 0; j < DEPTH; ++j) load_step(buf[j], j);
        bool alive = true;
        for (int64_t s0 = 0; s0 < nsteps && alive; s0 += DEPTH + 1) {
#pragma unroll
            for (int j = 0; j <= DEPTH; ++j) {
                const int64_t s = s0 + j;
                if (alive && s < nsteps) {
                    load_step(buf[(j + DEPTH) % (DEPTH + 1)], s + DEPTH);
                    alive = convert_step(buf[j], s) && !*abort_flag;
                }
            }
        }
    } else if (warp == MMA_WARP) {
        // ================================================= MMA issuer
        // The warp runs the loop; waits are taken by lane 0 and broadcast,
        // tcgen05 operations are issued by one elected lane.  The MMAs of a
        // step are the same for every step up to the stage base address, so
        // their descriptors are built once, in registers (issuing them from
        // a per-MMA computation costs several times the MMA itself).
        int64_t tile = -1;
        int steps_in_tile = 0, cur_slot = 0, cur_chg = 0;
        bool failed = false;
        uint32_t mma_phase = 0, phase = 0;
        int d = 0;
        const uint32_t dig_a = smem_addr(dig);
        uint64_t adesc[MAX_MMAS], bdesc[MAX_MMAS];
        uint32_t dtm[MAX_MMAS], idesc[MAX_MMAS];
        uint32_t first_mask = 0;  // MMAs of row block 0: they start a tile's accumulators
        int nmma = 0;
        {
            const int maxs = 256 / Qp;  // slices per MMA (N <= 256)
            int rb = 0, t0 = 0;
#pragma unroll
            for (int j = 0; j < MAX_MMAS; ++j) {
                const int s_a = stacked ? 2 * rb : rb;  // first slice index of this row block
                const int nt = S - s_a;                 // slices t with s_a + t <= S - 1
                const bool live = rb < L.nrb;
                const int cnt = min(maxs, nt - t0);
                adesc[j] = smem_desc(dig_a + (uint32_t)rb * 4096u, 128, 256);
                bdesc[j] = smem_desc(dig_a + L.a_bytes + (uint32_t)(t0 * Qp * 32), 128, 256);
                dtm[j] = tmem + (uint32_t)((s_a + t0) * Qp);
                idesc[j] = instr_desc(live ? cnt * Qp : 16);
                if (live && rb == 0) first_mask |= 1u << j;
                nmma += live ? 1 : 0;
                t0 += maxs;
                if (t0 >= nt) {
                    ++rb;
                    t0 = 0;
                }
            }
        }
        auto lane0_wait = [&](uint32_t b, uint32_t par, int code) {
            int ok = 1;
            if (lane == 0) ok = mbar_wait(b, par, tmo, prm.err, code, abort_flag);
            return __shfl_sync(0xffffffffu, ok, 0) != 0;
        };
        for (int64_t s = 0; s < nsteps; ++s) {
            if (!lane0_wait(bar(M_DIG_FULL + 8 * d), phase, 3)) {
                failed = true;
                break;
            }
            tc_fence_after();
            const bool chg = chg_step[d] == (int)s;
            const bool new_tile = tile < 0 || chg || steps_in_tile >= TILE_STEPS;
            if (new_tile) {
                if (tile >= 0) {
                    // hand the finished tile to the epilogue
                    if (elect_one()) mma_commit(bar(M_MMA_DONE));
                    __syncwarp();
                    if (!lane0_wait(bar(M_MMA_DONE), mma_phase, 4)) {
                        failed = true;
                        break;
                    }
                    mma_phase ^= 1;
                    if (lane == 0) {
                        *tile_info = cur_slot | (cur_chg << 10);
                        tc_fence_before();
                        mbar_arrive(bar(M_TILE_FULL));
                    }
                    if (!lane0_wait(bar(M_TMEM_EMPTY), (uint32_t)(tile & 1), 5)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                }
                ++tile;
                steps_in_tile = 0;
                cur_slot = (int)(tile % NEXP);
                cur_chg = chg ? 1 : 0;
                if (!lane0_wait(bar(M_EXP_EMPTY + 8 * cur_slot), (uint32_t)(((tile / NEXP) & 1) ^ 1), 8)) {
                    failed = true;
                    break;
                }
                const int* ex = exps + d * NE;
                int* sn = snap + cur_slot * NE;
                for (int i = lane; i < NE; i += 32) sn[i] = ex[i];
                __syncwarp();
            }
            ++steps_in_tile;
            // stage d's operands: the same descriptors moved by d stages (the
            // address field counts 16-byte units and stays below 2^14)
            const uint64_t so = (uint64_t)(((uint32_t)d * L.stage) >> 4);
            const uint32_t keep = new_tile ? ~first_mask : ~0u;
            if (elect_one()) {
#pragma unroll
                for (int j = 0; j < MAX_MMAS; ++j)
                    if (j < nmma) mma_f16(dtm[j], adesc[j] + so, bdesc[j] + so, idesc[j], (keep >> j) & 1u);
                mma_commit(bar(M_DIG_EMPTY + 8 * d));
            }
            __syncwarp();
            if (++d == ndig) {
                d = 0;
                phase ^= 1u;
            }
        }
        // last tile (or drain after a failure): no MMA may be in flight at exit
        if (elect_one()) mma_commit(bar(M_MMA_DONE));
        __syncwarp();
        if (lane == 0) {
            const bool drained = mbar_wait(bar(M_MMA_DONE), mma_phase, kDefaultTimeout, prm.err, 6, nullptr);
            if (!failed && drained && tile >= 0) {
                *tile_info = cur_slot | (1 << 8) | (cur_chg << 10);
                tc_fence_before();
                mbar_arrive(bar(M_TILE_FULL));
            } else if (tile < 0 && !failed) {
                *tile_info = 1 << 9;  // empty range: nothing to drain
                mbar_arrive(bar(M_TILE_FULL));
            } else {
                *abort_flag = 1;  // the epilogue stops waiting
            }
        }
        __syncwarp();
    } else {
        // ================================================= epilogue
        // Per (lane, column): an exact 64-bit integer sum of the tiles' W in
        // shared memory, at the scale of the current column exponents.  It
        // moves to binary64 (`flush`, this thread's own entries in global
        // memory) only when an exponent grows, when the integer sum would
        // overflow, and at the end -- not once per tile.  With 8 warps,
        // warps w and w + 4 share a lane quarter and split the columns.
        const int ew = warp - EPI_WARP0;
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;  // TMEM lane = accumulator row
        const int p = stacked ? (row & 63) : row;
        const int half = stacked ? (row >> 6) : 0;
        const bool prow = p < P;
        const int qh = prm.nepi == 8 ? Qp / 2 : Qp;  // a multiple of 8
        const int qlo = (ew >> 2) * qh, qhi = qlo + qh;
        double* flush = prm.flush + (int64_t)blockIdx.x * Qp * 128;
        for (int q = qlo; q < qhi; ++q) flush[q * 128 + row] = 0.0;
        auto scaled = [](long long a, int E) {
            return (E >= -1022 && E <= 1023) ? (double)a * __longlong_as_double((long long)(E + 1023) << 52)
                                             : scalbn((double)a, E);
        };
        auto flush_all = [&](const int* exs) {
            if (!prow) return;
            const int epf = exs[p];
            for (int q = qlo; q < min(qhi, Qw); ++q) {
                const long long a = iacc[q * 128 + row];
                if (a == 0) continue;
                iacc[q * 128 + row] = 0;
                flush[q * 128 + row] += scaled(a, epf + exs[P + q] - (8 * S + 6));
            }
        };
        int prev_slot = -1;
        for (int64_t tile = 0;; ++tile) {
            int w_ok = 1;
            if (lane == 0) w_ok = mbar_wait(bar(M_TILE_FULL), (uint32_t)(tile & 1), tmo, prm.err, 7, abort_flag);
            if (!__shfl_sync(0xffffffffu, w_ok, 0)) break;
            tc_fence_after();
            const int info = *tile_info;
            if (info & (1 << 9)) break;
            const int slot = info & 0xFF;
            const bool chg = (info >> 10) & 1;
            if (prev_slot >= 0) {
                if (chg) flush_all(snap + prev_slot * NE);  // sums so far carry the old scale
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(M_EXP_EMPTY + 8 * prev_slot));
            }
            const int* ex = snap + slot * NE;
            const int ep = prow ? ex[p] : 0;
            // the weight offset of a warp's rows is warp-uniform: one loop per value
            auto drain = [&](auto half_tag) {
                constexpr int H = decltype(half_tag)::value;
                for (int qb = qlo; qb < qhi; qb += 8) {
                    uint32_t v[S][8];
#pragma unroll
                    for (int j = 0; j < S; ++j)
                        tmem_ld8(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(j * Qp + qb), v[j]);
                    tmem_wait_ld();
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int q = qb + qq;
                        if (!prow || q >= Qw) continue;
                        const long long W = combine_w<H, S>(v, qq);
                        if (W == 0) continue;
                        long long* ap = &iacc[q * 128 + row];
                        const long long a = *ap;
                        long long sum = (long long)((unsigned long long)a + (unsigned long long)W);
                        if (((a ^ sum) & (W ^ sum)) < 0) {  // would overflow: move a to binary64
                            flush[q * 128 + row] += scaled(a, ep + ex[P + q] - (8 * S + 6));
                            sum = W;
                        }
                        *ap = sum;
                    }
                }
            };
            if (half)
                drain(std::integral_constant<int, 1>());
            else
                drain(std::integral_constant<int, 0>());
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(prm.tmem_cols));
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

// MMAs per step for a chunk width Qp: the kernel builds at most MAX_MMAS.
int count_mmas(int stacked, int Qp, int S) {
    const int maxs = 256 / Qp;
    int n = 0;
    for (int rb = 0; rb < (stacked ? (S + 1) / 2 : S); ++rb) {
        const int nt = S - (stacked ? 2 * rb : rb);
        n += (nt + maxs - 1) / maxs;
    }
    return n;
}

}  // namespace split

tsm_status validate_common(int dtype, int M, int N, int64_t K, const double* alpha, const double* beta);

}  // namespace tsm

using namespace tsm;

namespace tsm {
namespace split {

// Everything about a launch that depends on the shape only.
struct Plan {
    Params prm;     // shape fields filled; pointers, workspace and timeout are the caller's
    Layout L;
    int S = 6;      // slices per input
    int per = 8;    // rows per converter unit (R)
    int cps = 0;    // CTAs per SM
    int threads = 0;
    const void* fn = nullptr;
};

// The kernel instantiation for (units per thread, slices).
const void* kernel_for(int R, int S) {
    if (R == 4) return S == 4 ? (const void*)k_split<4, 4> : S == 5 ? (const void*)k_split<4, 5>
                                                                     : (const void*)k_split<4, 6>;
    return S == 4 ? (const void*)k_split<8, 4> : S == 5 ? (const void*)k_split<8, 5> : (const void*)k_split<8, 6>;
}

tsm_status make_plan(int cplx, int M, int N, int64_t K, int S, Plan* pl) {
    if (S < 4 || S > NSLICE_MAX) return TSM_ERR_NOT_SUPPORTED;
    pl->S = S;
    const DeviceInfo& di = device_info();
    Params& prm = pl->prm;
    const int c = cplx ? 2 : 1;
    const int P = M * c, Q = N * c;
    prm.P = P;
    prm.Q = Q;
    prm.K = K;
    prm.stacked = P <= 64 ? 1 : 0;
    // Y column chunks: one if S slices of it fit tensor memory (512
    // columns) and its conversion units fit the converter warps, else two
    // chunks split on an even column
    if (((Q + 15) & ~15) * S <= TMEM_COLS_MAX && conv_threads(P + Q, 8) <= Conv<8>::MAX_THREADS) {
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
    const int qmax = prm.qw[0] > prm.qw[1] ? prm.qw[0] : prm.qw[1];
    prm.Qp = (qmax + 15) & ~15;
    if (count_mmas(prm.stacked, prm.Qp, S) > MAX_MMAS) return TSM_ERR_NOT_SUPPORTED;

    // CTA shape.  Accumulators take S * Qp tensor-memory columns; the
    // allocation is the next power of two, so narrow chunks leave room for
    // several CTAs per SM, which then overlap one another's waits (drains,
    // load latency).  Shared memory is split between them and padded so that
    // no more CTAs than planned share an SM (a further one would block in its
    // tensor-memory allocation).
    int tcols = 32;
    while (tcols < S * prm.Qp) tcols <<= 1;
    prm.tmem_cols = tcols;
    // unit rows: 4 (more converter threads) when they fit, else 8
    pl->per = conv_threads(P + qmax, 4) <= Conv<4>::MAX_THREADS ? 4 : 8;
    prm.nconv = conv_threads(P + qmax, pl->per);
    if (prm.nconv > (pl->per == 4 ? Conv<4>::MAX_THREADS : Conv<8>::MAX_THREADS)) return TSM_ERR_NOT_SUPPORTED;
    pl->fn = kernel_for(pl->per, S);
    if (cudaFuncSetAttribute(pl->fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
        return TSM_ERR_LAUNCH;
    int cps_max = TMEM_COLS_MAX / tcols;
    if (cps_max > 4) cps_max = 4;
    // Co-residency is counted here from the kernel's registers and the SM's
    // limits (the occupancy query reports one CTA for this kernel although
    // two measurably run together): registers per warp are allocated in
    // units of 256 from each of the 4 sub-partitions' 16K, and every CTA's
    // shared memory carries a 1 KB reserve.
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, pl->fn) != cudaSuccess) return TSM_ERR_LAUNCH;
    const int regs_per_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int warps_per_sm = regs_per_warp > 0 ? 4 * (16384 / regs_per_warp) : 64;
    auto fits = [&](int thr, uint32_t smem) {
        const int by_regs = warps_per_sm / (thr / 32);
        const int by_smem = (int)(kSmemPerSM / (smem + 1024u));
        const int by_thr = 2048 / thr;
        return min(min(by_regs, by_smem), min(by_thr, 32));
    };
    pl->cps = 0;
    for (int cc = cps_max; cc >= 1 && !pl->cps; --cc) {
        // several CTAs per SM share the drains: 4 epilogue warps each; alone, 8
        const int nepi = cc > 1 ? 4 : 8;
        const int thr = prm.nconv + (1 + nepi) * 32;
        const uint32_t budget = cc == 1 ? kSmemBudget : ((kSmemPerSM / cc - 1024u) & ~127u);
        const uint32_t floor_b = kSmemPerSM / (cc + 1);
        const Layout L = make_layout(P, prm.Qp, qmax, prm.stacked, budget, floor_b, S);
        if (L.ndig < (cc > 1 ? 3 : 2) || L.total > (uint32_t)di.smem_optin) continue;
        if (fits(thr, L.total) == cc) {
            pl->cps = cc;
            pl->threads = thr;
            pl->L = L;
            prm.nepi = nepi;
            prm.smem_budget = (int)budget;
            prm.smem_floor = (int)floor_b;
        }
    }
    if (!pl->cps) return TSM_ERR_NOT_SUPPORTED;
    // the dynamic shared memory size of the chosen layout (the loop may have
    // set a larger one while trying more CTAs per SM)
    if (cudaFuncSetAttribute(pl->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->L.total) != cudaSuccess)
        return TSM_ERR_LAUNCH;

    const int64_t steps = (K + KSTEP - 1) / KSTEP;
    int n_kr = pl->cps * di.sm_count / prm.n_qc;
    if (n_kr < 1) n_kr = 1;
    if ((int64_t)n_kr > steps) n_kr = (int)(steps > 0 ? steps : 1);
    prm.steps_per_kr = (steps + n_kr - 1) / n_kr;
    if (prm.steps_per_kr < 1) prm.steps_per_kr = 1;
    n_kr = (int)((steps + prm.steps_per_kr - 1) / prm.steps_per_kr);
    if (n_kr < 1) n_kr = 1;
    prm.n_kr = n_kr;
    return TSM_OK;
}

}  // namespace split
}  // namespace tsm

namespace tsm {
namespace split {

tsm_status run(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha, const void* A,
               int64_t lda, const void* B, int64_t ldb, const double* beta, void* C, int64_t ldc, int kind,
               int slices, tsm_stream_t stream) {
    tsm_status st = validate_common(dtype, M, N, K, alpha, beta);
    if (st != TSM_OK) return st;
    if (kind != TSM_SPLIT_DIGITS_F16) return TSM_ERR_INVALID_VALUE;
    if (slices < 4 || slices > NSLICE_MAX) return TSM_ERR_NOT_SUPPORTED;
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
    Plan pl;
    if ((st = make_plan(cplx, M, N, K, slices, &pl)) != TSM_OK) return st;
    Params& prm = pl.prm;
    const int c = cplx ? 2 : 1;
    prm.X = (const double*)A;
    prm.ldx = lda * c;
    prm.Y = (const double*)B;
    prm.ldy = ldb * c;
    prm.timeout = g_timeout;
    const int n_kr = prm.n_kr, P = prm.P, Q = prm.Q;

    Workspace* ws = nullptr;
    const size_t part = (size_t)n_kr * P * Q * sizeof(double);
    const size_t flush = (size_t)n_kr * prm.n_qc * prm.Qp * 128 * sizeof(double);
    if ((st = workspace_get(s, part + flush + 256, 1, &ws)) != TSM_OK) return st;
    prm.ws = ws->partials;
    prm.flush = ws->partials + (size_t)n_kr * P * Q;
    prm.err = reinterpret_cast<int*>(ws->tickets) + 32;  // error word of this stream
    if (cudaMemsetAsync(prm.err, 0, sizeof(int), s) != cudaSuccess) return TSM_ERR_LAUNCH;
    void* args[] = {&prm};
    if (cudaLaunchKernel(pl.fn, dim3(n_kr * prm.n_qc), dim3(pl.threads), args, pl.L.total, s) != cudaSuccess)
        return TSM_ERR_LAUNCH;
    const int outs = M * N;
    k_split_combine<<<(outs + 127) / 128, 128, 0, s>>>(
        ws->partials, n_kr, P, Q, M, N, cplx, (cplx && opA == TSM_OP_C) ? 1 : 0, alpha[0], cplx ? alpha[1] : 0.0,
        beta[0], cplx ? beta[1] : 0.0, beta_zero, (double*)C, ldc, prm.err);
    if (cudaGetLastError() != cudaSuccess) return TSM_ERR_LAUNCH;
    return TSM_OK;
}

}  // namespace split
}  // namespace tsm

extern "C" tsm_status tsm_tsmttsm_split(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K,
                                        const double* alpha, const void* A, int64_t lda, const void* B,
                                        int64_t ldb, const double* beta, void* C, int64_t ldc,
                                        tsm_stream_t stream) {
    return split::run(opA, dtype, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, TSM_SPLIT_DIGITS_F16, 6, stream);
}

extern "C" tsm_status tsm_tsmttsm_split_ex(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K,
                                           const double* alpha, const void* A, int64_t lda, const void* B,
                                           int64_t ldb, const double* beta, void* C, int64_t ldc,
                                           tsm_split_kind kind, int slices, tsm_stream_t stream) {
    return split::run(opA, dtype, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, kind, slices, stream);
}

extern "C" tsm_status tsm_split_plan_ex(tsm_dtype dtype, int M, int N, int64_t K, int slices,
                                        tsm_split_plan_info* info) {
    if (!info || (dtype != TSM_R64 && dtype != TSM_C64) || K < 1) return TSM_ERR_INVALID_VALUE;
    if (M < 1 || N < 1 || M > 64 || N > 64 || slices < 4 || slices > split::NSLICE_MAX)
        return TSM_ERR_NOT_SUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSM_ERR_NO_DEVICE;
    const DeviceInfo& di = device_info();
    if (di.cc_major != 10 || di.cc_minor != 3) return TSM_ERR_NO_DEVICE;
    split::Plan pl;
    const tsm_status st = split::make_plan(dtype == TSM_C64, M, N, K, slices, &pl);
    if (st != TSM_OK) return st;
    info->ctas = pl.prm.n_kr * pl.prm.n_qc;
    info->ctas_per_sm = pl.cps;
    info->column_chunks = pl.prm.n_qc;
    info->converter_threads = pl.prm.nconv;
    info->epilogue_warps = pl.prm.nepi;
    info->threads_per_cta = pl.threads;
    info->digit_stages = pl.L.ndig;
    info->tmem_columns = pl.prm.tmem_cols;
    info->smem_bytes = (int)pl.L.total;
    return TSM_OK;
}

extern "C" tsm_status tsm_split_plan(tsm_dtype dtype, int M, int N, int64_t K, tsm_split_plan_info* info) {
    return tsm_split_plan_ex(dtype, M, N, K, 6, info);
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
