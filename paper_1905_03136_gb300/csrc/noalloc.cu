// TSMTTSM without device allocations: the per-CTA partial sums and the
// reduction ticket of the deterministic two-level reduction live in one
// fixed array compiled into the library, instead of the per-stream
// workspace that tsm_tsmttsm() grows with cudaMalloc.  For callers that must
// not allocate (memory arenas that own the device, paths that cannot afford
// the device synchronization a cudaMalloc implies).
#include <mutex>

#include "tsm_internal.h"
#include "tsm_noalloc.h"
#include "tune.h"

// Scratch of the allocation-free entry point (held by every GPU that loads
// the library, until exit).  In host code this name is only a handle: its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TSM_NOALLOC_SCRATCH_BYTES];

namespace tsm {

tsm_status validate_common(int dtype, int M, int N, int64_t K, const double* alpha, const double* beta);
tsm_status choose(tsm_kind kind, int dtype, int M, int N, int64_t K, int* variant, int* grid);

namespace {

std::mutex g_mu;
void* g_scratch_dev[64] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device with that device current.
tsm_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TSM_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TSM_ERR_LAUNCH;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return TSM_OK;
}

}  // namespace
}  // namespace tsm

using namespace tsm;

extern "C" tsm_status tsm_tsmttsm_noalloc(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K,
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
    cudaStream_t s = (cudaStream_t)stream;
    const int beta_zero = beta[0] == 0.0 && (!cplx || beta[1] == 0.0);
    if (K == 0 || alpha0)
        return launch_scale_small((double*)C, M, N, ldc, cplx, beta[0], cplx ? beta[1] : 0.0, beta_zero, s) ==
                       cudaSuccess
                   ? TSM_OK
                   : TSM_ERR_LAUNCH;

    int variant = -1, grid = 0;
    if ((st = choose(TSM_KIND_TSMTTSM, dtype, M, N, K, &variant, &grid)) != TSM_OK) return st;
    const Variant* var = variant_at(TSM_KIND_TSMTTSM, variant);
    if (!var || !var->tsmttsm) return TSM_ERR_INTERNAL;

    // The tuned grid, capped so that the CTA partial sums fit the array (its
    // last 256 bytes hold the ticket); a capped grid stays a multiple of the
    // SM count.  Only a shape whose partials do not fit even at one CTA per
    // SM is refused.
    const size_t per_cta = (size_t)M * N * (cplx ? 2 : 1) * sizeof(double);
    const size_t max_ctas = ((size_t)TSM_NOALLOC_SCRATCH_BYTES - 256) / per_cta;
    if (max_ctas < (size_t)di.sm_count) return TSM_ERR_NOT_SUPPORTED;
    if (grid > 65535) grid = 65535;
    if ((size_t)grid > max_ctas) grid = (int)(max_ctas / di.sm_count) * di.sm_count;

    void* scratch = nullptr;
    if ((st = scratch_address(&scratch)) != TSM_OK) return st;
    unsigned* ticket = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(scratch) +
                                                   TSM_NOALLOC_SCRATCH_BYTES - 256);
    if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess) return TSM_ERR_LAUNCH;

    TsmttsmArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = (const double*)A;
    a.lda = lda;
    a.B = (const double*)B;
    a.ldb = ldb;
    a.C = (double*)C;
    a.ldc = ldc;
    a.alpha_r = alpha[0];
    a.alpha_i = cplx ? alpha[1] : 0.0;
    a.beta_r = beta[0];
    a.beta_i = cplx ? beta[1] : 0.0;
    a.beta_zero = beta_zero;
    a.conj = (cplx && opA == TSM_OP_C) ? 1 : 0;
    a.ws = static_cast<double*>(scratch);
    a.ticket = ticket;
    // many partials: a separate final kernel sums them (it allocates nothing)
    a.final_pass = tsm_tsmttsm_kernels_per_call(dtype, M, N, grid) == 2 ? 1 : 0;
    // the ticket reset above already orders this launch after the previous
    // one; the record lets the next product know what this one writes
    std::lock_guard<std::mutex> lock(pdl_mutex());
    a.early = 0;
    if (var->tsmttsm(a, grid, s) != cudaSuccess) return TSM_ERR_LAUNCH;
    if (a.final_pass && launch_tsmttsm_final(a, grid, cplx, s) != cudaSuccess) return TSM_ERR_LAUNCH;
    pdl_note(s, operand_range(C, M, ldc, N, cplx), 0);
    return TSM_OK;
}
