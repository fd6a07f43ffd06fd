// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "tsm.h"

namespace tsm {

constexpr int kBlock = 256;  // threads per CTA of the FP64 kernels

// Arguments of one TSMTTSM launch (device pointers; alpha/beta by value).
struct TsmttsmArgs {
    int M, N;
    int64_t K;
    const double* A;  // K x lda (complex: interleaved pairs)
    int64_t lda;
    const double* B;  // K x ldb
    int64_t ldb;
    double* C;        // M x ldc
    int64_t ldc;
    double alpha_r, alpha_i, beta_r, beta_i;
    int beta_zero;    // 1: C is not read
    int conj;         // 1: A^H B
    double* ws;       // grid * M * N * c partial sums
    unsigned* ticket; // one counter, zero between launches
    int final_pass;   // 1: CTAs only write their partials; a separate final
                      // kernel (launch_tsmttsm_final) sums them afterwards
    int early;        // 1: A and B may be read before the previous launch on
                      // the stream completes (pdl_wait in fp64_common.cuh)
};

// Arguments of one TSMM launch.
struct TsmmArgs {
    int M, N;
    int64_t K;
    const double* A;  // K x lda
    int64_t lda;
    const double* Cm; // M x ldc
    int64_t ldc;
    double* B;        // K x ldb
    int64_t ldb;
    double alpha_r, alpha_i, beta_r, beta_i;
    int beta_zero;
    int beta_one;     // beta == 1 exactly: the old B value starts the FMA chain as it is
};

// Programmatic dependent launch.  The product kernels are launched with
// programmatic stream serialization, so the next product on the stream may
// be scheduled while this one drains; the kernels' pdl_trigger / pdl_wait
// (fp64_common.cuh) keep every dependency.  TSM_PDL=0 in the environment
// launches them the ordinary way.
bool pdl_enabled();
// Whether a launch of `grid` CTAs may start early.  A grid smaller than the
// kernel's resident capacity (occupancy x SMs) may not: its CTAs would be
// placed as the previous kernel's CTAs leave, the SMs that free up first
// taking several, and a grid sized for k CTAs per SM would run unevenly.
bool pdl_allowed(const void* kernel, int grid, int block, size_t smem);

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_allowed((const void*)kernel, grid, block, smem) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

typedef cudaError_t (*TsmttsmLaunch)(const TsmttsmArgs&, int grid, cudaStream_t);
typedef cudaError_t (*TsmmLaunch)(const TsmmArgs&, int grid, cudaStream_t);
// Resident CTAs per SM for this variant and shape (0 if it cannot run).
typedef int (*OccupancyFn)(int M, int N);

struct Variant {
    tsm_variant_info info;
    TsmttsmLaunch tsmttsm;  // exactly one of the two launchers is set
    TsmmLaunch tsmm;
    OccupancyFn occupancy;
};

// Variant tables, filled once in a fixed order (indices are stable within a
// build): hand-written families first, then code-generator output.
void register_fp64_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm);
void register_generated_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm);
void register_rt_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm);
void register_narrow_variants(std::vector<Variant>& tsmttsm, std::vector<Variant>& tsmm);

// Second pass of the TSMTTSM reduction when the partials are many
// (grid * M * N * c > kFinalThreshold doubles): one thread per entry of C
// sums the `grid` CTA partials in CTA order and applies alpha/beta.  Spread
// over ceil(M*N / 128) CTAs, this replaces the last CTA's single-SM sum,
// whose FP64 adds alone would take grid * M*N*c / 2 cycles on this part.
constexpr int kFinalThreshold = 32768;
cudaError_t launch_tsmttsm_final(const TsmttsmArgs& a, int grid, int cplx, cudaStream_t s);

// Per-launch choice of the runtime-threads-per-row TSMM variants (kernels_rt.cu).
void rt_tsmm_tpr(int N, int nptmax, int* tpr, int* npt);

// Device properties of the current device, cached.
struct DeviceInfo {
    int device;
    int sm_count;
    int cc_major, cc_minor;
    size_t smem_optin;
};
const DeviceInfo& device_info();

// Byte range [lo, hi) of a strided operand.
struct Range {
    uintptr_t lo, hi;
};
Range operand_range(const void* p, int64_t rows, int64_t ld, int cols, int cplx);

// Early-start bookkeeping for launch_pdl: per (device, stream), the outputs
// of the products launched since the last barrier (a product that waited at
// its start), which may still be running when the next one starts.  Call
// both with pdl_mutex() held, around the launch.  pdl_early is 1 when none
// of those outputs overlaps `in`; 0 when one does, when the list is full,
// or when the stream has no record (nothing known).  pdl_note records a
// launched product (early: whether it read before waiting).
std::mutex& pdl_mutex();
int pdl_early(cudaStream_t s, const Range* in, int nin);
void pdl_note(cudaStream_t s, Range out, int early);

// Per-(device, stream) scratch: partial sums + reduction tickets.
struct Workspace {
    double* partials;
    size_t partial_bytes;
    unsigned* tickets;
    int ticket_count;
    unsigned gs_gen;  // barrier generation of the fused Gram-Schmidt kernel (gs_fused.cu)
};
tsm_status workspace_get(cudaStream_t stream, size_t partial_bytes, int tickets, Workspace** out);

// The Gram-Schmidt step as one cooperative kernel (gs_fused.cu), and the
// rule by which tsm_gs_step picks it over the two products.
tsm_status gs_fused_run(tsm_dtype dtype, int M, int N, int64_t K, const void* A, int64_t lda, void* B,
                        int64_t ldb, void* C, int64_t ldc, cudaStream_t s);
bool gs_fused_preferred(tsm_dtype dtype, int M, int N, int64_t K);

// Scale-only updates (K == 0 or alpha == 0 paths).
cudaError_t launch_scale_small(double* C, int rows, int cols, int64_t ld, int cplx, double br,
                               double bi, int beta_zero, cudaStream_t s);
cudaError_t launch_scale_tall(double* B, int64_t rows, int cols, int64_t ld, int cplx, double br,
                              double bi, int beta_zero, cudaStream_t s);

}  // namespace tsm
