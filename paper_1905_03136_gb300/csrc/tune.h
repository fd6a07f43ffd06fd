// Tuning table and exhaustive autotuner (Sec. 5.1 and 7 of the paper: the
// best configuration per size is found by exhaustive search).
#pragma once

#include "tsm_internal.h"

namespace tsm {

// Looks up (kind, dtype, M, N, K bucket); TSM_OK with *variant >= 0 on a hit.
tsm_status tune_lookup(int kind, int dtype, int M, int N, int64_t K, int* variant, int* grid);

const Variant* variant_at(tsm_kind kind, int idx);
bool supports(tsm_kind kind, int idx, int dtype, int M, int N);
tsm_status run_tsmttsm(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                       const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                       int64_t ldc, int variant, int grid, cudaStream_t stream);
tsm_status run_tsmm(tsm_op opC, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                    const void* A, int64_t lda, const void* Cm, int64_t ldc, const double* beta, void* B,
                    int64_t ldb, int variant, int grid, cudaStream_t stream);

// K bucket of the tuning key: floor(log2(K)), 0 for K < 2.
int k_bucket(int64_t K);

}  // namespace tsm
