// C-ABI entry points of libtsm: argument validation, the variant registry,
// per-(device, stream) workspaces and dispatch.  Every product runs in the
// library's own kernels; there is no CPU fallback.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "pdl_book.h"
#include "tsm_internal.h"
#include "tune.h"

namespace tsm {

// ------------------------------------------------------------ device info

const DeviceInfo& device_info() {
    static thread_local DeviceInfo cache[64];
    static thread_local bool valid[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!valid[dev]) {
        DeviceInfo d;
        memset(&d, 0, sizeof(d));
        d.device = dev;
        cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        d.smem_optin = (size_t)optin;
        cache[dev] = d;
        valid[dev] = true;
    }
    return cache[dev];
}

// -------------------------------------------------------------- workspace

namespace {

std::mutex g_ws_mutex;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

}  // namespace

tsm_status workspace_get(cudaStream_t stream, size_t partial_bytes, int tickets, Workspace** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSM_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    Workspace*& w = g_ws[std::make_pair(dev, stream)];
    if (!w) {
        w = new Workspace();
        memset(w, 0, sizeof(*w));
    }
    if (w->partial_bytes < partial_bytes || w->ticket_count < tickets) {
        // Growing: earlier work on this stream may still read the old buffers.
        if (w->partials || w->tickets) {
            if (cudaStreamSynchronize(stream) != cudaSuccess) return TSM_ERR_LAUNCH;
            cudaFree(w->partials);
            cudaFree(w->tickets);
            w->partials = nullptr;
            w->tickets = nullptr;
        }
        size_t pb = partial_bytes > w->partial_bytes ? partial_bytes : w->partial_bytes;
        pb = (pb + 4095) & ~(size_t)4095;
        int tc = tickets > w->ticket_count ? tickets : w->ticket_count;
        if (tc < 64) tc = 64;
        if (cudaMalloc(&w->partials, pb) != cudaSuccess) {
            w->partials = nullptr;
            w->partial_bytes = 0;
            return TSM_ERR_ALLOC;
        }
        if (cudaMalloc(&w->tickets, sizeof(unsigned) * tc) != cudaSuccess) {
            cudaFree(w->partials);
            w->partials = nullptr;
            w->partial_bytes = 0;
            w->tickets = nullptr;
            return TSM_ERR_ALLOC;
        }
        if (cudaMemset(w->tickets, 0, sizeof(unsigned) * tc) != cudaSuccess) return TSM_ERR_LAUNCH;
        w->gs_gen = 0u;  // the barrier flag starts at zero again
        w->partial_bytes = pb;
        w->ticket_count = tc;
    }
    *out = w;
    return TSM_OK;
}

// ------------------------------------------------- early-start bookkeeping

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = getenv("TSM_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

namespace {
struct OccKey {
    const void* kernel;
    int block;
    size_t smem;
    bool operator<(const OccKey& o) const {
        if (kernel != o.kernel) return kernel < o.kernel;
        if (block != o.block) return block < o.block;
        return smem < o.smem;
    }
};
std::mutex g_occ_mutex;
std::map<std::pair<int, OccKey>, int> g_occ;  // (device, kernel shape) -> resident CTAs per SM
}  // namespace

bool pdl_allowed(const void* kernel, int grid, int block, size_t smem) {
    if (!pdl_enabled()) return false;
    const DeviceInfo& di = device_info();
    const auto key = std::make_pair(di.device, OccKey{kernel, block, smem});
    int occ = 0;
    {
        std::lock_guard<std::mutex> lock(g_occ_mutex);
        auto it = g_occ.find(key);
        if (it != g_occ.end()) {
            occ = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem) != cudaSuccess) {
                cudaGetLastError();
                occ = 0;
            }
            g_occ[key] = occ;
        }
    }
    return occ > 0 && (int64_t)grid >= (int64_t)occ * di.sm_count;
}

Range operand_range(const void* p, int64_t rows, int64_t ld, int cols, int cplx) {
    const pdl::Span sp = pdl::operand_span(p, rows, ld, cols, cplx);
    return Range{sp.lo, sp.hi};
}

namespace {

// A fixed table of per-stream books (pdl_book.h; no allocation, so the
// no-allocation entry point can use it); the least recently used record
// makes room for a new stream.
struct PdlRecord {
    int dev;
    cudaStream_t stream;
    unsigned long long used;
    pdl::Book book;
};
constexpr int kPdlRecords = 64;
PdlRecord g_pdl[kPdlRecords];
unsigned long long g_pdl_clock = 0;
std::mutex g_pdl_mutex;

PdlRecord* pdl_find(int dev, cudaStream_t s) {
    for (int i = 0; i < kPdlRecords; ++i)
        if (g_pdl[i].used && g_pdl[i].dev == dev && g_pdl[i].stream == s) return &g_pdl[i];
    return nullptr;
}

}  // namespace

std::mutex& pdl_mutex() { return g_pdl_mutex; }

int pdl_early(cudaStream_t s, const Range* in, int nin) {
    if (!pdl_enabled()) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const PdlRecord* r = pdl_find(dev, s);
    if (!r) return 0;
    pdl::Span sp[4];
    if (nin > 4) return 0;
    for (int i = 0; i < nin; ++i) sp[i] = pdl::Span{in[i].lo, in[i].hi};
    return pdl::may_read_early(r->book, sp, nin);
}

void pdl_note(cudaStream_t s, Range out, int early) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    PdlRecord* r = pdl_find(dev, s);
    if (!r) {
        r = &g_pdl[0];
        for (int i = 0; i < kPdlRecords; ++i) {
            if (!g_pdl[i].used) {
                r = &g_pdl[i];
                break;
            }
            if (g_pdl[i].used < r->used) r = &g_pdl[i];
        }
        r->dev = dev;
        r->stream = s;
        r->book.valid = false;  // a new record starts at this product
        r->book.n = 0;
    }
    r->used = ++g_pdl_clock;
    pdl::note_launch(r->book, pdl::Span{out.lo, out.hi}, early);
}

static tsm_status release_all() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSM_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    for (auto it = g_ws.begin(); it != g_ws.end();) {
        if (it->first.first == dev) {
            cudaFree(it->second->partials);
            cudaFree(it->second->tickets);
            delete it->second;
            it = g_ws.erase(it);
        } else {
            ++it;
        }
    }
    return TSM_OK;
}

// --------------------------------------------------------------- registry

struct Registry {
    std::vector<Variant> tsmttsm, tsmm;
    Registry() {
        register_fp64_variants(tsmttsm, tsmm);
        register_generated_variants(tsmttsm, tsmm);
        register_rt_variants(tsmttsm, tsmm);
        register_narrow_variants(tsmttsm, tsmm);
    }
};

static const Registry& registry() {
    static Registry r;
    return r;
}

static const std::vector<Variant>* table(tsm_kind kind) {
    if (kind == TSM_KIND_TSMTTSM) return &registry().tsmttsm;
    if (kind == TSM_KIND_TSMM || kind == TSM_KIND_TSMM_BETA) return &registry().tsmm;
    return nullptr;
}

static bool variant_supports(const Variant& v, int dtype, int M, int N) {
    if (v.info.dtype != dtype) return false;
    if (v.info.fixed_m && v.info.fixed_m != M) return false;
    if (v.info.fixed_n && v.info.fixed_n != N) return false;
    if (v.info.runtime_tile) return M >= 1 && N >= 1 && M <= 64 && N <= 64;  // a tile always exists
    if (v.info.kind == TSM_KIND_TSMTTSM) {
        const int P = ((M + v.info.tile_m - 1) / v.info.tile_m) * ((N + v.info.tile_n - 1) / v.info.tile_n);
        return P <= v.info.block;
    }
    return N <= v.info.threads_per_row * v.info.tile_n;
}

// Built-in choice when no tuning entry exists (the paper's rules of thumb:
// square-ish register tiles sized so that a CTA's threads all own one;
// TSMM with a multiple of 4 threads per row, Sec. 6.3).
static int heuristic_variant(tsm_kind kind, int dtype, int M, int N) {
    const std::vector<Variant>& t = *table(kind);
    auto find = [&](const char* name) -> int {
        for (size_t i = 0; i < t.size(); ++i)
            if (strcmp(t[i].info.name, name) == 0) return (int)i;
        return -1;
    };
    char name[64];
    const char* dt = dtype == TSM_C64 ? "c64" : "r64";
    if (kind == TSM_KIND_TSMTTSM) {
        // Hand-written tiles only: least padding waste (FMAs on guarded,
        // out-of-range tile entries), then the larger tile (fewer loads per
        // FMA, Sec. 3), then fewer rows unrolled.
        int best = -1;
        double best_waste = 1e30;
        int best_area = 0, best_u = 0;
        for (size_t i = 0; i < t.size(); ++i) {
            const tsm_variant_info& f = t[i].info;
            if (f.generated || !variant_supports(t[i], dtype, M, N)) continue;
            const int pm = (M + f.tile_m - 1) / f.tile_m, pn = (N + f.tile_n - 1) / f.tile_n;
            const double waste = (double)(pm * f.tile_m) * (pn * f.tile_n) / ((double)M * N);
            const int area = f.tile_m * f.tile_n;
            if (area * (dtype == TSM_C64 ? 2 : 1) > 32) continue;
            const bool better = waste < best_waste - 1e-9 ||
                                (waste < best_waste + 1e-9 && (area > best_area ||
                                                               (area == best_area && f.unroll > best_u)));
            if (better) {
                best = (int)i;
                best_waste = waste;
                best_area = area;
                best_u = f.unroll;
            }
        }
        if (best >= 0) return best;
        snprintf(name, sizeof(name), "tsmttsm_%s_direct_t1x1_u4", dt);
    } else {
        int tpr = N >= 16 ? 16 : (N >= 8 ? 8 : (N >= 4 ? 4 : (N >= 2 ? 2 : 1)));
        int npt = (N + tpr - 1) / tpr;
        int nptv = npt <= 1 ? 1 : npt <= 2 ? 2 : npt <= 4 ? 4 : npt <= 8 ? 8 : 16;
        const int u = nptv >= 8 ? 1 : (nptv >= 4 ? (tpr == 16 ? 2 : 2) : (nptv == 2 ? (tpr >= 8 ? 2 : 4) : 4));
        snprintf(name, sizeof(name), "tsmm_%s_smemc_tpr%d_npt%d_u%d", dt, tpr, nptv, u);
        // widths the power-of-two thread counts do not cover exactly: the
        // runtime variant (any threads per row, so no padded result slots)
        if (npt * tpr != N) {
            char rt[64];
            snprintf(rt, sizeof(rt), "tsmm_%s_rt_npt4_u2", dt);
            const int r = find(rt);
            if (r >= 0) return r;
        }
        int idx = find(name);
        if (idx >= 0) return idx;
        for (size_t i = 0; i < t.size(); ++i)
            if (variant_supports(t[i], dtype, M, N) && !t[i].info.fixed_m) return (int)i;
        return -1;
    }
    int idx = find(name);
    if (idx >= 0 && variant_supports(t[idx], dtype, M, N)) return idx;
    for (size_t i = 0; i < t.size(); ++i)
        if (variant_supports(t[i], dtype, M, N) && !t[i].info.fixed_m) return (int)i;
    return -1;
}

static int default_grid(const Variant& v, int M, int N) {
    const int occ = v.occupancy ? v.occupancy(M, N) : 1;
    return device_info().sm_count * (occ > 0 ? occ : 1);
}

tsm_status choose(tsm_kind kind, int dtype, int M, int N, int64_t K, int* variant, int* grid) {
    const std::vector<Variant>* t = table(kind);
    if (!t) return TSM_ERR_INVALID_VALUE;
    int v = -1, g = 0;
    auto looked_up = [&](tsm_kind k) {
        return tune_lookup(k, dtype, M, N, K, &v, &g) == TSM_OK && v >= 0 && v < (int)t->size() &&
               variant_supports((*t)[v], dtype, M, N);
    };
    // TSMM with beta != 0: its own entry first, else the beta = 0 one
    if (!looked_up(kind) && !(kind == TSM_KIND_TSMM_BETA && looked_up(TSM_KIND_TSMM))) {
        v = heuristic_variant(kind == TSM_KIND_TSMM_BETA ? TSM_KIND_TSMM : kind, dtype, M, N);
        g = 0;
    }
    if (v < 0) return TSM_ERR_NOT_SUPPORTED;
    if (g <= 0) g = default_grid((*t)[v], M, N);
    *variant = v;
    *grid = g;
    return TSM_OK;
}

const Variant* variant_at(tsm_kind kind, int idx) {
    const std::vector<Variant>* t = table(kind);
    if (!t || idx < 0 || idx >= (int)t->size()) return nullptr;
    return &(*t)[idx];
}

bool supports(tsm_kind kind, int idx, int dtype, int M, int N) {
    const Variant* v = variant_at(kind, idx);
    return v && variant_supports(*v, dtype, M, N);
}

// ------------------------------------------------------------- validation

static bool is_zero(const double* x, int cplx) { return x[0] == 0.0 && (!cplx || x[1] == 0.0); }

static tsm_status check_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSM_ERR_NO_DEVICE;
    const DeviceInfo& d = device_info();
    if (d.cc_major != 10 || d.cc_minor != 3) return TSM_ERR_NO_DEVICE;
    return TSM_OK;
}

tsm_status validate_common(int dtype, int M, int N, int64_t K, const double* alpha, const double* beta) {
    if (dtype != TSM_R64 && dtype != TSM_C64) return TSM_ERR_INVALID_VALUE;
    if (K < 0) return TSM_ERR_INVALID_VALUE;
    if (!alpha || !beta) return TSM_ERR_INVALID_VALUE;
    if (M < 1 || N < 1 || M > 64 || N > 64) return TSM_ERR_NOT_SUPPORTED;
    return TSM_OK;
}

tsm_status run_tsmttsm(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                       const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                       int64_t ldc, int variant, int grid, cudaStream_t stream) {
    tsm_status st = validate_common(dtype, M, N, K, alpha, beta);
    if (st != TSM_OK) return st;
    if (opA != TSM_OP_T && opA != TSM_OP_C) return TSM_ERR_INVALID_VALUE;
    if (lda < M || ldb < N || ldc < N) return TSM_ERR_INVALID_VALUE;
    if (!C) return TSM_ERR_INVALID_VALUE;
    const int cplx = dtype == TSM_C64;
    const bool scale_only = K == 0 || is_zero(alpha, cplx);
    if (!scale_only && (!A || !B)) return TSM_ERR_INVALID_VALUE;
    if ((st = check_device()) != TSM_OK) return st;

    const int beta_zero = is_zero(beta, cplx);
    if (scale_only) {
        if (launch_scale_small((double*)C, M, N, ldc, cplx, beta[0], cplx ? beta[1] : 0.0, beta_zero,
                               stream) != cudaSuccess)
            return TSM_ERR_LAUNCH;
        return TSM_OK;
    }
    int v = variant, g = grid;
    if (v < 0) {
        int gg = 0;
        if ((st = choose(TSM_KIND_TSMTTSM, dtype, M, N, K, &v, &gg)) != TSM_OK) return st;
        if (g <= 0) g = gg;
    }
    if (!supports(TSM_KIND_TSMTTSM, v, dtype, M, N)) return TSM_ERR_NOT_SUPPORTED;
    const Variant& var = *variant_at(TSM_KIND_TSMTTSM, v);
    if (g <= 0) g = default_grid(var, M, N);
    if (g > 65535) g = 65535;

    Workspace* ws = nullptr;
    const size_t pbytes = (size_t)g * M * N * (cplx ? 2 : 1) * sizeof(double);
    if ((st = workspace_get(stream, pbytes, 1, &ws)) != TSM_OK) return st;

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
    a.ws = ws->partials;
    a.ticket = ws->tickets;
    a.final_pass = tsm_tsmttsm_kernels_per_call(dtype, M, N, g) == 2 ? 1 : 0;
    const Range in[2] = {operand_range(A, K, lda, M, cplx), operand_range(B, K, ldb, N, cplx)};
    std::lock_guard<std::mutex> lock(pdl_mutex());
    a.early = pdl_early(stream, in, 2);
    if (var.tsmttsm(a, g, stream) != cudaSuccess) return TSM_ERR_LAUNCH;
    if (a.final_pass && launch_tsmttsm_final(a, g, cplx, stream) != cudaSuccess) return TSM_ERR_LAUNCH;
    pdl_note(stream, operand_range(C, M, ldc, N, cplx), a.early);
    return TSM_OK;
}

tsm_status run_tsmm(tsm_op opC, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                    const void* A, int64_t lda, const void* Cm, int64_t ldc, const double* beta, void* B,
                    int64_t ldb, int variant, int grid, cudaStream_t stream) {
    tsm_status st = validate_common(dtype, M, N, K, alpha, beta);
    if (st != TSM_OK) return st;
    if (opC != TSM_OP_N) return opC == TSM_OP_T || opC == TSM_OP_C ? TSM_ERR_NOT_SUPPORTED
                                                                    : TSM_ERR_INVALID_VALUE;
    if (lda < M || ldb < N || ldc < N) return TSM_ERR_INVALID_VALUE;
    if (K == 0) return TSM_OK;
    if (!B) return TSM_ERR_INVALID_VALUE;
    const int cplx = dtype == TSM_C64;
    const bool scale_only = is_zero(alpha, cplx);
    if (!scale_only && (!A || !Cm)) return TSM_ERR_INVALID_VALUE;
    if ((st = check_device()) != TSM_OK) return st;
    const int beta_zero = is_zero(beta, cplx);
    if (scale_only) {
        if (launch_scale_tall((double*)B, K, N, ldb, cplx, beta[0], cplx ? beta[1] : 0.0, beta_zero,
                              stream) != cudaSuccess)
            return TSM_ERR_LAUNCH;
        return TSM_OK;
    }
    int v = variant, g = grid;
    if (v < 0) {
        int gg = 0;
        const tsm_kind key = beta_zero ? TSM_KIND_TSMM : TSM_KIND_TSMM_BETA;
        if ((st = choose(key, dtype, M, N, K, &v, &gg)) != TSM_OK) return st;
        if (g <= 0) g = gg;
    }
    if (!supports(TSM_KIND_TSMM, v, dtype, M, N)) return TSM_ERR_NOT_SUPPORTED;
    const Variant& var = *variant_at(TSM_KIND_TSMM, v);
    if (g <= 0) g = default_grid(var, M, N);
    if (g > 65535) g = 65535;
    TsmmArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = (const double*)A;
    a.lda = lda;
    a.Cm = (const double*)Cm;
    a.ldc = ldc;
    a.B = (double*)B;
    a.ldb = ldb;
    a.alpha_r = alpha[0];
    a.alpha_i = cplx ? alpha[1] : 0.0;
    a.beta_r = beta[0];
    a.beta_i = cplx ? beta[1] : 0.0;
    a.beta_zero = beta_zero;
    a.beta_one = beta[0] == 1.0 && (!cplx || beta[1] == 0.0);
    std::lock_guard<std::mutex> lock(pdl_mutex());
    if (var.tsmm(a, g, stream) != cudaSuccess) return TSM_ERR_LAUNCH;
    pdl_note(stream, operand_range(B, K, ldb, N, cplx), 0);
    return TSM_OK;
}

}  // namespace tsm

using namespace tsm;

extern "C" {

tsm_status tsm_tsmttsm(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                       const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta, void* C,
                       int64_t ldc, tsm_stream_t stream) {
    return run_tsmttsm(opA, dtype, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, -1, 0,
                       (cudaStream_t)stream);
}

tsm_status tsm_tsmm(tsm_op opC, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                    const void* A, int64_t lda, const void* C, int64_t ldc, const double* beta, void* B,
                    int64_t ldb, tsm_stream_t stream) {
    return run_tsmm(opC, dtype, M, N, K, alpha, A, lda, C, ldc, beta, B, ldb, -1, 0, (cudaStream_t)stream);
}

tsm_status tsm_tsmttsm_ex(tsm_op opA, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                          const void* A, int64_t lda, const void* B, int64_t ldb, const double* beta,
                          void* C, int64_t ldc, int variant, int grid, tsm_stream_t stream) {
    return run_tsmttsm(opA, dtype, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, variant, grid,
                       (cudaStream_t)stream);
}

tsm_status tsm_tsmm_ex(tsm_op opC, tsm_dtype dtype, int M, int N, int64_t K, const double* alpha,
                       const void* A, int64_t lda, const void* C, int64_t ldc, const double* beta, void* B,
                       int64_t ldb, int variant, int grid, tsm_stream_t stream) {
    return run_tsmm(opC, dtype, M, N, K, alpha, A, lda, C, ldc, beta, B, ldb, variant, grid,
                    (cudaStream_t)stream);
}

tsm_status tsm_gs_step_ex(tsm_dtype dtype, int M, int N, int64_t K, const void* A, int64_t lda, void* B,
                          int64_t ldb, void* C, int64_t ldc, tsm_gs_mode mode, tsm_stream_t stream) {
    const double one[2] = {1.0, 0.0}, zero[2] = {0.0, 0.0}, minus_one[2] = {-1.0, 0.0};
    // every argument is checked before the first launch, so that an error
    // leaves B and C untouched
    tsm_status st = validate_common(dtype, M, N, K, one, zero);
    if (st != TSM_OK) return st;
    if (mode != TSM_GS_AUTO && mode != TSM_GS_TWO_PRODUCTS && mode != TSM_GS_FUSED) return TSM_ERR_INVALID_VALUE;
    if (lda < M || ldb < N || ldc < N || !C) return TSM_ERR_INVALID_VALUE;
    if (K > 0 && (!A || !B)) return TSM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    const bool fused = K > 0 && (mode == TSM_GS_FUSED || (mode == TSM_GS_AUTO && gs_fused_preferred(dtype, M, N, K)));
    if (fused) {
        if ((st = check_device()) != TSM_OK) return st;
        return gs_fused_run(dtype, M, N, K, A, lda, B, ldb, C, ldc, s);
    }
    if ((st = run_tsmttsm(TSM_OP_C, dtype, M, N, K, one, A, lda, B, ldb, zero, C, ldc, -1, 0, s)) != TSM_OK)
        return st;
    return run_tsmm(TSM_OP_N, dtype, M, N, K, minus_one, A, lda, C, ldc, one, B, ldb, -1, 0, s);
}

tsm_status tsm_gs_step(tsm_dtype dtype, int M, int N, int64_t K, const void* A, int64_t lda, void* B,
                       int64_t ldb, void* C, int64_t ldc, tsm_stream_t stream) {
    return tsm_gs_step_ex(dtype, M, N, K, A, lda, B, ldb, C, ldc, TSM_GS_AUTO, stream);
}

const char* tsm_status_string(tsm_status s) {
    switch (s) {
        case TSM_OK: return "success";
        case TSM_ERR_INVALID_VALUE: return "invalid argument";
        case TSM_ERR_NOT_SUPPORTED: return "not supported";
        case TSM_ERR_ALLOC: return "device allocation failed";
        case TSM_ERR_LAUNCH: return "kernel launch or CUDA runtime error";
        case TSM_ERR_TIMEOUT: return "device-side wait timed out";
        case TSM_ERR_INTERNAL: return "internal error";
        case TSM_ERR_NO_DEVICE: return "no usable sm_103 device";
    }
    return "unknown status";
}

const char* tsm_version(void) { return "0.1.0"; }

tsm_status tsm_release(void) { return release_all(); }

int tsm_variant_count(tsm_kind kind) {
    const std::vector<Variant>* t = table(kind);
    return t ? (int)t->size() : -1;
}

tsm_status tsm_variant_get(tsm_kind kind, int index, tsm_variant_info* info) {
    const Variant* v = variant_at(kind, index);
    if (!v || !info) return TSM_ERR_INVALID_VALUE;
    *info = v->info;
    return TSM_OK;
}

tsm_status tsm_variant_shape(tsm_kind kind, int index, tsm_dtype dtype, int M, int N, tsm_variant_info* info) {
    const Variant* v = variant_at(kind, index);
    if (!v || !info) return TSM_ERR_INVALID_VALUE;
    if (!variant_supports(*v, dtype, M, N)) return TSM_ERR_NOT_SUPPORTED;
    *info = v->info;
    if (v->info.runtime_tile) {
        if (kind == TSM_KIND_TSMM || kind == TSM_KIND_TSMM_BETA)
            rt_tsmm_tpr(N, v->info.tile_n, &info->threads_per_row, &info->tile_n);
    }
    return TSM_OK;
}

int tsm_tsmttsm_kernels_per_call(tsm_dtype dtype, int M, int N, int grid) {
    if (M < 1 || N < 1 || M > 64 || N > 64 || grid < 1 || (dtype != TSM_R64 && dtype != TSM_C64)) return -1;
    return (int64_t)grid * M * N * (dtype == TSM_C64 ? 2 : 1) > kFinalThreshold ? 2 : 1;
}

int tsm_variant_supports(tsm_kind kind, int index, tsm_dtype dtype, int M, int N) {
    return supports(kind, index, dtype, M, N) ? 1 : 0;
}

tsm_status tsm_choose(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K, int* variant, int* grid) {
    if (!variant || !grid) return TSM_ERR_INVALID_VALUE;
    if (M < 1 || N < 1 || M > 64 || N > 64) return TSM_ERR_NOT_SUPPORTED;
    if (check_device() != TSM_OK) return TSM_ERR_NO_DEVICE;
    return choose(kind, dtype, M, N, K, variant, grid);
}

}  // extern "C"
