// Seeded synthetic inputs on the device (input generation only; not part of
// either product).  Element (k, c) of a rows x ld block (rows row0 .. of the
// full matrix) takes output i = (row0 + k) * ld + c of a SplitMix64 stream
// (Steele, Lea, Flood, OOPSLA 2014) seeded with `seed`: z = seed + (i + 1) *
// 0x9E3779B97F4A7C15, then the generator's xor-shift-multiply finaliser.
// Complex elements take outputs 2i (real part) and 2i + 1 (imaginary part).
// The host-side generator of the test suite implements the same definition
// independently; a GPU test compares the two bit for bit.
#include "tsm_internal.h"

namespace tsm {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Bit-exact maps from a 64-bit draw to a double (see the table in tsm.h).
__device__ __forceinline__ double draw_to_double(uint64_t h, int dist) {
    switch (dist) {
        case 0:  // uniform [-1, 1): (h >> 11) * 2^-52 - 1, exact
            return (double)(h >> 11) * 0x1p-52 - 1.0;
        case 1: {  // log-uniform magnitudes 2^-20 .. 2^20
            const double mant = (double)(h >> 12) * 0x1p-52 + 1.0;
            const int e = (int)(((h & 0x7FFull) * 40ull) >> 11) - 20;
            const double v = scalbn(mant, e);
            return ((h >> 11) & 1ull) ? -v : v;
        }
        case 2:  // integers in [-8, 7]
            return (double)(h >> 60) - 8.0;
        default:
            return 1.0;
    }
}

__global__ void k_fill(double* dst, int cplx, int64_t rows, int64_t ld, int64_t row0, uint64_t seed,
                       int dist) {
    const int64_t n = rows * ld;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
         o += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t i = (uint64_t)(row0 * ld + o);
        if (!cplx) {
            dst[o] = dist == 3 ? 1.0 : draw_to_double(splitmix64(seed, i), dist);
        } else {
            dst[2 * o] = dist == 3 ? 1.0 : draw_to_double(splitmix64(seed, 2 * i), dist);
            dst[2 * o + 1] = dist == 3 ? 1.0 : draw_to_double(splitmix64(seed, 2 * i + 1), dist);
        }
    }
}

}  // namespace
}  // namespace tsm

extern "C" tsm_status tsm_fill_random(void* dst, tsm_dtype dtype, int64_t rows, int64_t ld, int64_t row0,
                                      uint64_t seed, int dist, tsm_stream_t stream) {
    if (rows < 0 || ld < 0 || row0 < 0 || dist < 0 || dist > 3) return TSM_ERR_INVALID_VALUE;
    if (dtype != TSM_R64 && dtype != TSM_C64) return TSM_ERR_INVALID_VALUE;
    if (rows == 0 || ld == 0) return TSM_OK;
    if (!dst) return TSM_ERR_INVALID_VALUE;
    const int grid = tsm::device_info().sm_count * 8;
    tsm::k_fill<<<grid, 256, 0, (cudaStream_t)stream>>>((double*)dst, dtype == TSM_C64, rows, ld, row0, seed,
                                                        dist);
    return cudaGetLastError() == cudaSuccess ? TSM_OK : TSM_ERR_LAUNCH;
}
