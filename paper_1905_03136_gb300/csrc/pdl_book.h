// Host-only bookkeeping behind the early reads of programmatic dependent
// launch (no CUDA calls, so the host tests compile it on its own).
//
// A stream's book holds the byte ranges written by the products launched
// since the last barrier -- a product that waited for its predecessor at
// its start, so that every product before it had completed when the ones
// after it were scheduled.  Those products may still be running when the
// next product starts; it may read its inputs before waiting only if none
// of them overlaps a range in the book.
#pragma once

#include <stdint.h>

namespace tsm {
namespace pdl {

// Byte range [lo, hi).
struct Span {
    uintptr_t lo, hi;
};

inline bool overlaps(const Span& a, const Span& b) { return a.lo < b.hi && b.lo < a.hi; }

// Bytes of a row-major operand of `rows` rows of `cols` elements with
// leading dimension `ld` (elements of 8 bytes, 16 when complex); empty for
// a null pointer or no rows or columns.
inline Span operand_span(const void* p, int64_t rows, int64_t ld, int cols, int cplx) {
    Span r = {0, 0};
    if (!p || rows <= 0 || cols <= 0) return r;
    r.lo = (uintptr_t)p;
    r.hi = r.lo + (uintptr_t)(((uint64_t)(rows - 1) * (uint64_t)ld + (uint64_t)cols) * (cplx ? 16u : 8u));
    return r;
}

constexpr int kOuts = 8;

struct Book {
    bool valid;        // false: nothing is known about this stream
    int n;             // ranges in use
    Span out[kOuts];   // outputs since the last barrier, the barrier's first
};

// 1 if a product reading `in[0..nin)` may read them before its predecessor
// completes: the book is known, not full, and no range in it overlaps an
// input.
inline int may_read_early(const Book& b, const Span* in, int nin) {
    if (!b.valid || b.n >= kOuts) return 0;
    for (int j = 0; j < b.n; ++j)
        for (int i = 0; i < nin; ++i)
            if (overlaps(in[i], b.out[j])) return 0;
    return 1;
}

// Records a product just launched that writes `out`; `early` says whether
// it read before waiting.  A product that waited at its start is a barrier
// and starts a new list; so does a full list (its next product waits, since
// may_read_early refuses a full book).
inline void note_launch(Book& b, Span out, int early) {
    if (!b.valid) {
        b.valid = true;
        early = 0;
    }
    if (!early || b.n >= kOuts) b.n = 0;
    b.out[b.n++] = out;
}

}  // namespace pdl
}  // namespace tsm
