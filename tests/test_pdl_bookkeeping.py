"""Host logic of the early reads of programmatic dependent launch
(`csrc/pdl_book.h`, no GPU): a product may read its inputs before its
predecessor completes only if no product launched since the last barrier
(a product that waited at its start) wrote any of them.

A small C++ program compiled against the header replays launch sequences
given on its standard input and prints each decision; the cases below fix
what must and must not be allowed.
"""

import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1905_03136_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "pdl_book.h"
using namespace tsm::pdl;
// commands, one per line:
//   q lo hi [lo hi ...]   -> prints may_read_early for these input ranges
//   n lo hi early         -> note_launch
//   s p rows ld cols cplx -> prints operand_span lo hi
int main() {
    Book b;
    b.valid = false;
    b.n = 0;
    char cmd[8];
    while (std::scanf("%7s", cmd) == 1) {
        if (!std::strcmp(cmd, "q")) {
            int k;
            std::scanf("%d", &k);
            Span in[8];
            for (int i = 0; i < k; ++i) {
                unsigned long long lo, hi;
                std::scanf("%llu %llu", &lo, &hi);
                in[i] = Span{(uintptr_t)lo, (uintptr_t)hi};
            }
            std::printf("%d\n", may_read_early(b, in, k));
        } else if (!std::strcmp(cmd, "n")) {
            unsigned long long lo, hi;
            int e;
            std::scanf("%llu %llu %d", &lo, &hi, &e);
            note_launch(b, Span{(uintptr_t)lo, (uintptr_t)hi}, e);
        } else if (!std::strcmp(cmd, "s")) {
            unsigned long long p;
            long long rows, ld;
            int cols, cplx;
            std::scanf("%llu %lld %lld %d %d", &p, &rows, &ld, &cols, &cplx);
            Span sp = operand_span((const void*)(uintptr_t)p, rows, ld, cols, cplx);
            std::printf("%llu %llu\n", (unsigned long long)sp.lo, (unsigned long long)sp.hi);
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def run():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "book.cpp")
    exe = os.path.join(d, "book")
    with open(src, "w") as f:
        f.write(DRIVER)
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", CSRC, src, "-o", exe])

    def go(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split("\n")[:-1]
    yield go
    shutil.rmtree(d, ignore_errors=True)


def q(*ranges):
    return "q %d %s" % (len(ranges), " ".join("%d %d" % r for r in ranges))


def test_unknown_stream_waits(run):
    assert run([q((0, 100))]) == ["0"]


def test_output_of_previous_product_is_not_read_early(run):
    assert run(["n 1000 2000 0", q((0, 100)), q((1500, 1600)), q((0, 1001))]) == ["1", "0", "0"]


def test_half_open_ranges_touching_do_not_overlap(run):
    assert run(["n 1000 2000 0", q((2000, 3000)), q((0, 1000)), q((1999, 2000))]) == ["1", "1", "0"]


def test_every_output_since_the_last_barrier_counts(run):
    # barrier X, then two early products Y, Z: X, Y, Z may all still run
    seq = ["n 100 200 0", "n 300 400 1", "n 500 600 1",
           q((150, 160)), q((350, 360)), q((550, 560)), q((700, 800))]
    assert run(seq) == ["0", "0", "0", "1"]


def test_a_barrier_retires_what_came_before(run):
    # X, early Y, then a barrier Z: X and Y completed before Z's successors
    seq = ["n 100 200 0", "n 300 400 1", "n 500 600 0", q((150, 160)), q((350, 360)), q((550, 560))]
    assert run(seq) == ["1", "1", "0"]


def test_all_inputs_are_checked(run):
    assert run(["n 100 200 0", q((0, 50), (300, 400), (199, 250))]) == ["0"]


def test_a_full_book_forces_a_wait_then_restarts(run):
    seq = ["n 0 1 0"] + ["n %d %d 1" % (10 * i, 10 * i + 1) for i in range(1, 8)]  # 8 ranges
    seq += [q((5000, 6000))]                      # full: refused
    seq += ["n 9000 9001 0", q((5000, 6000)), q((10, 11))]  # the waiting product is a barrier
    assert run(seq) == ["0", "1", "1"]


def test_operand_span(run):
    # rows 3, ld 5, cols 4 of doubles: (2 * 5 + 4) * 8 = 112 bytes; complex 224
    out = run(["s 4096 3 5 4 0", "s 4096 3 5 4 1", "s 0 3 5 4 0", "s 4096 0 5 4 0", "s 4096 1 1 1 0"])
    assert out == ["4096 4208", "4096 4320", "0 0", "0 0", "4096 4104"]
