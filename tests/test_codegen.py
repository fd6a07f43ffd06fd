"""Host-side checks of the code generator (Sec. 2.1): every square width
gets a register tile within the accumulator and thread limits and with at
most a few per cent of padded work, and TSMM thread counts that cover N
without padding; the default variant set is unique and covers every width."""

import math

from paper_1905_03136_gb300 import codegen


def test_tile_for_every_width_is_within_limits_and_nearly_unpadded():
    for cplx in (False, True):
        c = 2 if cplx else 1
        worst = 0.0
        for w in range(1, 65):
            tm, tn = codegen.tile_for_width(w, cplx)
            P = math.ceil(w / tm) * math.ceil(w / tn)
            assert tm * tn * c <= 40 and P <= codegen.BLOCK, (w, cplx, tm, tn)
            waste = P * tm * tn / (w * w)
            worst = max(worst, waste)
            # a width with a divisor pair inside the limits has no padding
            exact = [(a, b) for a in range(1, w + 1) for b in range(1, w + 1)
                     if w % a == 0 and w % b == 0 and a * b * c <= 40 and (w // a) * (w // b) <= codegen.BLOCK]
            if exact:
                assert waste == 1.0, (w, cplx, tm, tn)
        assert worst <= 1.05, (cplx, worst)


def test_tile_with_two_lanes_and_none_when_impossible():
    for cplx in (False, True):
        for w in range(1, 65):
            t = codegen.tile_for_width(w, cplx, min_lanes=2)
            if t is not None:
                P = math.ceil(w / t[0]) * math.ceil(w / t[1])
                assert codegen.BLOCK // P >= 2
    assert codegen.tile_for_width(64, True, cap=2) is None   # 1 x 1 tiles: 4096 threads


def test_tsmm_thread_counts_cover_n_exactly():
    for cplx in (False, True):
        for N in range(1, 65):
            opts = codegen.tpr_options(N, cplx, 2)
            assert opts and len({t for t, _ in opts}) == len(opts)
            t, npt = opts[0]
            assert t * npt == N and t <= 64 and npt <= (8 if cplx else 16)
            assert codegen.tpr_for_width(N, cplx) == (t, npt)


def test_default_specs_are_unique_and_cover_every_square_width():
    tsmttsm, tsmm = codegen.default_specs()
    names = [codegen._name_tsmttsm(s) for s in tsmttsm]
    mnames = [codegen._name_tsmm(s) for s in tsmm]
    assert len(set(names)) == len(names) and len(set(mnames)) == len(mnames)
    for cplx in (False, True):
        have_t = {s["M"] for s in tsmttsm if s["cplx"] == cplx and s["M"] == s["N"]}
        have_m = {s["M"] for s in tsmm if s["cplx"] == cplx and s["M"] == s["N"]}
        assert have_m == set(range(1, 65))
        # complex 64 x 64 is served by the hand-written 8 x 4 tiles
        assert have_t | ({64} if cplx else set()) == set(range(1, 65))


def test_emitted_kernels_guard_only_border_entries():
    # a padding-free tile needs no guards; a padded one guards only the tile
    # entries that can cross the border: with 4 x 4 tiles on 7 x 7 (PM = PN
    # = 2, entry i at row pm + 2i) that is entry 3 alone in each direction
    src = codegen.emit_tsmttsm(dict(cplx=False, M=37, N=37, TM=1, TN=37, U=1))
    assert "const bool g" not in src
    src = codegen.emit_tsmttsm(dict(cplx=False, M=7, N=7, TM=4, TN=4, U=1))
    guards = sorted(l.strip() for l in src.splitlines() if "const bool g" in l)
    assert guards == ["const bool gm3 = pm + 6 < 7;", "const bool gn3 = pn + 6 < 7;"]
