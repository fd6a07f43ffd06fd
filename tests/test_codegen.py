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


def test_warp_fill_counts_partly_filled_warps():
    # width 26, tile 13 x 2: P = 26 threads per row lane; 256 threads hold 9
    # lanes (234 active), the eighth warp has 10 active lanes but issues all
    # 32, so 234 of 256 FMA slots are useful
    assert abs(codegen.warp_fill(26, 13, 2, 256) - 234 / 256) < 1e-12
    # 416 threads hold 16 lanes: 13 full warps
    assert codegen.warp_fill(26, 13, 2, 416) == 1.0
    # padding counts too: width 7 with 4 x 4 tiles (P = 4, 64 lanes)
    assert abs(codegen.warp_fill(7, 4, 4, 256) - 49 / 64) < 1e-12
    assert codegen.warp_fill(64, 1, 1, 256) == 0.0  # 4096 threads per lane do not fit


def test_fullwarp_tile_for_every_width():
    """Every square width gets a tile and CTA size that keeps at least 93 %
    of the FP64 issue slots useful (most widths 96-100 %), within 1024
    threads, a multiple of 32, and one CTA per SM by the register estimate;
    the generated set holds that kernel for every non-sweep width."""
    tsmttsm, _ = codegen.default_specs()
    names = {codegen._name_tsmttsm(s) for s in tsmttsm}
    fills = []
    for cplx in (False, True):
        c = 2 if cplx else 1
        for w in range(1, 65):
            tm, tn, blk = codegen.fullwarp_tile(w, cplx)
            assert tm * tn * c <= 40 and blk % 32 == 0 and 128 <= blk <= 1024
            assert codegen.tile_regs(tm, tn, cplx) * blk <= 65536
            f = codegen.warp_fill(w, tm, tn, blk)
            fills.append(f)
            assert f >= 0.93, (w, cplx, tm, tn, blk, f)
            # never worse than the 256-thread least-padded tile
            a, b = codegen.tile_for_width(w, cplx)
            assert f >= codegen.warp_fill(w, a, b, codegen.BLOCK) - 1e-9
            if w not in codegen.SWEEP_SQUARE:
                u = 4 if tm * tn <= 2 else (2 if tm * tn <= 8 else 1)
                while u > 1 and codegen.tile_regs(tm, tn, cplx, u) * blk > 65536:
                    u //= 2
                spec = dict(cplx=cplx, M=w, N=w, TM=tm, TN=tn, U=u, B=blk)
                assert codegen._name_tsmttsm(spec if blk != codegen.BLOCK else
                                             dict(spec, B=codegen.BLOCK)) in names, (w, cplx)
    assert sorted(fills)[len(fills) // 2] >= 0.99
