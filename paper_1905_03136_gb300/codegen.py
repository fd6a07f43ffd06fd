"""Code generator for width-specialised FP64 kernels (Sec. 2.1 of the paper).

Like the paper's generator, this script writes CUDA source for fixed sizes:
every loop over the small dimensions is unrolled into straight-line code
with one named scalar per accumulator (Listing 3), index arithmetic uses
compile-time constants, and guards are emitted only for the tile entries
that can cross the matrix border (entries that every thread owns inside the
matrix get none).  The kernels reuse the hand-written deterministic
reduction epilogue and C staging from ``csrc/fp64_common.cuh``.

Generated kernels register themselves in the library's variant table with
``fixed_m``/``fixed_n`` set, so dispatch and the autotuner only offer them for
their own shape.  The default variant set covers the widths of the
benchmark sweep (M = N in powers of two up to 64 plus four off-diagonal
pairs) with a few tile / threads-per-row choices each; ``--specs`` adds more.

Usage:  python -m paper_1905_03136_gb300.codegen OUT_DIR [--shards N]
"""

import argparse
import math
import os

SWEEP_SQUARE = (1, 2, 4, 8, 16, 32, 64)
SWEEP_OFFDIAG = ((1, 64), (64, 1), (8, 32), (32, 8))
TSMM_OFFDIAG = ((4, 64), (64, 4))
BLOCK = 256


def _tiles_for(M, N, cplx):
    """Up to three register tiles (T_M, T_N) for a TSMTTSM shape, preferring
    divisors of M and N (no guards, no idle threads; Sec. 5.2) and tiles whose
    thread count P = ceil(M/T_M) ceil(N/T_N) fits one CTA."""
    cap = 16 if cplx else 32          # accumulators per thread (doubles)
    cands = []
    for tm in (1, 2, 4, 8, 16):
        for tn in (1, 2, 4, 8, 16):
            if tm > M or tn > N:
                continue
            acc = tm * tn * (2 if cplx else 1)
            if acc > cap:
                continue
            P = math.ceil(M / tm) * math.ceil(N / tn)
            if P > BLOCK:
                continue
            divides = (M % tm == 0) and (N % tn == 0)
            squareness = -abs(math.log2(tm) - math.log2(tn))
            cands.append((divides, tm * tn, squareness, tm, tn))
    cands.sort(reverse=True)
    out = []
    for c in cands:
        if (c[3], c[4]) not in out:
            out.append((c[3], c[4]))
        if len(out) == 3:
            break
    return out


def tile_for_width(w, cplx, cap=40, min_lanes=1):
    """Register tile (T_M, T_N) for the square width w: the least padded
    work P T_M T_N / w^2 (a guarded FMA still costs its FP64 issue slot),
    then the larger tile (fewer loads per FMA), then the squarer one;
    at most `cap` accumulator doubles, and at least `min_lanes` row lanes
    (256 // P) per CTA.  None if no tile meets the limits."""
    best = None
    c = 2 if cplx else 1
    for tm in range(1, w + 1):
        for tn in range(1, w + 1):
            if tm * tn * c > cap:
                continue
            P = math.ceil(w / tm) * math.ceil(w / tn)
            if P > BLOCK // min_lanes:
                continue
            waste = P * tm * tn / (w * w)
            key = (round(waste, 6), -tm * tn, abs(math.log2(tm) - math.log2(tn)), -tm)
            if best is None or key < best[0]:
                best = (key, tm, tn)
    return None if best is None else (best[1], best[2])


def tile_regs(tm, tn, cplx, rows=1):
    """Rough register count of a TSMTTSM thread with a tm x tn tile: the
    accumulators, the operands of `rows` rows in flight and about 24 for
    addresses and the loop."""
    c = 2 if cplx else 1
    return 2 * c * (tm * tn + rows * (tm + tn)) + 24


def warp_fill(w, tm, tn, block):
    """Share of the FP64 issue slots a CTA of `block` threads spends on
    useful FMAs for the square width w and tile tm x tn: its L = block // P
    row lanes hold L * P active threads, every warp with at least one of
    them issues all 32 lanes' FMAs (an idle lane of a partly filled warp
    still takes its slot of this part's FP64 pipe), and the tile's padded
    entries are wasted too."""
    P = math.ceil(w / tm) * math.ceil(w / tn)
    L = block // P
    if L < 1:
        return 0.0
    return w * w * L / (math.ceil(L * P / 32) * 32 * tm * tn)


def fullwarp_tile(w, cplx, cap=40):
    """(T_M, T_N, block) for the square width w that maximises warp_fill
    over tiles of at most `cap` accumulator doubles and CTAs of 128..1024
    threads (multiples of 32) whose estimated registers fit one CTA per SM;
    ties go to fewer registers, then to the block closest to 256."""
    c = 2 if cplx else 1
    best = None
    for tm in range(1, w + 1):
        for tn in range(1, w + 1):
            if tm * tn * c > cap:
                continue
            r = tile_regs(tm, tn, cplx)
            for block in range(128, 1025, 32):
                if r * block > 65536 or r > 255:
                    break
                key = (-round(warp_fill(w, tm, tn, block), 3), r, abs(block - 256), tm)
                if best is None or key < best[0]:
                    best = (key, tm, tn, block)
    return best[1], best[2], best[3]


def tpr_options(N, cplx, k=2):
    """Up to k TSMM (threads per row t, results per thread npt) choices for
    N columns: the least padding npt t - N, then npt closest to 4 (the
    measured optimum of the tuned widths), then the larger npt."""
    opts = []
    for npt in range(1, (8 if cplx else 16) + 1):
        t = math.ceil(N / npt)
        if t > 64 or any(o[1] == t for o in opts):
            continue
        opts.append(((npt * t - N, abs(npt - 4), -npt), t, npt))
    opts.sort()
    return [(t, npt) for _, t, npt in opts[:k]]


def tsmm_fill(N, tpr, npt, block):
    """Share of the FP64 issue slots a TSMM CTA of `block` threads spends on
    useful FMAs: block // tpr rows per step, every warp with an active
    thread issues all 32 lanes, and npt * tpr - N padded result slots are
    wasted."""
    rpc = block // tpr
    return N * rpc / (math.ceil(rpc * tpr / 32) * 32 * npt)


def tsmm_block(N, tpr, npt):
    """CTA size for a TSMM kernel with `tpr` threads per row: a multiple of
    lcm(tpr, 32) (every warp full) in 128..1024 closest to 256 when that
    fills the warps better than 256 threads, else 256."""
    lcm = tpr * 32 // math.gcd(tpr, 32)
    sizes = [lcm * j for j in range(1, 1024 // lcm + 1) if lcm * j >= 128]
    if not sizes:
        return BLOCK
    b = min(sizes, key=lambda x: (abs(x - BLOCK), x))
    return b if tsmm_fill(N, tpr, npt, b) > tsmm_fill(N, tpr, npt, BLOCK) + 1e-9 else BLOCK


def tpr_for_width(N, cplx):
    """The first of tpr_options: (threads per row, results per thread)."""
    return tpr_options(N, cplx, 1)[0]


def default_specs():
    tsmttsm, tsmm = [], []
    shapes = [(w, w) for w in SWEEP_SQUARE] + list(SWEEP_OFFDIAG)
    for cplx in (False, True):
        for (M, N) in shapes:
            for (tm, tn) in _tiles_for(M, N, cplx):
                U = 4 if tm * tn <= 2 else (2 if tm * tn <= 8 else 1)
                tsmttsm.append(dict(cplx=cplx, M=M, N=N, TM=tm, TN=tn, U=U))
    # one width-specialised kernel per product for every other square width
    # (every w in 1..64 has a kernel without padding, or with at most a few
    # per cent of it, as the paper's generator does for each size, Sec. 2.1)
    # Two or three candidates per width for the tuner: the least-padded
    # tile, the same tile with two rows in flight per thread (U = 2) when its
    # accumulators leave room, and, when the least-padded tile leaves a
    # single row lane per CTA, the best tile with at least two; for TSMM the
    # two best thread counts per row.
    for cplx in (False, True):
        c = 2 if cplx else 1
        for w in range(1, 65):
            if w in SWEEP_SQUARE:
                continue
            tiles = []
            tm, tn = tile_for_width(w, cplx)
            U = 4 if tm * tn <= 2 else (2 if tm * tn <= 8 else 1)
            tiles.append((tm, tn, U))
            if U == 1 and tm * tn * c <= 24:
                tiles.append((tm, tn, 2))
            P = math.ceil(w / tm) * math.ceil(w / tn)
            if BLOCK // P < 2:
                t2 = tile_for_width(w, cplx, min_lanes=2)
                if t2 is not None and t2 != (tm, tn):
                    tiles.append((t2[0], t2[1], 4 if t2[0] * t2[1] <= 2 else (2 if t2[0] * t2[1] <= 8 else 1)))
            specs = [dict(cplx=cplx, M=w, N=w, TM=a, TN=b, U=u) for (a, b, u) in tiles]
            # the tile and CTA size that keep every warp's lanes busy
            # (warp_fill); added unless a 256-thread candidate already is it
            fm, fn, fb = fullwarp_tile(w, cplx)
            fu = 4 if fm * fn <= 2 else (2 if fm * fn <= 8 else 1)
            while fu > 1 and tile_regs(fm, fn, cplx, fu) * fb > 65536:
                fu //= 2
            if not (fb == BLOCK and any((x["TM"], x["TN"]) == (fm, fn) for x in specs)):
                specs.append(dict(cplx=cplx, M=w, N=w, TM=fm, TN=fn, U=fu, B=fb))
            tsmttsm.extend(specs)
            for tpr, npt in tpr_options(w, cplx, 2):
                spec = dict(cplx=cplx, M=w, N=w, TPR=tpr, U=2 if npt * c <= 8 else 1)
                blk = tsmm_block(w, tpr, npt)
                if blk != BLOCK:
                    spec["B"] = blk
                tsmm.append(spec)
    tshapes = [(w, w) for w in SWEEP_SQUARE] + list(TSMM_OFFDIAG)
    for cplx in (False, True):
        for (M, N) in tshapes:
            tprs = sorted({min(t, N) for t in (4, 8, 16)})
            for tpr in tprs:
                npt = math.ceil(N / tpr)
                U = 2 if npt * (2 if cplx else 1) <= 8 else 1
                tsmm.append(dict(cplx=cplx, M=M, N=N, TPR=tpr, U=U))
    return tsmttsm, tsmm


def _name_tsmttsm(s):
    name = "gen_tsmttsm_%s_m%dn%d_t%dx%d_u%d" % ("c64" if s["cplx"] else "r64", s["M"], s["N"],
                                                 s["TM"], s["TN"], s["U"])
    return name + ("_b%d" % s["B"] if s.get("B", BLOCK) != BLOCK else "")


def _name_tsmm(s):
    name = "gen_tsmm_%s_m%dn%d_tpr%d_u%d" % ("c64" if s["cplx"] else "r64", s["M"], s["N"],
                                             s["TPR"], s["U"])
    return name + ("_b%d" % s["B"] if s.get("B", BLOCK) != BLOCK else "")


def emit_tsmttsm(s):
    """One TSMTTSM kernel for fixed M, N, tile and unroll."""
    M, N, TM, TN, U, cplx = s["M"], s["N"], s["TM"], s["TN"], s["U"], s["cplx"]
    BLK = s.get("B", BLOCK)
    CC = 2 if cplx else 1
    PM, PN = math.ceil(M / TM), math.ceil(N / TN)
    P = PM * PN
    L = BLK // P
    name = _name_tsmttsm(s)
    # entry i is always in range iff the largest pm (PM - 1) still fits
    gm = [(PM - 1) + i * PM >= M for i in range(TM)]
    gn = [(PN - 1) + j * PN >= N for j in range(TN)]
    o = []
    w = o.append
    w("template <bool CONJ>")
    w("__global__ void __launch_bounds__(%d) %s(const TsmttsmArgs a) {" % (BLK, name))
    w("    tsmttsm_begin(a);")
    w("    constexpr int PM = %d, PN = %d, P = %d, L = %d;" % (PM, PN, P, L))
    w("    const int t = threadIdx.x;")
    w("    const int lane = t / P, p = t - lane * P;")
    w("    const int pm = p % PM, pn = p / PM;")
    w("    const bool active = %s;" % ("lane < L" if L * P < BLK else "true"))
    for i in range(TM):
        if gm[i]:
            w("    const bool gm%d = pm + %d < %d;" % (i, i * PM, M))
    for j in range(TN):
        if gn[j]:
            w("    const bool gn%d = pn + %d < %d;" % (j, j * PN, N))
    for i in range(TM):
        for j in range(TN):
            for c in range(CC):
                w("    double c%d_%d_%d = 0.0;" % (i, j, c))
    w("    const int64_t G = gridDim.x;")
    w("    const int64_t k0 = a.K * (int64_t)blockIdx.x / G;")
    w("    const int64_t k1 = a.K * ((int64_t)blockIdx.x + 1) / G;")
    w("    const double* __restrict__ Ab = a.A + pm * %d;" % CC)
    w("    const double* __restrict__ Bb = a.B + pn * %d;" % CC)
    w("    const int64_t sa = a.lda * %d, sb = a.ldb * %d;" % (CC, CC))

    def body(rows):
        lines = []
        for u in range(rows):
            off = "" if u == 0 else " + (int64_t)%d * L" % u
            lines.append("            const double* ar%d = Ab + (k%s) * sa;" % (u, off))
            lines.append("            const double* br%d = Bb + (k%s) * sb;" % (u, off))
        for u in range(rows):
            for i in range(TM):
                for c in range(CC):
                    ld = "__ldg(ar%d + %d)" % (u, i * PM * CC + c)
                    if gm[i]:
                        ld = "gm%d ? %s : 0.0" % (i, ld)
                    lines.append("            const double a%d_%d_%d = %s;" % (u, i, c, ld))
            for j in range(TN):
                for c in range(CC):
                    ld = "__ldg(br%d + %d)" % (u, j * PN * CC + c)
                    if gn[j]:
                        ld = "gn%d ? %s : 0.0" % (j, ld)
                    lines.append("            const double b%d_%d_%d = %s;" % (u, j, c, ld))
        for u in range(rows):
            for i in range(TM):
                for j in range(TN):
                    guard = []
                    if gm[i]:
                        guard.append("gm%d" % i)
                    if gn[j]:
                        guard.append("gn%d" % j)
                    pre = ("if (%s) " % " && ".join(guard)) if guard else ""
                    if not cplx:
                        lines.append("            %sc%d_%d_0 = fma(a%d_%d_0, b%d_%d_0, c%d_%d_0);"
                                     % (pre, i, j, u, i, u, j, i, j))
                    else:
                        A_r, A_i = "a%d_%d_0" % (u, i), "a%d_%d_1" % (u, i)
                        B_r, B_i = "b%d_%d_0" % (u, j), "b%d_%d_1" % (u, j)
                        cr, ci = "c%d_%d_0" % (i, j), "c%d_%d_1" % (i, j)
                        lines.append("            %s{" % pre)
                        lines.append("                %s = fma(%s, %s, %s);" % (cr, A_r, B_r, cr))
                        lines.append("                %s = fma(CONJ ? %s : -%s, %s, %s);" % (cr, A_i, A_i, B_i, cr))
                        lines.append("                %s = fma(%s, %s, %s);" % (ci, A_r, B_i, ci))
                        lines.append("                %s = fma(CONJ ? -%s : %s, %s, %s);" % (ci, A_i, A_i, B_r, ci))
                        lines.append("            }")
        return lines

    w("    if (active) {")
    w("        int64_t k = k0 + lane;")
    if U > 1:
        w("        for (; k + (int64_t)%d * L < k1; k += (int64_t)%d * L) {" % (U - 1, U))
        o.extend(body(U))
        w("        }")
    w("        for (; k < k1; k += L) {")
    o.extend(body(1))
    w("        }")
    w("    }")
    accs = ", ".join("c%d_%d_%d" % (i, j, c) for i in range(TM) for j in range(TN) for c in range(CC))
    w("    const double acc[%d] = {%s};" % (TM * TN * CC, accs))
    w("    tsmttsm_finish<%d, %d, %d, %d>(a, acc, PM, PN, L, lane, p, active);" % (TM, TN, CC, BLK))
    w("}")
    w("")
    w("cudaError_t launch_%s(const TsmttsmArgs& a, int grid, cudaStream_t s) {" % name)
    if cplx:
        w("    if (a.conj) return launch_pdl(%s<true>, grid, %d, 0, s, a);" % (name, BLK))
        w("    return launch_pdl(%s<false>, grid, %d, 0, s, a);" % (name, BLK))
    else:
        w("    return launch_pdl(%s<false>, grid, %d, 0, s, a);" % (name, BLK))
    w("}")
    w("int occ_%s(int, int) {" % name)
    w("    int n = 0;")
    w("    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, %s<false>, %d, 0) != cudaSuccess) return 0;"
      % (name, BLK))
    w("    return n;")
    w("}")
    w("")
    return "\n".join(o)


def emit_tsmm(s):
    """One TSMM kernel for fixed M, N, threads per row and unroll; C comes
    from shared memory (Sec. 4.2), the m loop is fully unrolled."""
    M, N, TPR, U, cplx = s["M"], s["N"], s["TPR"], s["U"], s["cplx"]
    BLK = s.get("B", BLOCK)
    CC = 2 if cplx else 1
    NPT = math.ceil(N / TPR)
    RPC = BLK // TPR
    name = _name_tsmm(s)
    gn = [(TPR - 1) + j * TPR >= N for j in range(NPT)]
    o = []
    w = o.append
    # Kernels with at most 8 threads per row are instantiated twice, for beta
    # in {0, 1} and for any other beta (tsmm_acc_init); the others keep one
    # instantiation (tsmm_acc_init_kept): measured side by side, the split
    # helped the former and slowed the latter.
    split = TPR <= 8
    if split:
        w("template <bool GEN>")
    w("__global__ void __launch_bounds__(%d) %s(const TsmmArgs a) {" % (BLK, name))
    w("    extern __shared__ double cs[];")
    w("    tsmm_begin(a);")
    w("    tsmm_stage_c<%d>(a, cs);" % CC)
    w("    constexpr int TPR = %d, RPC = %d;" % (TPR, RPC))
    w("    const int r = threadIdx.x / TPR, q = threadIdx.x - r * TPR;")
    # threads past RPC * TPR (TPR not dividing the block) hold no row
    live = "" if BLK % TPR == 0 else "r < RPC && "
    for j in range(NPT):
        if gn[j]:
            w("    const bool gn%d = q + %d < %d;" % (j, j * TPR, N))
    w("    const int64_t sa = a.lda * %d, sb = a.ldb * %d;" % (CC, CC))
    w("    const int64_t step = (int64_t)gridDim.x * RPC * %d;" % U)
    w("    for (int64_t base = (int64_t)blockIdx.x * RPC * %d + r; base - r < a.K; base += step) {" % U)
    for u in range(U):
        w("        const bool rok%d = %sbase + %d < a.K;" % (u, live, u * RPC))
        w("        const double* ar%d = a.A + (rok%d ? base + %d : 0) * sa;" % (u, u, u * RPC))
    for u in range(U):
        for j in range(NPT):
            for c in range(CC):
                w("        double x%d_%d_%d = 0.0, o%d_%d_%d = 0.0;" % (u, j, c, u, j, c))
    # beta != 0: the old B values are loaded before the FMAs, so their
    # latency overlaps them instead of stalling the stores, and the beta
    # term opens each FMA chain (no extra FP64 operation for beta = 1)
    w("        if (!a.beta_zero) {")
    for u in range(U):
        w("            if (rok%d) {" % u)
        w("                const double* bo = a.B + (base + %d) * sb;" % (u * RPC))
        for j in range(NPT):
            guard = ("if (gn%d) " % j) if gn[j] else ""
            w("                %s{" % guard)
            for c in range(CC):
                w("                    o%d_%d_%d = bo[(q + %d) * %d + %d];" % (u, j, c, j * TPR, CC, c))
            w("                    %s(a, o%d_%d_0, o%d_%d_%d, x%d_%d_0, x%d_%d_%d);"
              % (("tsmm_acc_init<%d, GEN>" if split else "tsmm_acc_init_kept<%d>") % CC,
                 u, j, u, j, CC - 1, u, j, u, j, CC - 1))
            w("                }")
        w("            }")
    w("        }")
    for m in range(M):
        for u in range(U):
            for c in range(CC):
                w("        const double a%d_%d_%d = rok%d ? __ldg(ar%d + %d) : 0.0;" % (u, m, c, u, u, m * CC + c))
        for j in range(NPT):
            guard = ("if (gn%d) " % j) if gn[j] else ""
            w("        %s{" % guard)
            for c in range(CC):
                w("            const double c%d = cs[(%d * %d + q + %d) * %d + %d];" % (c, m, N, j * TPR, CC, c))
            for u in range(U):
                if not cplx:
                    w("            x%d_%d_0 = fma(a%d_%d_0, c0, x%d_%d_0);" % (u, j, u, m, u, j))
                else:
                    w("            x%d_%d_0 = fma(a%d_%d_0, c0, x%d_%d_0);" % (u, j, u, m, u, j))
                    w("            x%d_%d_0 = fma(-a%d_%d_1, c1, x%d_%d_0);" % (u, j, u, m, u, j))
                    w("            x%d_%d_1 = fma(a%d_%d_0, c1, x%d_%d_1);" % (u, j, u, m, u, j))
                    w("            x%d_%d_1 = fma(a%d_%d_1, c0, x%d_%d_1);" % (u, j, u, m, u, j))
            w("        }")
    for u in range(U):
        w("        if (rok%d) {" % u)
        w("            double* out = a.B + (base + %d) * sb;" % (u * RPC))
        for j in range(NPT):
            guard = ("if (gn%d) " % j) if gn[j] else ""
            w("            %stsmm_store_plain<%d>(out, q + %d, x%d_%d_0, x%d_%d_%d);"
              % (guard, CC, j * TPR, u, j, u, j, CC - 1))
        w("        }")
    w("    }")
    w("}")
    w("")
    smem = M * N * CC * 8
    # with the split, a beta other than 0 and 1 takes GEN = true
    base = name + "<false>" if split else name
    w("cudaError_t launch_%s(const TsmmArgs& a, int grid, cudaStream_t s) {" % name)
    if split:
        w("    const bool gen = tsmm_general_beta(a);")
        if smem > 48 * 1024:
            w("    cudaError_t e = cudaFuncSetAttribute(gen ? %s<true> : %s<false>, "
              "cudaFuncAttributeMaxDynamicSharedMemorySize, %d);" % (name, name, smem))
            w("    if (e != cudaSuccess) return e;")
        w("    if (gen) return launch_pdl(%s<true>, grid, %d, %d, s, a);" % (name, BLK, smem))
        w("    return launch_pdl(%s<false>, grid, %d, %d, s, a);" % (name, BLK, smem))
    else:
        if smem > 48 * 1024:
            w("    cudaError_t e = cudaFuncSetAttribute(%s, cudaFuncAttributeMaxDynamicSharedMemorySize, %d);"
              % (name, smem))
            w("    if (e != cudaSuccess) return e;")
        w("    return launch_pdl(%s, grid, %d, %d, s, a);" % (name, BLK, smem))
    w("}")
    w("int occ_%s(int, int) {" % name)
    if smem > 48 * 1024:
        w("    if (cudaFuncSetAttribute(%s, cudaFuncAttributeMaxDynamicSharedMemorySize, %d) != cudaSuccess)"
          " return 0;" % (base, smem))
    w("    int n = 0;")
    w("    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, %s, %d, %d) != cudaSuccess) return 0;"
      % (base, BLK, smem))
    w("    return n;")
    w("}")
    w("")
    return "\n".join(o)


HEADER = """// GENERATED by paper_1905_03136_gb300/codegen.py -- do not edit.
#include <cstdio>
#include <cstring>
#include "fp64_common.cuh"
#include "tsm_internal.h"
namespace tsm {
"""


def _reg_tsmttsm(s):
    name = _name_tsmttsm(s)
    return ("    { Variant v; memset(&v, 0, sizeof(v)); snprintf(v.info.name, sizeof(v.info.name), \"%s\");"
            " v.info.kind = TSM_KIND_TSMTTSM; v.info.dtype = %d; v.info.fixed_m = %d; v.info.fixed_n = %d;"
            " v.info.tile_m = %d; v.info.tile_n = %d; v.info.unroll = %d; v.info.block = %d;"
            " v.info.generated = 1; v.tsmttsm = launch_%s; v.occupancy = occ_%s; t.push_back(v); }"
            % (name, 1 if s["cplx"] else 0, s["M"], s["N"], s["TM"], s["TN"], s["U"], s.get("B", BLOCK), name,
               name))


def _reg_tsmm(s):
    name = _name_tsmm(s)
    npt = math.ceil(s["N"] / s["TPR"])
    return ("    { Variant v; memset(&v, 0, sizeof(v)); snprintf(v.info.name, sizeof(v.info.name), \"%s\");"
            " v.info.kind = TSM_KIND_TSMM; v.info.dtype = %d; v.info.fixed_m = %d; v.info.fixed_n = %d;"
            " v.info.tile_n = %d; v.info.threads_per_row = %d; v.info.unroll = %d; v.info.block = %d;"
            " v.info.generated = 1; v.tsmm = launch_%s; v.occupancy = occ_%s; m.push_back(v); }"
            % (name, 1 if s["cplx"] else 0, s["M"], s["N"], npt, s["TPR"], s["U"], s.get("B", BLOCK), name,
               name))


def generate(out_dir, shards=16, specs=None):
    """Writes gen_shard{i}.cu (kernels) and gen_registry.cu; returns the list
    of written files.  Files whose content is unchanged are not rewritten,
    so incremental builds skip them."""
    tsmttsm, tsmm = specs if specs is not None else default_specs()
    os.makedirs(out_dir, exist_ok=True)
    items = [("t", s) for s in tsmttsm] + [("m", s) for s in tsmm]
    # balance shards by a rough code-size estimate
    def cost(it):
        k, s = it
        if k == "t":
            return s["TM"] * s["TN"] * s["U"] * (4 if s["cplx"] else 1) + 8
        return s["M"] * math.ceil(s["N"] / s["TPR"]) * s["U"] * (4 if s["cplx"] else 1) + 8
    bins = [[] for _ in range(shards)]
    loads = [0] * shards
    for it in sorted(items, key=cost, reverse=True):
        b = loads.index(min(loads))
        bins[b].append(it)
        loads[b] += cost(it)
    files = []
    decls = []
    for i, b in enumerate(bins):
        src = [HEADER]
        for k, s in b:
            src.append(emit_tsmttsm(s) if k == "t" else emit_tsmm(s))
        src.append("}  // namespace tsm\n")
        files.append(_write(os.path.join(out_dir, "gen_shard%d.cu" % i), "\n".join(src)))
    for s in tsmttsm:
        n = _name_tsmttsm(s)
        decls.append("cudaError_t launch_%s(const TsmttsmArgs&, int, cudaStream_t); int occ_%s(int, int);" % (n, n))
    for s in tsmm:
        n = _name_tsmm(s)
        decls.append("cudaError_t launch_%s(const TsmmArgs&, int, cudaStream_t); int occ_%s(int, int);" % (n, n))
    reg = [HEADER] + decls + ["void register_generated_variants(std::vector<Variant>& t, std::vector<Variant>& m) {"]
    reg += [_reg_tsmttsm(s) for s in tsmttsm] + [_reg_tsmm(s) for s in tsmm]
    reg += ["}", "}  // namespace tsm", ""]
    files.append(_write(os.path.join(out_dir, "gen_registry.cu"), "\n".join(reg)))
    return files


def _write(path, text):
    if os.path.exists(path):
        with open(path) as f:
            if f.read() == text:
                return path
    with open(path, "w") as f:
        f.write(text)
    return path


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("out_dir")
    ap.add_argument("--shards", type=int, default=16)
    args = ap.parse_args()
    for f in generate(args.out_dir, args.shards):
        print(f)


if __name__ == "__main__":
    main()
