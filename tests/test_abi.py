"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/*.h, describes its variants consistently, and rejects
malformed arguments before touching a device."""

import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_03136_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tsm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_headers_declare_entry_points():
    names = _declared_functions()
    for required in ("tsm_tsmttsm", "tsm_tsmm", "tsm_status_string", "tsm_tune", "tsm_fill_random"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1905_03136_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(tsm_\w+)", out))
    missing = _declared_functions() - exported
    assert not missing, "declared but not exported: %s" % sorted(missing)


def test_binding_covers_declared_functions(lib):
    import importlib
    import pkgutil
    import paper_1905_03136_gb300 as pkg
    from paper_1905_03136_gb300 import _lib
    # sub-modules register the signatures of their headers on import
    for m in pkgutil.iter_modules(pkg.__path__):
        if m.name not in ("build", "codegen", "__main__", "libtsm"):
            importlib.import_module("paper_1905_03136_gb300." + m.name)
    missing = _declared_functions() - set(_lib.SIGNATURES)
    assert not missing, "no Python binding for: %s" % sorted(missing)


def test_kernels_per_call_rule(lib):
    """One launch per TSMTTSM call, two when grid * M * N * c CTA partial
    doubles exceed 32768 (the final reduction pass); -1 for bad shapes."""
    import paper_1905_03136_gb300 as t
    assert lib.tsm_tsmttsm_kernels_per_call(t.R64, 1, 1, 304) == 1
    assert lib.tsm_tsmttsm_kernels_per_call(t.R64, 16, 16, 128) == 1      # 32768: not above
    assert lib.tsm_tsmttsm_kernels_per_call(t.R64, 16, 16, 129) == 2
    assert lib.tsm_tsmttsm_kernels_per_call(t.C64, 64, 64, 152) == 2
    assert lib.tsm_tsmttsm_kernels_per_call(t.C64, 8, 8, 256) == 1       # 32768 complex doubles
    for bad in ((0, 1, 1), (65, 1, 1), (1, 1, 0)):
        assert lib.tsm_tsmttsm_kernels_per_call(t.R64, bad[0], bad[1], bad[2]) == -1


def test_timed_tuning_entry_round_trip(lib, tmp_path):
    """tsm_set_tuning_timed records (variant, grid, ms) under its key and the
    table file keeps them; a variant that cannot run the shape is refused.
    Host-only table logic: no device needed.  The loaded table is restored."""
    import paper_1905_03136_gb300 as t
    from paper_1905_03136_gb300 import _lib
    saved = str(tmp_path / "saved.txt").encode()
    _lib.call("tsm_save_tuning", saved)
    try:
        lib.tsm_clear_tuning()
        vs = t.variants(t.KIND_TSMTTSM)
        gen = [v for v in vs if v["name"] == "gen_tsmttsm_r64_m37n37_t1x37_u1"
               or (v["fixed_m"] == 37 and v["dtype"] == 0)]
        assert gen, "no generated kernel for real width 37"
        v = gen[0]
        assert lib.tsm_set_tuning_timed(t.KIND_TSMTTSM, t.R64, 37, 37, 1 << 24, v["index"], 304,
                                        ctypes.c_float(12.5)) == 0
        # a kernel fixed to width 37 cannot run 36 x 36
        assert lib.tsm_set_tuning_timed(t.KIND_TSMTTSM, t.R64, 36, 36, 1 << 24, v["index"], 304,
                                        ctypes.c_float(1.0)) == 1
        out = str(tmp_path / "t.txt")
        _lib.call("tsm_save_tuning", out.encode())
        lines = [l.split() for l in open(out) if not l.startswith("#")]
        assert lines == [["0", "0", "37", "37", "24", v["name"], "304", "12.500000"]]
    finally:
        lib.tsm_clear_tuning()
        _lib.call("tsm_load_tuning", saved)


def test_status_strings(lib):
    for s in range(8):
        assert lib.tsm_status_string(s)
    assert lib.tsm_status_string(99) == b"unknown status"


def test_variant_table(lib):
    import paper_1905_03136_gb300 as t
    for kind in (t.KIND_TSMTTSM, t.KIND_TSMM):
        vs = t.variants(kind)
        assert len(vs) > 10
        names = [v["name"] for v in vs]
        assert len(set(names)) == len(names)
        assert any(v["generated"] for v in vs) and any(not v["generated"] for v in vs)
        for v in vs:
            assert v["kind"] == kind and v["dtype"] in (0, 1)
    info = t.VariantInfo()
    assert lib.tsm_variant_get(0, 10 ** 6, ctypes.byref(info)) == 1
    assert lib.tsm_variant_count(7) == -1
    # the TSMM-with-beta tuning key names the TSMM variants
    assert lib.tsm_variant_count(t.KIND_TSMM_BETA) == lib.tsm_variant_count(t.KIND_TSMM)


def test_generic_variant_supports_every_shape(lib):
    import paper_1905_03136_gb300 as t
    for kind in (t.KIND_TSMTTSM, t.KIND_TSMM):
        for dt in (t.R64, t.C64):
            for M in (1, 3, 17, 64):
                for N in (1, 5, 32, 64):
                    ok = [i for i in range(lib.tsm_variant_count(kind))
                          if lib.tsm_variant_supports(kind, i, dt, M, N)]
                    assert ok, (kind, dt, M, N)


def _call_tsmttsm(lib, op=1, dt=0, M=4, N=4, K=10, lda=4, ldb=4, ldc=4, A=1, B=1, C=1, alpha=True,
                  beta=True):
    from paper_1905_03136_gb300._lib import scalar
    return lib.tsm_tsmttsm(op, dt, M, N, K, scalar(1.0, 1) if alpha else None, ctypes.c_void_p(A),
                           lda, ctypes.c_void_p(B), ldb, scalar(0.0, 1) if beta else None,
                           ctypes.c_void_p(C), ldc, None)


def test_argument_validation_without_device(lib):
    INVALID, UNSUPPORTED = 1, 2
    assert _call_tsmttsm(lib, M=0) == UNSUPPORTED
    assert _call_tsmttsm(lib, N=65) == UNSUPPORTED
    assert _call_tsmttsm(lib, K=-1) == INVALID
    assert _call_tsmttsm(lib, op=0) == INVALID
    assert _call_tsmttsm(lib, op=7) == INVALID
    assert _call_tsmttsm(lib, dt=5) == INVALID
    assert _call_tsmttsm(lib, lda=3) == INVALID
    assert _call_tsmttsm(lib, ldb=2) == INVALID
    assert _call_tsmttsm(lib, ldc=3) == INVALID
    assert _call_tsmttsm(lib, C=0) == INVALID
    assert _call_tsmttsm(lib, A=0) == INVALID
    assert _call_tsmttsm(lib, alpha=False) == INVALID
    assert _call_tsmttsm(lib, beta=False) == INVALID
    from paper_1905_03136_gb300._lib import scalar
    # TSMM: only op N; transposed C is a valid request this library does not implement
    one, zero = scalar(1.0, 0), scalar(0.0, 0)
    assert lib.tsm_tsmm(1, 0, 4, 4, 10, one, ctypes.c_void_p(1), 4, ctypes.c_void_p(1), 4, zero,
                        ctypes.c_void_p(1), 4, None) == UNSUPPORTED
    assert lib.tsm_tsmm(9, 0, 4, 4, 10, one, ctypes.c_void_p(1), 4, ctypes.c_void_p(1), 4, zero,
                        ctypes.c_void_p(1), 4, None) == INVALID
    assert lib.tsm_tsmm(0, 0, 4, 4, 10, one, ctypes.c_void_p(1), 3, ctypes.c_void_p(1), 4, zero,
                        ctypes.c_void_p(1), 4, None) == INVALID
    assert lib.tsm_tsmm(0, 0, 4, 4, 10, one, ctypes.c_void_p(1), 4, ctypes.c_void_p(1), 4, zero,
                        ctypes.c_void_p(0), 4, None) == INVALID
    assert lib.tsm_fill_random(ctypes.c_void_p(1), 0, 4, 4, 0, 0, 9, None) == INVALID
    # split path precision knobs: an unknown split kind is malformed, a slice
    # count outside [4, 6] is valid but not implemented
    from paper_1905_03136_gb300 import split  # noqa: F401  (registers the signatures)

    def split_ex(kind, slices):
        return lib.tsm_tsmttsm_split_ex(1, 0, 4, 4, 10, one, ctypes.c_void_p(1), 4, ctypes.c_void_p(1), 4, zero,
                                        ctypes.c_void_p(1), 4, kind, slices, None)
    assert split_ex(1, 6) == INVALID
    assert split_ex(-1, 6) == INVALID
    for bad in (0, 3, 7, 8):
        assert split_ex(0, bad) == UNSUPPORTED, bad
    info = split.PlanInfo()
    for bad in (3, 7):
        assert lib.tsm_split_plan_ex(0, 4, 4, 100, bad, ctypes.byref(info)) == UNSUPPORTED


def test_no_device_is_an_error_not_a_fallback(lib):
    """Without a GPU a well-formed call must fail (NO_DEVICE), never compute
    on the host."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    assert _call_tsmttsm(lib) == 7
