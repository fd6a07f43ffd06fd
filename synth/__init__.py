"""Seeded synthetic inputs for tall & skinny block vectors.

This module is the only code shared by the CPU oracle side and the CUDA
side.  It holds no arithmetic of the matrix products; it only turns
(seed, linear element index) into a double with a stated distribution.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  The i-th output of a
SplitMix64 stream seeded with ``seed`` is ``mix(seed + (i + 1) * GAMMA)``,
so every element can be computed independently of the others
(counter-based).  The CUDA library carries its own implementation of the
same definition (``tsm_fill_random``); a GPU test checks the two bitwise.

Element addressing: a row-major block vector with leading dimension ``ld``
stores element (k, m) at linear index ``i = k * ld + m``.  A real element
draws output ``i``; a complex element draws outputs ``2 i`` (real part) and
``2 i + 1`` (imaginary part).  Padding elements (m >= width) are drawn too,
so a buffer's contents do not depend on the logical width.

Distributions:
  * ``uniform``     : ``(h >> 11) * 2**-52 - 1``, uniform on [-1, 1) in
                      steps of 2**-52 (exact in binary64).
  * ``loguniform``  : sign from bit 11, binary exponent
                      ``e = -20 + ((h & 0x7ff) * 40 >> 11)`` in [-20, 19],
                      52-bit mantissa ``h >> 12``; value
                      ``+-(1 + mant * 2**-52) * 2**e`` (magnitudes spread over
                      2**-20 .. 2**20, exact in binary64).
  * ``smallint``    : ``(h >> 60) - 8``, integers in [-8, 7]; products and
                      sums of these stay exact in binary64.
  * ``ones``        : all 1.0 (no draw).

Default seeds (matrix tags): A = 0, B = 1, C = 2.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DISTS = ("uniform", "loguniform", "smallint", "ones")
DIST_CODE = {"uniform": 0, "loguniform": 1, "smallint": 2, "ones": 3}

SEED_A, SEED_B, SEED_C = 0, 1, 2


def _mix(z):
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed, idx):
    """Outputs number ``idx`` (uint64 array) of the stream seeded with ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * GAMMA
        return _mix(z)


def _to_double(h, dist):
    if dist == "uniform":
        return (h >> np.uint64(11)).astype(np.float64) * 2.0**-52 - 1.0
    if dist == "loguniform":
        mant = (h >> np.uint64(12)).astype(np.float64) * 2.0**-52 + 1.0
        e = ((h & np.uint64(0x7FF)) * np.uint64(40)) >> np.uint64(11)
        e = e.astype(np.int64) - 20
        sign = np.where((h >> np.uint64(11)) & np.uint64(1), -1.0, 1.0)
        return sign * np.ldexp(mant, e)
    if dist == "smallint":
        return (h >> np.uint64(60)).astype(np.float64) - 8.0
    if dist == "ones":
        return np.ones(h.shape, dtype=np.float64)
    raise ValueError(f"unknown distribution {dist!r}")


def values(seed, idx, dist="uniform"):
    """Doubles for linear draw indices ``idx``."""
    idx = np.asarray(idx, dtype=np.uint64)
    if dist == "ones":
        return np.ones(idx.shape, dtype=np.float64)
    return _to_double(splitmix64(seed, idx), dist)


def block_vector(seed, rows, width, ld=None, complex_=False, dist="uniform",
                 row0=0):
    """Row-major block vector of ``rows`` x ``ld`` elements (rows starting at
    ``row0``), as a numpy array of shape (rows, ld), float64 or complex128.
    Only the first ``width`` columns are logically part of the matrix."""
    ld = width if ld is None else ld
    if ld < width:
        raise ValueError("ld < width")
    lin = (np.arange(rows, dtype=np.uint64)[:, None] + np.uint64(row0)) * np.uint64(ld) \
        + np.arange(ld, dtype=np.uint64)[None, :]
    if not complex_:
        return values(seed, lin, dist)
    re = values(seed, lin * np.uint64(2), dist)
    im = values(seed, lin * np.uint64(2) + np.uint64(1), dist)
    return re + 1j * im


def column(seed, rows, col, ld, complex_=False, dist="uniform", row0=0):
    """One column (length ``rows``) of a block vector, without generating
    the rest; used to check single entries of very tall products."""
    lin = (np.arange(rows, dtype=np.uint64) + np.uint64(row0)) * np.uint64(ld) + np.uint64(col)
    if not complex_:
        return values(seed, lin, dist)
    return values(seed, lin * np.uint64(2), dist) + 1j * values(seed, lin * np.uint64(2) + np.uint64(1), dist)


def rows_at(seed, row_idx, ld, complex_=False, dist="uniform"):
    """Selected rows (array of row indices) of a block vector, shape (len, ld)."""
    row_idx = np.asarray(row_idx, dtype=np.uint64)
    lin = row_idx[:, None] * np.uint64(ld) + np.arange(ld, dtype=np.uint64)[None, :]
    if not complex_:
        return values(seed, lin, dist)
    return values(seed, lin * np.uint64(2), dist) + 1j * values(seed, lin * np.uint64(2) + np.uint64(1), dist)


def small_matrix(seed, M, N, ld=None, complex_=False, dist="uniform"):
    """Dense row-major M x ld small matrix (the C operand)."""
    return block_vector(seed, M, N, ld, complex_, dist)
