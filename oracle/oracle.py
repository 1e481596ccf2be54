"""ctypes wrapper over the CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this module.  It never imports the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib: Optional[ctypes.CDLL] = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_matmul_mod_rows.argtypes = [_i64, _i64, _i64, _i64, _u64, _u64p, _i64, _u64p, _i64, _u64p, _i64, ctypes.c_int]
        L.oracle_matmul_mod.argtypes = [_i64, _i64, _i64, _u64, _u64p, _i64, _u64p, _i64, _u64p, _i64, ctypes.c_int]
        L.oracle_matmul_entries.argtypes = [_i64, _u64, _u64p, _i64, _u64p, _i64, _i64p, _i64p, _i64, _u64p, ctypes.c_int]
        L.oracle_freivalds.argtypes = [_i64, _i64, _i64, _u64, _u64p, _i64, _u64p, _i64, _u64p, _i64, _u64p, ctypes.c_int]
        L.oracle_freivalds.restype = ctypes.c_int64
        L.oracle_split_alpha.argtypes = [_u64p, _i64, _u64, ctypes.c_int, _u64p]
        L.oracle_split_signed8.argtypes = [_u64p, _i64, _u64, ctypes.c_int, _i32p]
        L.oracle_split_signed_bits.argtypes = [_u64p, _i64, _u64, ctypes.c_int, ctypes.c_int, _i32p]
        L.oracle_diag_sums.argtypes = [_i64, _i64, _i64, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i64p, ctypes.c_int]
        L.oracle_recombine_pow.argtypes = [_i64p, ctypes.c_int, _i64, _u64, _u64, _u64p]
        L.oracle_mod_vec.argtypes = [_f64p, _i64, _u64, _u64p]
        L.oracle_mulmod_vec.argtypes = [_u64p, _u64p, _i64, _u64, _u64p]
        L.oracle_ceil_root.argtypes = [_u64, ctypes.c_int]
        L.oracle_ceil_root.restype = _u64
        L.oracle_lambda.argtypes = [_u64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_lambda.restype = _u64
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def matmul_mod(A: np.ndarray, B: np.ndarray, p: int, nthreads: int = 0) -> np.ndarray:
    """C = A B mod p (Sec. 1), exact 128-bit accumulation."""
    A = _c(A, np.uint64)
    B = _c(B, np.uint64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.zeros((m, n), dtype=np.uint64)
    rc = lib().oracle_matmul_mod(m, n, k, p, _p(A, _u64p), max(k, 1), _p(B, _u64p), max(n, 1),
                                 _p(C, _u64p), max(n, 1), nthreads)
    if rc:
        raise RuntimeError("oracle_matmul_mod failed (%d)" % rc)
    return C


def matmul_mod_rows(A: np.ndarray, B: np.ndarray, p: int, r0: int, r1: int, nthreads: int = 0) -> np.ndarray:
    """Rows r0..r1-1 of A B mod p."""
    A = _c(A, np.uint64)
    B = _c(B, np.uint64)
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((r1 - r0, n), dtype=np.uint64)
    # shift A so that row r0 lands in C[0]
    Ash = A[r0:r1]
    rc = lib().oracle_matmul_mod_rows(0, r1 - r0, n, k, p, _p(np.ascontiguousarray(Ash), _u64p), max(k, 1),
                                      _p(B, _u64p), max(n, 1), _p(C, _u64p), max(n, 1), nthreads)
    if rc:
        raise RuntimeError("oracle_matmul_mod_rows failed (%d)" % rc)
    return C


def matmul_entries(A: np.ndarray, B: np.ndarray, p: int, rows, cols, nthreads: int = 0) -> np.ndarray:
    A = _c(A, np.uint64)
    B = _c(B, np.uint64)
    rows = _c(rows, np.int64)
    cols = _c(cols, np.int64)
    k = A.shape[1]
    out = np.zeros(rows.shape[0], dtype=np.uint64)
    lib().oracle_matmul_entries(k, p, _p(A, _u64p), A.shape[1], _p(B, _u64p), B.shape[1],
                                _p(rows, _i64p), _p(cols, _i64p), rows.shape[0], _p(out, _u64p), nthreads)
    return out


def freivalds(A: np.ndarray, B: np.ndarray, C: np.ndarray, p: int, x: np.ndarray, nthreads: int = 0) -> int:
    """Number of rows where C x != A (B x) mod p."""
    A = _c(A, np.uint64)
    B = _c(B, np.uint64)
    C = _c(C, np.uint64)
    x = _c(x, np.uint64)
    m, k = A.shape
    n = B.shape[1]
    bad = lib().oracle_freivalds(m, n, k, p, _p(A, _u64p), max(k, 1), _p(B, _u64p), max(n, 1),
                                 _p(C, _u64p), max(n, 1), _p(x, _u64p), nthreads)
    if bad < 0:
        raise RuntimeError("oracle_freivalds failed")
    return int(bad)


def split_alpha(M: np.ndarray, alpha: int, u: int) -> np.ndarray:
    """Alg. 4 words, shape (u,) + M.shape."""
    M = _c(M, np.uint64)
    W = np.zeros((u,) + M.shape, dtype=np.uint64)
    rc = lib().oracle_split_alpha(_p(M, _u64p), M.size, alpha, u, _p(W, _u64p))
    if rc:
        raise RuntimeError("oracle_split_alpha failed (%d)" % rc)
    return W


def split_signed8(M: np.ndarray, p: int, u: int) -> np.ndarray:
    """INT8 words (balanced base-2^8 digits of the signed representative)."""
    M = _c(M, np.uint64)
    W = np.zeros((u,) + M.shape, dtype=np.int32)
    rc = lib().oracle_split_signed8(_p(M, _u64p), M.size, p, u, _p(W, _i32p))
    if rc:
        raise ValueError("oracle_split_signed8: u=%d too small for p=%d" % (u, p))
    return W


def split_signed(M: np.ndarray, p: int, u: int, bits: int) -> np.ndarray:
    """Balanced base-2^bits digits of the signed representative: u - 1 in
    [-2^(bits-1), 2^(bits-1) - 1], the top one in [-2^(bits-1), 2^(bits-1)]."""
    M = _c(M, np.uint64)
    W = np.zeros((u,) + M.shape, dtype=np.int32)
    rc = lib().oracle_split_signed_bits(_p(M, _u64p), M.size, p, u, bits, _p(W, _i32p))
    if rc:
        raise ValueError("oracle_split_signed_bits: u=%d too small for p=%d (bits %d)" % (u, p, bits))
    return W


def diag_sums(Aw: np.ndarray, Bw: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """S_s = sum_{i+j=s} A_i B_j (exact int64); Aw [u][m][k], Bw [v][k][n]."""
    Aw = _c(Aw, np.int32)
    Bw = _c(Bw, np.int32)
    u, m, k = Aw.shape
    v, k2, n = Bw.shape
    assert k == k2
    out = np.zeros((u + v - 1, m, n), dtype=np.int64)
    lib().oracle_diag_sums(m, n, k, u, v, _p(Aw, _i32p), _p(Bw, _i32p), _p(out, _i64p), nthreads)
    return out


def recombine_pow(S: np.ndarray, radix: int, p: int) -> np.ndarray:
    """sum_s radix^s S[s] mod p."""
    S = _c(S, np.int64)
    ns = S.shape[0]
    out = np.zeros(S.shape[1:], dtype=np.uint64)
    lib().oracle_recombine_pow(_p(S, _i64p), ns, out.size, radix, p, _p(out, _u64p))
    return out


def mod_vec(x: np.ndarray, p: int) -> np.ndarray:
    """x mod p for integer-valued doubles (the value Alg. 1 must return)."""
    x = _c(x, np.float64)
    out = np.zeros(x.shape, dtype=np.uint64)
    if lib().oracle_mod_vec(_p(x, _f64p), x.size, p, _p(out, _u64p)):
        raise ValueError("mod_vec: non-integer or out-of-range input")
    return out


def mulmod_vec(x: np.ndarray, y: np.ndarray, p: int) -> np.ndarray:
    """x y mod p (the value Alg. 2 must return)."""
    x = _c(x, np.uint64)
    y = _c(y, np.uint64)
    out = np.zeros(x.shape, dtype=np.uint64)
    lib().oracle_mulmod_vec(_p(x, _u64p), _p(y, _u64p), x.size, p, _p(out, _u64p))
    return out


def ceil_root(p: int, u: int) -> int:
    return int(lib().oracle_ceil_root(p, u))


def lam(p: int, u: int, v: int, t: int = 53) -> int:
    """Largest block size allowed by Prop. 3.3 ((1,1): Sec. 2.2); 0 if none."""
    return int(lib().oracle_lambda(p, u, v, t))


def digit_words(p: int, bits: int) -> int:
    """Fewest balanced base-2^bits digits (u - 1 in [-h, h - 1], the top one
    in [-h, h], h = 2^(bits-1)) that represent every signed representative
    in [-(p-1)/2, (p-1)/2]: with R = 2^bits and B = R^(u-1) the largest such
    value is h B + (h - 1) (B - 1) / (R - 1)."""
    R, h = 1 << bits, 1 << (bits - 1)
    u = 1
    while h * R ** (u - 1) + (h - 1) * (R ** (u - 1) - 1) // (R - 1) < (p - 1) // 2:
        u += 1
    return u


def int8_words(p: int) -> int:
    """Fewest base-2^8 digits that represent every signed representative in
    [-(p-1)/2, (p-1)/2] with u - 1 balanced digits in [-128, 127] and a top
    digit in [-128, 128]: with B = 256^(u-1) the largest such value is
    128 B + 127 (B - 1) / 255."""
    u = 1
    while 128 * 256 ** (u - 1) + 127 * (256 ** (u - 1) - 1) // 255 < (p - 1) // 2:
        u += 1
    return u


# ---- multimodular (CRT) comparison form, Sec. 5.2 ------------------------
# Plain big-integer definitions: the moduli, the signed residues each side is
# split into, and the Chinese-remainder reconstruction of an integer.

def crt_moduli(p: int, k: int) -> list:
    """Moduli of the CRT form: the largest primes below 256 (largest first),
    the fewest whose product M exceeds 2 k (p-1)^2.  Sec. 5.2 needs
    M > k (p-1)^2 for the integer product; the factor 2 keeps that product
    below M / 2, the margin the reconstruction's quotient estimate uses."""
    primes = [c for c in range(255, 2, -1) if all(c % d for d in range(2, int(c ** 0.5) + 1))]
    target = 2 * max(k, 1) * (p - 1) ** 2
    out, prod = [], 1
    for q in primes:
        if prod > target:
            break
        out.append(q)
        prod *= q
    if prod <= target:
        raise ValueError("not enough primes below 256 for p=%d, k=%d" % (p, k))
    return out


def crt_residues(M: np.ndarray, moduli) -> np.ndarray:
    """Signed residues of every entry modulo each m_i, in
    [-(m_i-1)/2, (m_i-1)/2]; shape (s,) + M.shape, int32."""
    M = _c(M, np.uint64)
    out = np.empty((len(moduli),) + M.shape, dtype=np.int32)
    for i, m in enumerate(moduli):
        r = (M % np.uint64(m)).astype(np.int64)
        out[i] = np.where(r > (m - 1) // 2, r - m, r)
    return out


def crt_reconstruct(residues, moduli) -> int:
    """The unique x in [0, M), M = prod(moduli), with x = residues[i] mod
    moduli[i] (pairwise coprime moduli; textbook formula with big integers)."""
    M = 1
    for m in moduli:
        M *= m
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += (int(r) % m) * Mi * pow(Mi, -1, m)
    return x % M
