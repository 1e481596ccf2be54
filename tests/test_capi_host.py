"""The C-ABI library without a GPU: it loads, exports every symbol that
include/mwmm.h declares, and its planner (pure host logic) agrees with the
oracle's block sizes and the paper's variant choices."""
import ctypes
import os

import numpy as np
import pytest

from paper_2601_07508_b300 import build, inputs

SWEEP = {b: inputs.largest_prime_below_pow2(b) for b in inputs.SWEEP_BITS}


@pytest.fixture(scope="module")
def M():
    build.build()
    from paper_2601_07508_b300 import mwmm
    mwmm.lib()
    return mwmm


def test_library_exports_every_declared_symbol(M):
    L = ctypes.CDLL(M.LIB_PATH)
    names = M.declared_symbols()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(M):
    assert M.mwmm_status_str(0) == "ok"
    assert "prime" in M.mwmm_status_str(2) or "p must" in M.mwmm_status_str(2)
    assert "sm_103a" in M.mwmm_version()


@pytest.mark.parametrize("b", inputs.SWEEP_BITS)
@pytest.mark.parametrize("uv", [(1, 1), (1, 2), (1, 3), (1, 4), (2, 2), (2, 3)])
def test_fp64_plan_block_size_matches_oracle(M, oracle, b, uv):
    p = SWEEP[b]
    u, v = uv
    lam = oracle.lam(p, u, v)
    if lam < 1:
        with pytest.raises(M.MwmmError) as e:
            M.mwmm_plan(64, 64, 64, p, u, v, "fp64")
        assert e.value.status == 3  # MWMM_ERR_BOUND
        return
    h = M.mwmm_plan(64, 64, 64, p, u, v, "fp64")
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["lambda_max"] == min(lam, 2 ** 63 - 1)
    assert d["lambda"] == d["lambda_max"]
    assert d["alpha"] == oracle.ceil_root(p, u) and d["beta"] == oracle.ceil_root(p, v)
    assert d["q"] == 1.0 / p


def test_fp64_bound_rule_of_the_sweep(M, oracle):
    """(1,1) where its block size is >= 1, else (1,2), else (2,2): the rule the
    bitsize sweep uses; it is reproduced here from the oracle's block sizes."""
    expect = {}
    for b, p in SWEEP.items():
        for uv in ((1, 1), (1, 2), (2, 2)):
            if oracle.lam(p, *uv) >= 1:
                expect[b] = uv
                break
    assert expect == {20: (1, 1), 23: (1, 1), 26: (1, 1), 32: (1, 2), 40: (2, 2), 48: (2, 2), 52: (2, 2)}


def test_fp64_auto_variant_follows_cost_model(M, oracle):
    # With k large the modelled cost u v (1 + 6 / lambda) decides; the paper's
    # Table 4 (GPU, square) picks (2,3) at 46-52 bits and (1,1) at small bitsizes.
    for b, want in ((20, (1, 1)), (52, (2, 3)), (40, (2, 2))):
        h = M.mwmm_plan(4096, 4096, 4096, SWEEP[b], 0, 0, "fp64")
        d = M.mwmm_plan_info(h)
        M.mwmm_plan_destroy(h)
        assert (d["u"], d["v"]) == want, (b, d["u"], d["v"])


@pytest.mark.parametrize("p", list(SWEEP.values()) + [5, 7, 257, (1 << 31) - 1])
@pytest.mark.parametrize("bits", [0, 8, 9])
def test_int8_plan_digits_match_oracle(M, oracle, p, bits):
    h = M.mwmm_plan(100, 300, 5000, p, 0, 0, "int8", tc_digit_bits=bits)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    want = bits or (9 if oracle.digit_words(p, 9) < oracle.digit_words(p, 8) else 8)
    u = oracle.digit_words(p, want)
    assert d["tc_digit_bits"] == want
    assert (d["u"], d["v"], d["alpha"], d["nsums"]) == (u, u, 2 ** want, 2 * u - 1)
    # INT32 sums hold kc * min(u, v) products of magnitude <= 2^(2 bits - 2)
    prod = 2 ** (2 * want - 2)
    assert d["kc"] % 64 == 0 and d["kc"] * min(u, u) * prod < 2 ** 31
    assert d["nkc"] == -(-5000 // d["kc"])
    assert d["tc_chunk"] == 2 ** 24 // prod  # FP32 chunk: 1024 (8-bit) or 256 (9-bit) products
    assert d["A_rows"] == 128 and d["B_rows"] == 512  # m = 100: one row tile


def test_int8_digit_width_choice_on_the_sweep(M, oracle):
    """9-bit digits where they save a digit (26 and 52 bits of the sweep),
    8-bit ones elsewhere; explicit words of one width are checked against it."""
    got = {}
    for b, p in SWEEP.items():
        h = M.mwmm_plan(64, 64, 64, p, 0, 0, "int8")
        d = M.mwmm_plan_info(h)
        M.mwmm_plan_destroy(h)
        got[b] = (d["tc_digit_bits"], d["u"])
    assert got == {20: (8, 3), 23: (8, 3), 26: (9, 3), 32: (8, 4), 40: (8, 5), 48: (8, 6), 52: (9, 6)}
    with pytest.raises(M.MwmmError) as e:  # 6 digits of 8 bits cannot hold a 52-bit residue
        M.mwmm_plan(64, 64, 64, SWEEP[52], 6, 6, "int8")
    assert e.value.status == 3
    h = M.mwmm_plan(64, 64, 64, SWEEP[52], 6, 6, "int8", tc_digit_bits=9)
    M.mwmm_plan_destroy(h)
    for bad in (7, 10, -1):
        with pytest.raises(M.MwmmError) as e:
            M.mwmm_plan(64, 64, 64, SWEEP[52], 0, 0, "int8", tc_digit_bits=bad)
        assert e.value.status == 1


def test_plan_errors(M):
    for p in (2, 4, 3, 1 << 52, (1 << 52) + 1, 1 << 60):
        with pytest.raises(M.MwmmError) as e:
            M.mwmm_plan(8, 8, 8, p)
        assert e.value.status == 2
    with pytest.raises(M.MwmmError) as e:
        M.mwmm_plan(-1, 8, 8, SWEEP[40])
    assert e.value.status == 1
    with pytest.raises(M.MwmmError) as e:  # (1,1) cannot handle 40-bit primes
        M.mwmm_plan(8, 8, 8, SWEEP[40], 1, 1, "fp64")
    assert e.value.status == 3
    with pytest.raises(M.MwmmError) as e:  # too few INT8 digits
        M.mwmm_plan(8, 8, 8, SWEEP[52], 3, 3, "int8")
    assert e.value.status == 3
    with pytest.raises(M.MwmmError) as e:  # lambda override beyond the bound
        M.mwmm_plan(8, 8, 8, SWEEP[48], 2, 2, "fp64", lam=32)
    assert e.value.status == 3


def test_workspace_layout_sizes(M):
    p = SWEEP[40]
    h = M.mwmm_plan(300, 200, 100, p, 2, 2, "fp64")
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    nkb = -(-100 // 16)
    assert d["nkb"] == nkb and d["A_rows"] == 320 and d["B_rows"] == 256
    assert d["B_off"] >= 2 * nkb * 320 * 128
    assert d["workspace_bytes"] >= d["B_off"] + 2 * nkb * 256 * 128
    h = M.mwmm_plan(0, 200, 100, p, 2, 2, "fp64")
    assert M.mwmm_workspace_size(h) == 0
    M.mwmm_plan_destroy(h)


@pytest.mark.parametrize("m,n,pair,want_pair,want_rows", [
    (100, 300, False, 0, 128),   # unfused: one-CTA kernel, 128-row tiles
    (700, 300, False, 0, 768),
    (129, 300, True, 1, 256),    # the pair kernel needs 256-row tiles
    (700, 20, True, 0, 768),     # narrow n (diagonal windows): one-CTA kernel only
    (100, 300, True, 0, 128),    # a single row tile cannot be shared by a pair
])
def test_int8_unfused_plan_tile_kernel_choice(M, m, n, pair, want_pair, want_rows):
    h = M.mwmm_plan(m, n, 1000, SWEEP[52], 0, 0, "int8", tc_pair=pair, tc_fused=1)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["tc_fused"] == 0 and d["tc_pair"] == want_pair and d["A_rows"] == want_rows
    assert d["workspace_bytes"] >= d["S_off"] + d["nsums"] * d["nkc"] * d["A_rows"] * d["B_rows"] * 4


@pytest.mark.parametrize("m,n,k,b,form,want", [
    (4096, 4096, 4096, 20, "int8", 1),   # 8-bit digits, 16 x 16 x 5 = 1280 pair items
    (4096, 4096, 4096, 48, "int8", 1),
    (2048, 2048, 2048, 20, "int8", 1),   # 8 x 8 x 5 = 320 items
    (4096, 4096, 4096, 26, "int8", 0),   # 9-bit digits: one CTA per tile
    (4096, 4096, 4096, 52, "int8", 0),
    (1024, 1024, 4096, 20, "int8", 0),   # 4 x 4 x 5 = 80 items: too few waves of pairs
    (1100, 4096, 4096, 20, "int8", 0),   # 1280 rows instead of 1152: 11% padding
    (4000, 4096, 4096, 40, "int8", 1),   # 4096 rows either way
    (900, 8192, 4096, 20, "int8", 0),    # m < 1024
    (4096, 100, 4096, 20, "int8", 0),    # narrow n: diagonal windows, one-CTA kernel
    (4096, 4096, 4096, 40, "crt8", 1),   # CRT residues: 1024-product chunks, as 8-bit digits
    (4096, 4096, 512, 52, "crt8", 1),
    (1024, 1024, 4096, 52, "crt8", 0),   # 4 x 4 x 16 = 256 items
])
def test_default_tile_kernel_choice(M, m, n, k, b, form, want):
    """tc_pair = 0 (None in Python): the two-CTA kernel for 8-bit digits and
    CRT residues on large products (m >= 1024, at most 3% more padded rows,
    >= 296 items of 256 x 256), else one CTA per tile; True / False force
    either kernel."""
    p = SWEEP[b] if b in SWEEP else inputs.largest_prime_below_pow2(b)
    d = M.Plan(m, n, k, p, form=form).info
    assert d["tc_pair"] == want
    assert d["A_rows"] % (256 if want else 128) == 0
    assert M.Plan(m, n, k, p, form=form, tc_pair=False).info["tc_pair"] == 0
    if n > 128:
        assert M.Plan(m, n, k, p, form=form, tc_pair=True).info["tc_pair"] == 1


def test_tile_kernel_option_range(M):
    p = SWEEP[20]
    for bad in (2, -2):
        with pytest.raises(M.MwmmError):
            M.mwmm_plan(4096, 4096, 4096, p, 0, 0, "int8", tc_pair=bad)


@pytest.mark.parametrize("m,n,opt,want", [
    (700, 300, 0, 0), (700, 300, 1, 0),   # default and 1: diagonal sums in the workspace
    (700, 300, 2, 1), (129, 129, 2, 1),   # 2: fused whenever n > 128
    (100, 300, 2, 1), (1, 129, 2, 1),
    (700, 128, 2, 0),                     # narrow n (diagonal windows): unfused
])
def test_int8_fused_plan_choice_and_layout(M, m, n, opt, want):
    h = M.mwmm_plan(m, n, 1000, SWEEP[52], 0, 0, "int8", tc_fused=opt, tc_pair=True)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["tc_fused"] == want
    if not want:
        return
    # 256 x 128 tiles on CTA pairs; INT32 sums over one segment; no sums in the workspace
    assert d["tc_pair"] == 0 and d["A_rows"] == -(-m // 256) * 256 and d["B_rows"] == -(-n // 128) * 128
    assert d["tc_seg"] == 16 and d["kc"] == 1024 and d["nkc"] == 1  # k = 1000: one segment of 16 k-blocks
    assert d["kc"] * d["u"] * 2 ** 14 < 2 ** 31
    parts = d["ksplit"]
    assert d["workspace_bytes"] == (d["S_off"] + (parts * m * (n + n % 2) * 8 if parts > 1 else 0) + 255) // 256 * 256


@pytest.mark.parametrize("m,n,k,want", [
    (4096, 4096, 4096, 1),   # 16 x 32 = 512 tiles: 6.9 waves of 74 pairs, no parts
    (512, 512, 4096, 8),     # 8 tiles: the most parts (8) give 64 units
    (2048, 2048, 4096, 4),   # 128 tiles: 1-3 parts fill 86% of the last wave, 4 parts (512 units) 99%
    (2048, 2048, 64, 1),     # one k-block: one part
])
def test_int8_fused_plan_k_parts(M, m, n, k, want):
    h = M.mwmm_plan(m, n, k, SWEEP[40], 0, 0, "int8", tc_fused=2)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    tiles = (d["A_rows"] // 256) * (d["B_rows"] // 128)
    units = tiles * d["ksplit"]
    assert d["tc_fused"] == 1 and d["ksplit"] == want, (tiles, d["ksplit"])
    # the fewest parts whose units fill >= 90% of the last wave, else the best filling
    eff = units / (-(-units // 74) * 74)
    assert eff >= 0.9 or d["ksplit"] == min(8, d["nkb"])


def test_int8_fused_plan_options(M):
    p = SWEEP[52]
    h = M.mwmm_plan(700, 300, 5000, p, 0, 0, "int8", tc_fused=2, tc_seg=3, ksplit=5)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["tc_seg"] == 3 and d["kc"] == 192 and d["nkc"] == -(-5000 // 192) and d["ksplit"] == 5
    h = M.mwmm_plan(700, 300, 50000, p, 0, 0, "int8", tc_fused=2)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["tc_seg"] == 64 and d["kc"] * d["u"] * 2 ** 14 < 2 ** 31  # default segment: 64 k-blocks
    for kw in ({"tc_fused": 3}, {"tc_fused": -1}, {"tc_seg": -1}, {"tc_seg": 1 << 20}, {"ksplit": 65}):
        with pytest.raises(M.MwmmError) as e:
            M.mwmm_plan(700, 300, 5000, p, 0, 0, "int8", **dict({"tc_fused": 2}, **kw))
        assert e.value.status == 1, kw


@pytest.mark.parametrize("n,v,opt,want,slots", [
    (32, 2, 0, 1, 2), (20, 3, 0, 1, 4), (63, 4, 0, 1, 4), (64, 2, 0, 0, 1),   # auto: narrow n, 2 <= v <= 4
    (32, 1, 0, 0, 1), (32, 2, 1, 0, 1), (200, 2, 2, 1, 2),
])
def test_fp64_plan_concatenation(M, n, v, opt, want, slots):
    p = {1: SWEEP[20], 2: SWEEP[32], 3: SWEEP[32], 4: SWEEP[40]}[v]  # bitsizes each (1, v) handles
    h = M.mwmm_plan(1000, n, 4096, p, 1, v, "fp64", f64_concat=opt)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["f64_concat"] == want
    w = 64 // slots
    assert d["B_rows"] == -(-n // w) * w
    assert d["workspace_bytes"] >= d["B_off"] + v * d["nkb"] * d["B_rows"] * 128


@pytest.mark.parametrize("m,n,u,v,opt,want", [
    (20, 3000, 2, 2, 0, 2),    # m is the narrow side: A's words
    (20, 3000, 2, 3, 0, 2),
    (3000, 20, 2, 3, 0, 1),    # n is: B's words
    (20, 30, 2, 2, 0, 2),      # both narrow: the smaller outer dimension, m
    (20, 3000, 1, 2, 0, 0),    # one A word: nothing to concatenate on the narrow side
    (500, 500, 2, 2, 3, 2),    # forced
])
def test_fp64_plan_concatenation_side(M, m, n, u, v, opt, want):
    h = M.mwmm_plan(m, n, 1000, SWEEP[32] if u == 1 else SWEEP[40], u, v, "fp64", f64_concat=opt)
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["f64_concat"] == want
    if want == 2:
        w = 64 // (2 if u == 2 else 4)
        assert d["A_rows"] == -(-m // w) * w
        assert d["B_off"] >= u * d["nkb"] * d["A_rows"] * 128


def test_fp64_plan_concatenation_errors(M):
    for v, p in ((1, SWEEP[20]), (5, SWEEP[20])):
        with pytest.raises(M.MwmmError) as e:
            M.mwmm_plan(100, 20, 100, p, 1, v, "fp64", f64_concat=2)
        assert e.value.status == 1
    with pytest.raises(M.MwmmError) as e:  # A concatenation needs 2 <= u <= 4
        M.mwmm_plan(100, 20, 100, SWEEP[32], 1, 2, "fp64", f64_concat=3)
    assert e.value.status == 1
    with pytest.raises(M.MwmmError) as e:
        M.mwmm_plan(100, 20, 100, SWEEP[32], 1, 2, "fp64", f64_concat=4)
    assert e.value.status == 1


@pytest.mark.parametrize("m,n,k,want", [
    (4096, 4096, 4096, 1),     # 4096 tiles: the last wave is already 99% full
    (10923, 32, 32768, 5),     # 171 tiles (concatenated (1,2)): 5 ranges fill 96% of 3 waves
    (8192, 64, 8192, 9),       # 128 tiles: 9 ranges
    (64, 64, 64, 1),           # 4 k-blocks: ranges of at least 8 k-blocks
])
def test_fp64_plan_k_ranges(M, m, n, k, want):
    h = M.mwmm_plan(m, n, k, SWEEP[32], 1, 2, "fp64")
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    assert d["ksplit"] == want
    if want > 1:
        assert d["workspace_bytes"] >= d["S_off"] + want * m * n * 8
    with pytest.raises(M.MwmmError):
        M.mwmm_plan(m, n, k, SWEEP[32], 1, 2, "fp64", ksplit=65)


def test_selftest_wait_rejects_limits_out_of_range(M):
    """Argument checks happen before any device call (runs without a GPU)."""
    for cycles in (0, -5, (1 << 34) + 1):
        assert M.mwmm_selftest_wait_timeout(cycles, stream=0) == 1  # 0: the legacy default stream


def test_autotune_cache_file_round_trip(M, tmp_path):
    """The autotuner's cache is host state: JSON lines load, count, save and
    clear without a GPU."""
    M.mwmm_autotune_cache_clear()
    assert M.mwmm_autotune_cache_entries() == 0
    src = tmp_path / "cache.jsonl"
    src.write_text(
        '{"key": "f2.b52.m12.n12.k12.single.sm148", "form": 2, "u": 7, "v": 7, "tc_chunk": 0, "kc": 0, '
        '"tc_pair": 0, "tc_digit_bits": 9, "f64_concat": 0, "ksplit": 0, "ms": 4.250000, "tried": 3}\n'
        '{"key": "f1.b40.m11.n11.k11.batch.sm148", "form": 1, "u": 2, "v": 2, "tc_chunk": 0, "kc": 0, '
        '"tc_pair": 0, "tc_digit_bits": 0, "f64_concat": 1, "ksplit": 1, "ms": 59.400000, "tried": 4}\n'
        'not a cache line\n')
    M.mwmm_autotune_cache_load(str(src))
    assert M.mwmm_autotune_cache_entries() == 2
    out = tmp_path / "saved.jsonl"
    M.mwmm_autotune_cache_save(str(out))
    lines = out.read_text().splitlines()
    assert len(lines) == 2 and all(l.startswith('{"key": "f') for l in lines)
    assert '"u": 2, "v": 2' in lines[0] and '"ksplit": 1' in lines[0]  # keys sorted: f1... before f2...
    M.mwmm_autotune_cache_clear()
    M.mwmm_autotune_cache_load(str(out))
    assert M.mwmm_autotune_cache_entries() == 2
    M.mwmm_autotune_cache_clear()
    with pytest.raises(M.MwmmError):
        M.mwmm_autotune_cache_load(str(tmp_path / "missing.jsonl"))


def test_autotuned_plan_rejects_bad_arguments_before_any_device_call(M):
    for args in ((-1, 8, 8, SWEEP[40]), (8, 8, 8, 4), (8, 8, 8, 1 << 52)):
        with pytest.raises(M.MwmmError):
            M.mwmm_plan_autotuned(*args, form="fp64", stream=0)


@pytest.mark.parametrize("b", [20, 26, 32, 40, 48, 52])
@pytest.mark.parametrize("k", [1, 100, 4096, 40000])
def test_crt_plan_moduli_match_oracle(M, oracle, b, k):
    p = SWEEP[b]
    h = M.mwmm_plan(300, 200, k, p, 0, 0, "crt8")
    d = M.mwmm_plan_info(h)
    M.mwmm_plan_destroy(h)
    ms = oracle.crt_moduli(p, k)
    assert d["form"] == 3 and d["u"] == d["v"] == d["nsums"] == len(ms)
    assert d["crt_m"][:len(ms)] == ms and all(x == 0 for x in d["crt_m"][len(ms):])
    assert d["kc"] * 2 ** 14 < 2 ** 31  # one residue product per INT32 sum
    assert d["workspace_bytes"] >= d["S_off"] + len(ms) * d["nkc"] * d["A_rows"] * d["B_rows"] * 4


def test_crt_plan_errors(M):
    with pytest.raises(M.MwmmError) as e:  # words are fixed by the moduli
        M.mwmm_plan(8, 8, 8, SWEEP[40], 2, 2, "crt8")
    assert e.value.status == 1
    with pytest.raises(M.MwmmError) as e:  # 2 k (p-1)^2 beyond what 24 moduli below 256 cover
        M.mwmm_plan(8, 8, 1 << 23, SWEEP[52], 0, 0, "crt8")
    assert e.value.status == 1


@pytest.mark.parametrize("form", ["int8", "crt8"])
def test_underfill_k_split_plans(M, form):
    """tc_fill = 0 (default) shortens the K ranges of a product whose longest
    item (a diagonal's pairs over all of K) exceeds an SM's share of the work;
    large products, explicit kc, tc_fill = 1 and the fused form keep the
    INT32-bound K range."""
    p = SWEEP[26]
    small = M.Plan(256, 256, 4096, p, form=form).info
    assert small["nkc"] > 1 and small["kc"] % 64 == 0 and small["nkc"] == -(-4096 // small["kc"])
    assert M.Plan(256, 256, 4096, p, form=form, tc_fill=1).info["nkc"] == 1
    assert M.Plan(256, 256, 4096, p, form=form, kc=4096).info["nkc"] == 1
    assert M.Plan(4096, 4096, 4096, p, form=form).info["nkc"] == 1
    if form == "int8":
        assert M.Plan(256, 256, 4096, p, form=form, tc_fused=2).info["tc_fused"] == 1
    with pytest.raises(M.MwmmError):
        M.Plan(256, 256, 4096, p, form=form, tc_fill=2)


def test_certified_chunk_plans(M):
    """9-bit digits on 256-wide column tiles get certified 512-product chunks
    (tc_cert_chunk) and a squared-digit region after the item counter; 8-bit
    digits, narrow n, an explicit tc_chunk and the fused form keep the
    worst-case chunk only; the pair kernel certifies too."""
    p26, p20 = SWEEP[26], SWEEP[20]
    d = M.Plan(300, 700, 1000, p26, form="int8").info
    assert d["tc_digit_bits"] == 9 and d["tc_chunk"] == 256 and d["tc_cert_chunk"] == 512
    sums = d["nsums"] * d["nkc"] * d["A_rows"] * d["B_rows"] * 4
    t = (d["S_off"] + sums + 255) // 256 * 256
    sqa = d["u"] * d["nkb"] * (d["A_rows"] // 64) * 4
    sqb = d["v"] * d["nkb"] * (d["B_rows"] // 64) * 4
    assert d["workspace_bytes"] == (t + 256 + (sqa + 255) // 256 * 256 + sqb + 255) // 256 * 256
    assert M.Plan(300, 700, 1000, p20, form="int8").info["tc_cert_chunk"] == 0
    assert M.Plan(300, 100, 1000, p26, form="int8").info["tc_cert_chunk"] == 0
    assert M.Plan(300, 700, 1000, p26, form="int8", tc_chunk=128).info["tc_cert_chunk"] == 0
    dp = M.Plan(300, 700, 1000, p26, form="int8", tc_pair=True).info
    assert dp["tc_pair"] == 1 and dp["tc_cert_chunk"] == 512
    assert M.Plan(300, 700, 1000, p26, form="int8", tc_fused=2).info["tc_cert_chunk"] == 0
    assert M.Plan(300, 700, 1000, p26, form="crt8").info["tc_cert_chunk"] == 0


def test_tensor_form_choice_follows_the_cost_model(M):
    """AUTO's tensor form for batches and serving: at 4096^3 the digit form
    at 23-27 bits (9 digit products, 9-bit digits from 25 bits, against 8-9
    moduli plus a costlier CRT reconstruction), the CRT form from 28 bits
    (16 / 25 / 36 / 36 digit products against 10-16 moduli); small products
    stay INT8 (the CRT split and reconstruction grow with the moduli);
    k > 2^22 cannot use CRT."""
    P = {b: inputs.largest_prime_below_pow2(b) for b in (23, 24, 26, 27, 28, 32, 40, 48, 52)}
    for b in (23, 24, 26, 27):
        assert M.mwmm_tensor_form(4096, 4096, 4096, P[b]) == "int8", b
    for b in (28, 32, 40, 48, 52):
        assert M.mwmm_tensor_form(4096, 4096, 4096, P[b]) == "crt8", b
        assert M.mwmm_tensor_form(64, 64, 64, P[b]) == "int8", b
    assert M.mwmm_tensor_form(64, 64, (1 << 22) + 64, P[52]) == "int8"
    assert M.mwmm_tensor_form(4, 4, 4, 4) == "auto"  # no form plans an even p


def test_noalloc_wrapper_rejects_mismatched_operands_before_any_launch(M):
    """mwmm_matmul_noalloc's C entry point sees only pointers and sizes, so
    its binding checks the shapes and the device first: a B with the wrong
    number of rows, a C of the wrong shape, or operands off the GPU raise
    ValueError without reaching the library (no kernel could then read or
    write outside the tensors)."""
    torch = pytest.importorskip("torch")
    p = SWEEP[40]
    A = torch.zeros((8, 6), dtype=torch.int64)
    with pytest.raises(ValueError, match="rows"):
        M.mwmm_matmul_noalloc(A, torch.zeros((5, 4), dtype=torch.int64), torch.zeros((8, 4), dtype=torch.int64), p)
    with pytest.raises(ValueError, match="product is 8 x 4"):
        M.mwmm_matmul_noalloc(A, torch.zeros((6, 4), dtype=torch.int64), torch.zeros((4, 8), dtype=torch.int64), p)
    with pytest.raises(ValueError, match="2-D"):
        M.mwmm_matmul_noalloc(A, torch.zeros(6, dtype=torch.int64), torch.zeros((8, 4), dtype=torch.int64), p)
    with pytest.raises(ValueError, match="CUDA device"):
        M.mwmm_matmul_noalloc(A, torch.zeros((6, 4), dtype=torch.int64), torch.zeros((8, 4), dtype=torch.int64), p)


def test_bindings_reject_operands_that_do_not_match_the_product(M):
    """Every binding that hands matrices to the C ABI passes only pointers and
    leading dimensions, so it checks the operands' shapes against the plan's
    m x k, k x n and m x n (and, for device calls, that they share a device)
    first: a smaller matrix would otherwise be read or written past its end
    by the kernels.  The checks raise ValueError before any library call."""
    torch = pytest.importorskip("torch")
    p = SWEEP[40]
    plan = M.Plan(8, 4, 6, p, form="int8")
    z = lambda *s: torch.zeros(s, dtype=torch.int64)  # noqa: E731
    with pytest.raises(ValueError, match="A is"):
        M.mwmm_matmul(plan.handle, z(8, 5), z(6, 4), z(8, 4))
    with pytest.raises(ValueError, match="B is"):
        plan.matmul(z(8, 6), z(5, 4), z(8, 4))
    with pytest.raises(ValueError, match="C is"):
        plan.matmul(z(8, 6), z(6, 4), z(4, 8))
    with pytest.raises(ValueError, match="C is"):
        plan.matmul_reuse_a(z(6, 4), z(8, 3))
    with pytest.raises(ValueError, match="B is"):
        M.mwmm_matmul_host(plan.handle, np.zeros((8, 6), np.uint64), np.zeros((6, 3), np.uint64),
                           np.zeros((8, 4), np.uint64))
    with pytest.raises(ValueError, match="C is"):
        M.mwmm_matmul_host(plan.handle, np.zeros((8, 6), np.uint64), np.zeros((6, 4), np.uint64),
                           np.zeros((8, 3), np.uint64))
    with pytest.raises(ValueError, match="A is"):
        M.mwmm_split(plan.handle, 0, z(8, 7), torch.zeros(1 << 20, dtype=torch.uint8))
    with pytest.raises(ValueError, match="words holds"):
        M.mwmm_split(plan.handle, 1, z(6, 4), torch.zeros(16, dtype=torch.uint8))
    # batches and the serving loop take each problem's m, k from A and n from B
    with pytest.raises(ValueError, match="B of problem 1"):
        M._problems([(z(8, 6), z(6, 4), z(8, 4), p), (z(8, 6), z(7, 4), z(8, 4), p)])
    with pytest.raises(ValueError, match="C of problem 0"):
        M._problems([(z(8, 6), z(6, 4), z(8, 5), p)])


def test_binding_shape_check_edge_cases(M):
    """Empty products: a plan with k = 0 reads no A or B entries, so their k
    extent is free (a 1-column stand-in is accepted); C must still be m x n.
    m = 0 or n = 0 needs exactly empty operands on that side."""
    torch = pytest.importorskip("torch")
    z = lambda *s: torch.zeros(s, dtype=torch.int64)  # noqa: E731
    M._shape(z(7, 1), 7, 0, "A", 0)
    M._shape(z(1, 9), 0, 9, "B", 0)
    M._shape(z(7, 0), 7, 0, "A", 0)
    with pytest.raises(ValueError, match="C is"):
        M._shape(z(7, 1), 7, 0, "C")  # the k = 0 freedom is for A and B only
    with pytest.raises(ValueError, match="A is"):
        M._shape(z(6, 1), 7, 0, "A", 0)  # rows still count
    M._shape(z(0, 5), 0, 5, "A", 5)
    with pytest.raises(ValueError, match="A is"):
        M._shape(z(1, 5), 0, 5, "A", 5)
    with pytest.raises(ValueError, match="B is"):
        M._shape(z(5), 5, 1, "B", 5)  # not a matrix
    M._one_device(z(2, 2), None, z(2, 2))  # CPU tensors: one device, no current-device rule
