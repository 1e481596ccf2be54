// Internal declarations shared by the libmwmm translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "mwmm.h"

namespace mwmm {

constexpr int kMaxWords = 8;            // u, v <= 8 in the multiword forms
constexpr int kMaxCrt = 24;             // moduli of the CRT form (recombine.cu instantiates 1..24)
constexpr int kMaxWindows = 32;         // tcgen05 item groups (diagonal windows or moduli)
constexpr int kTileBytes = 128;         // one k-block row chunk of the word layout
// FP64 form tiling
constexpr int kF64KB = 16;              // doubles per k-block (128 B)
constexpr int kF64BM = 64;              // CTA rows
constexpr int kF64BN = 64;              // CTA cols
// INT8 (tcgen05) form tiling
constexpr int kTcKB = 64;               // bf16 digits per k-block (128 B)
constexpr int kTcBM = 128;              // MMA M (one CTA, TMEM lanes)
constexpr int kTcBN = 256;              // MMA N
constexpr int kTcMaxChunk = 1024;       // 2^24 / 2^14 digit products per FP32 chunk (8-bit digits)
constexpr int64_t kInt32SumLimit = 131071; // floor((2^31 - 1) / 2^14): products per INT32 sum (8-bit digits)
// Digits of b bits (magnitude <= 2^(b-1)) have products of magnitude <= 2^(2b-2):
// an FP32 chunk holds 2^(26 - 2b) of them, an INT32 sum floor((2^31 - 1) / 2^(2b-2)).
inline int64_t tc_chunk_limit(int bits) { return int64_t(1) << (26 - 2 * bits); }
inline int64_t int32_sum_limit(int bits) { return ((int64_t(1) << 31) - 1) >> (2 * bits - 2); }
constexpr int kFusedSeg = 64;           // fused form: default k-blocks per segment (4096 k)
constexpr int kFusedPairs = 74;         // fused form: CTA pairs the planner assumes (148 SMs)
constexpr int64_t kPairMinM = 1024;     // default two-CTA kernel: rows at least
constexpr int64_t kPairMinItems = 4 * 74;  // and at least four waves of 256 x 256 items

// One work item of the tcgen05 kernel: the word products of the diagonals
// s0 .. s0 + ndiag - 1 over k-blocks [kb0, kb0 + nkbc) for the 128-row tile mt
// and column tile nt of one problem.  Column block d (nb columns) of the
// 128 x (ndiag nb) accumulator holds diagonal s0 + d; A word i contributes to
// it through B word j = s0 + d - i when 0 <= j < v (the B words of a window
// are concatenated along N, Alg. 6's concatenation).  nb = 256 (ndiag = 1)
// when n > 128; otherwise nb is n padded to 16, 32, 64 or 128 and one item
// covers 256 / nb diagonals.
struct TcItem {
    const uint8_t *Aw, *Bw;  // word bases of the problem's A and B
    int32_t *S;              // S of diagonal s0, K-range kc, at the tile's origin (row stride B_rows)
    const uint32_t *sqA, *sqB;  // the problem's squared-digit maxima (certified chunks), or nullptr
    int64_t A_rows, B_rows, nkb, kb0, nkbc, mt, nt;
    int64_t plane;           // int32 elements between the S planes of consecutive diagonals
    int64_t b_wstride, b_kstride;  // bytes between consecutive B words / k-blocks
    int32_t s0, ndiag, nb, i0, ni, v, b_wpad;
    int32_t rv, cv;          // rows of the tile inside m, columns of each diagonal block inside n
    int32_t f16;             // 1: the words are fp16 (9-bit digits), 0: bf16
    int32_t chunk;           // k-block x pair steps per FP32 chunk (the problem's tc_chunk / 64)
};

struct Plan {
    int64_t m = 0, n = 0, k = 0;
    uint64_t p = 0;
    int form = 0;
    int u = 0, v = 0;
    uint64_t alpha = 0, beta = 0;
    int64_t lambda = 0, lambda_max = 0;
    double pd = 0, q = 0;
    int validate = 0;
    // FP64 form recombination constants, indexed i * v + j
    double gamma[kMaxWords * kMaxWords] = {};
    double gamma26[kMaxWords * kMaxWords] = {};  // gamma * 2^26 mod p
    int big_p = 0;                               // p > 2^52 / 3: split Alg. 2
    int f64_concat = 0;  // 1: B words concatenated along n, 2: A words along m (Alg. 6)
    int f64_vs = 1;      // word slots per 64-wide tile side (2 or 4 when concatenated)
    int f64_w = 64;      // output columns (B) or rows (A) per tile: 64 / f64_vs
    int ksplit = 1;      // K ranges of the FP64 kernel (partial results summed mod p)
    int64_t kbr = 0;     // k-blocks per K range
    // CRT form (MWMM_FORM_CRT8): moduli m_i, y_i = (M / m_i)^-1 mod m_i,
    // w_i = (M / m_i) mod p, W = M mod p
    int crt_s = 0;
    uint32_t crt_m[kMaxCrt] = {}, crt_y[kMaxCrt] = {};
    uint64_t crt_w[kMaxCrt] = {};
    uint64_t crt_W = 0;
    // autotuner outcome (0 when the plan was not tuned)
    double tuned_ms = 0;
    int tuned_tried = 0;
    // INT8 form
    int digit_bits = 8;  // 8: bf16-carried digits in [-128, 128]; 9: fp16-carried digits in [-256, 256]
    int64_t tc_chunk = 0, kc = 0;
    int tc_pair = 0;  // 1: 2-CTA kernel, A rows padded to 256 (the planner's choice or the caller's)
    // Fused recombination (gemm_tc_fused.cu): 256 x 128 tiles on CTA pairs,
    // A rows padded to 256 and B rows to 128; segments of tc_seg k-blocks;
    // K parts = ksplit (of kbr k-blocks), their residues in ksplit planes of
    // m x tc_ldr uint64 at S_off when ksplit > 1
    int tc_fused = 0;
    int tc_seg = 0;
    int64_t tc_ldr = 0;
    int tc_nb = 256;  // B rows per word slice of a tile (256, or n padded to 16/32/64/128)
    int tc_ndiag = 1; // diagonals per work item (256 / tc_nb, at most nsums)
    int nkc = 0, nsums = 0;
    // layout
    int64_t kb_elems = 0, nkb = 0, A_rows = 0, B_rows = 0;
    // B word layout: chunk(word w, k-block kb, row r) at
    // ((kb * B_kstride + (w + B_wpad) * B_wstride) + r) * 128; plain layout:
    // B_wstride = nkb * B_rows, B_kstride = B_rows, B_wpad = 0.  Narrow n
    // (diagonal windows): k-block major with B_wpad zero words on each side,
    // B_wstride = B_rows, B_kstride = (v + 2 B_wpad) * B_rows.
    int64_t B_wstride = 0, B_kstride = 0;
    int B_wpad = 0;
    // A word layout: chunk(word w, k-block kb, row r) at
    // (w A_wstride + kb A_kstride + r) * 128; k-block major (A_wstride =
    // A_rows, A_kstride = u A_rows) only for the FP64 form with A concatenated
    int64_t A_wstride = 0, A_kstride = 0;
    uint64_t A_off = 0, B_off = 0, S_off = 0, ws_bytes = 0;
    uint64_t sched_off = 0;  // tensor forms (unfused): the word-product kernel's item counter (256 bytes)
    // Certified chunks (INT8 form, 9-bit digits, one-CTA kernel, 256-wide
    // column tiles): the split writes, per word, k-block and group of 64
    // rows (A) or columns (B), the largest sum of squared digits over the
    // k-block (uint32, [word][k-block][group]) at sq_off (A) and
    // sq_off + sqB_off (B); the word-product kernel runs an item with FP32
    // chunks of tc_cert_chunk products when Cauchy-Schwarz on these sums
    // bounds every partial sum of each chunk by 2^24.  0: not used.
    int tc_cert_chunk = 0;
    uint64_t sq_off = 0, sqB_off = 0;
    // owned device resources (lazily created)
    int device = -1;
    void *own_ws = nullptr;
    uint64_t own_ws_bytes = 0;
    int *err_dev = nullptr;      // [0]: timeout, [1]: range violation
    uint64_t *hostbuf_dev = nullptr;  // A, B, C device copies for mwmm_matmul_host
    uint64_t hostbuf_bytes = 0;
};

// plan.cpp
mwmm_status make_plan(Plan *pl, int64_t m, int64_t n, int64_t k, uint64_t p, int u, int v,
                      int form, const mwmm_plan_opts *opts);
uint64_t ceil_root(uint64_t p, int u);
uint64_t block_size(uint64_t p, int u, int v);  // Prop. 3.3 / Sec. 2.2, 0 if none
int int8_digits(uint64_t p);
int signed_digits(uint64_t p, int bits);  // fewest balanced base-2^bits digits
uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t p);

// launches (return cudaError_t as int)
// sq: the plan's squared-digit maxima for this side (plan_sq), or nullptr
int launch_split(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words, void *stream,
                 uint32_t *sq = nullptr);
// The squared-digit maxima of a plan with certified chunks in workspace ws
// (side 0: A, 1: B), else nullptr.
inline uint32_t *plan_sq(const Plan &pl, uint8_t *ws, int side) {
    if (!pl.tc_cert_chunk) return nullptr;
    return reinterpret_cast<uint32_t *>(ws + pl.sq_off + (side ? pl.sqB_off : 0));
}
// part: ksplit x m x n partial results (workspace at S_off) when pl.ksplit > 1
int launch_gemm_fp64(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, uint64_t *part,
                     int *err, void *stream);
// sqA, sqB: the squared-digit maxima written by the splits (certified
// chunks), or nullptr (worst-case chunks only)
int launch_gemm_tc(const Plan &pl, const void *Aw, const void *Bw, int32_t *S, int *err, void *stream,
                   const uint32_t *sqA = nullptr, const uint32_t *sqB = nullptr);
int launch_recombine(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *stream);
// Fused form (pl.tc_fused): word products, reduction and recombination in one
// kernel, plus the K-part sum when pl.ksplit > 1 (R = workspace at S_off).
int launch_gemm_tc_fused(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, uint64_t *R,
                         int *err, void *stream);
int prepare_tc_fused_attributes();
// The word products and recombination of a tensor-form plan (fused or not),
// on the words in ws, writing C; one or two launches (three with K parts).
int launch_tensor_products(const Plan &pl, uint8_t *ws, uint64_t *C, int64_t ldc, int *err, void *stream);
// batched split: job records are opaque blobs of split_job_bytes() bytes
size_t split_job_bytes();
void split_job(const Plan &pl, int side, const uint64_t *M, int64_t ld, void *words, void *job, int job_index,
               std::vector<int> &blocks, uint32_t *sq = nullptr);
// sq: some job writes squared-digit maxima (SplitParams.sq set)
int launch_split_batched(const void *jobs, const int *blocks, int nblocks, int fp64, void *stream, int sq = 0);
size_t recombine_job_bytes();
void recombine_job(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *rec, int index,
                   std::vector<int> &jobs);
int launch_recombine_batched(const void *probs, const int *jobs, int njobs, void *stream);
size_t crt_job_bytes();
void crt_job(const Plan &pl, const int32_t *S, uint64_t *C, int64_t ldc, void *rec, int index, std::vector<int> &jobs);
int launch_crt_batched(const void *probs, const int *jobs, int njobs, void *stream);
size_t fp64_job_bytes();
void fp64_job(const Plan &pl, const void *Aw, const void *Bw, uint64_t *C, int64_t ldc, int *err, void *rec,
              int index, std::vector<int> &jobs);
int launch_gemm_fp64_batched(const void *probs, const int *jobs, int njobs, void *stream);
int prepare_kernel_attributes();  // dynamic shared-memory limits, once per device (call before capturing)
int tc_sm_count();
// SM count, resident CTAs of the one-CTA word-product kernel, co-resident
// clusters of the pair kernel on the current device (cudaError_t).
int tc_residency(int *sms, int *ctas, int *clusters);
// 1 when the pair kernel's co-resident clusters cover every SM of the
// current device, 0 when they do not, -1 when unknown (no device).
int tc_pairs_fill_device();
// Items claimed in table order from the counter at cta_off[2] (cleared by
// the launch): cta_off = {0, nitems, counter}.
// cert: some item carries squared-digit maxima (certified chunks)
int launch_gemm_tc_table(const TcItem *items, int64_t *cta_off, int64_t nitems, int ctas, int chunk_blocks, int *err,
                         void *stream, int cert = 0);
int launch_fmod(const double *x, int64_t count, uint64_t p, double *out, void *stream);
int launch_mulmod(const double *x, const double *y, int64_t count, uint64_t p, double *out, void *stream);
int launch_wait_probe(int64_t cycles, int *err, void *stream);

// autotune.cpp: the fastest configuration measured on the device (or cached)
// for this problem; batch = only configurations the batched kernels run.
mwmm_status autotune(int form_req, int64_t m, int64_t n, int64_t k, uint64_t p, const uint64_t *dA, int64_t lda,
                     const uint64_t *dB, int64_t ldb, bool batch, void *stream, int *form, int *u, int *v,
                     mwmm_plan_opts *opts, double *ms, int *tried);
// capi.cu
void describe_plan(const Plan &P, mwmm_plan_desc *d);

// Host-side tables of a batch of products (batch.cu).
struct BatchTables {
    std::vector<uint8_t> split_jobs;
    std::vector<int> split_blocks;
    std::vector<TcItem> items;
    std::vector<int64_t> cta_off;
    std::vector<uint8_t> rec_recs;
    std::vector<int> rec_jobs;
    std::vector<uint8_t> f64_recs;
    std::vector<int> f64_jobs;
    std::vector<uint8_t> crt_recs;
    std::vector<int> crt_jobs;
    int nsplit = 0, nrec = 0, nf64 = 0, ncrt = 0, ctas = 0;
    int cert = 0;  // some problem runs certified chunks: its splits write squared-digit maxima
};
constexpr int kBatchTables = 10;
// Tables for problems[0..count) whose workspaces start at ws_base[i] (device).
// Every plan is FP64, or every plan is INT8 or CRT8 (the two tensor forms
// share the word-product kernel and may mix).
void build_batch_tables(const Plan *plans, const mwmm_problem *probs, uint8_t *const *ws_base, int count,
                        int *err, BatchTables &T);
// One 256-byte-aligned blob holding the tables; off[i] = offset of table i.
uint64_t pack_batch_tables(const BatchTables &T, std::vector<uint8_t> &blob, uint64_t off[kBatchTables]);
// One product with the plan's own (computed-item) kernels on `stream`:
// split A and B, word products, recombination / reconstruction; ws is the
// plan's workspace.  k = 0 launches nothing (the caller zeroes C).
int launch_product(const Plan &pl, const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb, uint64_t *dC,
                   int64_t ldc, uint8_t *ws, void *stream);
// Work items a batch's tables would hold for this plan (tcgen05 items, or
// FP64 tiles).
int64_t batch_items(const Plan &pl);
// The same layout written into dst when it fits in capacity; returns the size either way.
uint64_t pack_batch_tables_to(const BatchTables &T, uint8_t *dst, uint64_t capacity, uint64_t off[kBatchTables]);
// Launch the batch's kernels with its tables at dtables (device copy of the blob).
int launch_batch_tables(const BatchTables &T, const uint8_t *dtables, const uint64_t off[kBatchTables], int fp64,
                        int chunk_blocks, int *err, void *stream);
// The tensor form (MWMM_FORM_INT8 or MWMM_FORM_CRT8) with the smaller
// modelled time for this product: word products at the tensor rate plus the
// split and recombination / reconstruction traffic (calibrated on 4096^3).
int choose_tensor_form(int64_t m, int64_t n, int64_t k, uint64_t p);

}  // namespace mwmm
