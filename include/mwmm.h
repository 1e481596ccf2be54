/*
 * mwmm.h -- C ABI of libmwmm: the multiword modular matrix product
 *           C = A B mod p for primes p < 2^52, on one B300 GPU (sm_103a).
 *
 * Method: Berthomieu, Graillat, Lesnoff, Mary, "Multiword matrix
 * multiplication over large finite fields in floating-point arithmetic".
 * A and B are split into words, A = sum_i alpha^i A_i and
 * B = sum_j beta^j B_j (Alg. 4), the u*v word products A_i B_j are
 * accumulated exactly in K-chunks that no partial sum can overflow
 * (Alg. 3, Prop. 2.3, Prop. 3.3), each chunk is reduced mod p (Alg. 1), and
 * the products are recombined with alpha^i beta^j mod p (Alg. 2, Alg. 5).
 *
 * Three forms compute the same, unique result (every output in [0, p)):
 *
 *   MWMM_FORM_FP64  the paper's method as stated: FP64 words from Alg. 4
 *                   with alpha = ceil(p^(1/u)), FP64 (DFMA) accumulation with
 *                   an Alg. 1 reduction every lambda k-steps (lambda from
 *                   Prop. 3.3, or Sec. 2.2 for (u,v) = (1,1)), and the
 *                   Alg. 2 scaling by gamma_ij = alpha^i beta^j mod p fused
 *                   into the epilogue (the workspace variant of Sec. 3.2).
 *
 *   MWMM_FORM_INT8  the narrower-word form of the paper's second
 *                   perspective (Sec. 6): words are base-2^8 digits of
 *                   magnitude <= 128 (balanced, the top one in [-128, 128])
 *                   of the signed representative of each
 *                   entry (so alpha = beta = 256), multiplied on the tcgen05
 *                   tensor pipe.  On sm_103a the tensor pipe has no INT8
 *                   kind, so the INT8 digits are carried exactly in bf16 and
 *                   accumulated in FP32 tensor memory, which is exact while
 *                   |partial sum| <= 2^24: a chunk holds at most 1024 digit
 *                   products (2^24 / 2^14).  Chunks are drained into exact
 *                   INT32 sums S_s = sum_{i+j=s} A_i B_j, K-chunked so that
 *                   |S_s| < 2^31, and C = sum_s 256^s S_s mod p is
 *                   recombined with exact 64-bit integer arithmetic.
 *
 *   MWMM_FORM_CRT8  the multimodular approach the paper compares against
 *                   (Sec. 5.2), run on the same tensor pipe: residues modulo
 *                   s primes below 256 instead of digits, one product per
 *                   modulus, and CRT reconstruction of the integer product.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major uint64 with a leading dimension (in elements)
 *     >= the row length.  A is m x k, B is k x n, C is m x n.
 *   - Entries of A and B must lie in [0, p) (the paper's inputs are in F_p);
 *     with plan option `validate` an entry >= p is reported as
 *     MWMM_ERR_RANGE, otherwise the result is unspecified.
 *   - C must not overlap A, B or the workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device-pointer calls are asynchronous on that stream; their
 *     device-side errors (range violation, expired bounded wait) are
 *     reported by mwmm_plan_check(), which synchronises the stream.
 *   - Every call returns a status; nothing exits, traps or prints.
 *   - A plan is not thread-safe: calls on one plan must be serialised and
 *     the plan's own workspace is shared by its calls on one stream.
 *   - A plan's device-side state is allocated on the device current at its
 *     first device call; a later call made with another device current
 *     returns MWMM_ERR_ARG.
 */
#ifndef MWMM_H
#define MWMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MWMM_OK = 0,
    MWMM_ERR_ARG = 1,         /* null pointer, bad size or leading dimension */
    MWMM_ERR_PRIME = 2,       /* p even, p < 5 or p >= 2^52 */
    MWMM_ERR_BOUND = 3,       /* no block size >= 1 for the requested (u,v) */
    MWMM_ERR_RANGE = 4,       /* an input entry >= p (validation on) */
    MWMM_ERR_NOMEM = 5,       /* device allocation failed */
    MWMM_ERR_BUDGET = 6,      /* request larger than the memory budget */
    MWMM_ERR_CUDA = 7,        /* a CUDA runtime call failed */
    MWMM_ERR_TIMEOUT = 8,     /* a bounded device-side wait expired */
    MWMM_ERR_BUSY = 9,        /* queue full / workspace too small */
    MWMM_ERR_UNSUPPORTED = 10 /* form not available on this device */
} mwmm_status;

typedef enum {
    MWMM_FORM_AUTO = 0, /* plans: the INT8 form (faster than FP64 on B300 at
                           every bitsize); batches and the serving loop: INT8
                           or CRT per problem, see mwmm_tensor_form */
    MWMM_FORM_FP64 = 1,
    MWMM_FORM_INT8 = 2,
    MWMM_FORM_CRT8 = 3  /* multimodular comparison form (Sec. 5.2): residues of A
                           and B modulo the s largest primes below 256 (s the
                           fewest whose product exceeds 2 k (p-1)^2), one
                           tcgen05 product per modulus (signed residues exact
                           in bf16, FP32 chunks of 1024, INT32 sums), and CRT
                           reconstruction of the integer product, reduced mod p.
                           u = v = nsums = s in the plan description. */
} mwmm_form;

typedef struct mwmm_plan_s *mwmm_plan_t;

/* Optional plan settings; pass NULL for defaults (all fields zero). */
typedef struct {
    int64_t lambda;   /* FP64 form: block size to use, 1..lambda_max (0: lambda_max) */
    int32_t validate; /* nonzero: check 0 <= entry < p on the device */
    int32_t tc_chunk; /* INT8 form: digit products per FP32 chunk, a multiple of
                         64 in [64, 1024] (0: 1024) */
    int64_t kc;       /* INT8 form: k-range of one INT32 sum, a multiple of 64
                         (0: the largest allowed by |S_s| < 2^31) */
    int32_t tc_pair;  /* INT8 and CRT forms, m > 128, n > 128: the tile kernel.
                         1 = the two-CTA tcgen05 kernel (256 x 256 tiles on an
                         SM pair, cta_group::2), -1 = the one-CTA kernel
                         (128 x 256 tiles), 0 = the planner's choice: two-CTA
                         for 8-bit digits and CRT residues when m >= 1024,
                         256-row tiles pad
                         m by at most 3%, there are at least 296 items and
                         (with a device present) the kernel's co-resident
                         clusters cover every SM (mwmm_tc_residency);
                         measured on B300: 3-4% faster there; else one-CTA.
                         Results are identical either way; other values:
                         MWMM_ERR_ARG */
    int32_t f64_concat; /* FP64 form, Alg. 6: 0 = automatic (when min(m, n) < 64,
                         concatenate the words of the narrower side: B's
                         along n when n <= m and 2 <= v <= 4, else A's along m
                         when 2 <= u <= 4), 1 = never, 2 = B's words
                         (needs 2 <= v <= 4), 3 = A's words (2 <= u <= 4) */
    int32_t ksplit;     /* FP64 form and INT8 fused form: K ranges computed by
                         separate CTAs (pairs) and added mod p afterwards,
                         1..64 (0: chosen so that the last wave is nearly
                         full) */
    int32_t autotune;   /* mwmm_batch_create / mwmm_matmul_batched only:
                         nonzero picks (u,v) and the K-range per bitsize
                         group by timing candidates (see mwmm_plan_autotuned) */
    int32_t tc_fused;   /* INT8 form: 2 = fuse the reduction and recombination
                         into the word-product kernel's epilogue when n > 128
                         (256 x 128 tiles on CTA pairs, residues in tensor
                         memory, no diagonal sums in memory: the workspace is
                         the words only, plus K-part planes when ksplit > 1);
                         0 (default) or 1 = diagonal sums to the workspace,
                         then the recombination kernel -- the faster form on
                         B300 (the fused tiles are half as wide) */
    int32_t tc_seg;     /* INT8 fused form: k-blocks of 64 per segment, the
                         k-range of one INT32 sum (0: 64, or fewer when the
                         INT32 bound requires) */
    int32_t tc_digit_bits; /* INT8 form, digit width: 8 = digits in [-128, 128]
                         carried in bf16 (FP32 chunks of <= 1024 products);
                         9 = digits in [-256, 256] carried in fp16 (chunks of
                         <= 256 products, INT32 sums of <= 32767 products);
                         0 = 9 when that needs fewer digits (u, v = 0 only),
                         else 8 */
    int32_t tc_fill;  /* INT8 and CRT forms with the diagonal sums in the
                         workspace and kc = 0: 0 (default) = when one K
                         range would leave the SMs under-filled (the longest
                         work item -- a tile's diagonal, up to min(u, v) word
                         pairs, over all of K -- longer than an SM's share of
                         the work), shorten the K ranges until it is not
                         (more INT32 sum planes, all added by the
                         recombination); 1 = never.  Batches, the serving
                         loop and mwmm_matmul_noalloc plan with 1: their
                         launches interleave many products */
} mwmm_plan_opts;

/* What a plan decided (mwmm_plan_info). */
typedef struct {
    int64_t m, n, k;
    uint64_t p;
    int32_t form;           /* MWMM_FORM_FP64 or MWMM_FORM_INT8 */
    int32_t u, v;           /* words of A and of B */
    uint64_t alpha, beta;   /* word radices: ceil(p^(1/u)), ceil(p^(1/v)); 256 for INT8 */
    int64_t lambda;         /* FP64: k-steps between Alg. 1 reductions */
    int64_t lambda_max;     /* FP64: largest block size allowed by Prop. 3.3 */
    int64_t tc_chunk;       /* INT8: digit products per FP32 tensor-memory chunk */
    int64_t kc;             /* INT8: k-range of one INT32 diagonal sum */
    int32_t tc_pair;        /* INT8: 1 when the two-CTA kernel computes the word products */
    int32_t nkc;            /* INT8: number of k-ranges, ceil(k / kc) */
    int32_t nsums;          /* INT8: number of diagonal sums u + v - 1 */
    double q;               /* fl(1/p) */
    /* Workspace layout (byte offsets into the workspace).
     * Words of side X (A: rows = m; B: rows = n, i.e. B is stored transposed,
     * K-contiguous) are stored as 128-byte row chunks:
     *   chunk(word w, k-block kb, row r) at X_off + ((w * nkb + kb) * X_rows + r) * 128
     * where nkb = ceil(k / kb_elems) and X_rows = A_rows or B_rows (padded).
     * INT8 form with n <= 128 only, for B: k-block major with B_wpad zero
     * words on each side,
     *   chunk(word w, k-block kb, row r) at
     *     B_off + ((kb * (v + 2 B_wpad) + w + B_wpad) * B_rows + r) * 128
     * (words -B_wpad .. -1 and v .. v + B_wpad - 1 are all zero).
     * FP64 form with f64_concat = 1, for B: k-block major without padding,
     *   chunk(word w, k-block kb, row r) at B_off + ((kb * v + w) * B_rows + r) * 128;
     * with f64_concat = 2 the same for A: A_off + ((kb * u + w) * A_rows + r) * 128.
     * Inside a chunk the 16-byte granule g (elements g*E .. g*E+E-1 of the
     * k-block, E = 16 / element size) is stored at granule position
     * g ^ (r mod 8).  Element type: double (FP64 form, kb_elems = 16) or
     * bf16 holding an integer digit (INT8 form, kb_elems = 64).  Padding is 0.
     * INT8 form: S (int32) at S_off, laid out [nsums][nkc][A_rows][B_rows];
     * unfused, then 256 bytes (the word-product kernel's item counter) at
     * T = S_off + the sums' bytes rounded up to 256; with tc_cert_chunk > 0,
     * the squared-digit maxima (uint32) at T + 256: A's laid out
     * [u][nkb][A_rows / 64], then, from T + 256 + (u nkb (A_rows / 64) 4
     * rounded up to 256), B's laid out [v][nkb][B_rows / 64] (for each 64-row
     * group, the largest sum over the k-block of a row's squared digits).
     * fused (tc_fused = 1): nothing at S_off unless ksplit > 1, then the K
     * parts' residues (uint64) laid out [ksplit][m][n rounded up to even].
     * FP64 form with ksplit > 1: the partial results of the K ranges
     * (uint64 residues) at S_off, laid out [ksplit][m][n]. */
    int64_t kb_elems, nkb, A_rows, B_rows;
    int32_t B_wpad;
    int32_t tc_fused;       /* INT8: 1 when the reduction and recombination run in the word-product
                               kernel's epilogue (then kc = 64 tc_seg is the k-range of one INT32 sum,
                               nkc = ceil(k / kc), and ksplit K parts each write a partial plane) */
    uint64_t A_off, B_off, S_off;
    uint64_t workspace_bytes;
    int32_t f64_concat;     /* FP64: 1 when B's words are concatenated along n, 2 when A's along m (Alg. 6) */
    int32_t ksplit;         /* FP64 and INT8 fused: K ranges (1: none) */
    double tuned_ms;        /* mwmm_plan_autotuned: measured time of the chosen configuration (0: not tuned) */
    int32_t tuned_tried;    /* candidates timed (0 when the choice came from the cache) */
    int32_t tc_seg;         /* INT8 fused: k-blocks per segment */
    uint32_t crt_m[24];     /* CRT form: the moduli m_0 > m_1 > ... (u of them); word i of A and of B
                               holds the signed residues modulo m_i, sum plane i their product */
    int32_t tc_digit_bits;  /* INT8: 8 (bf16 words) or 9 (fp16 words); alpha = beta = 2^tc_digit_bits */
    int32_t tc_cert_chunk;  /* INT8, 9-bit digits, 256-wide column tiles: the
                               FP32 chunk (512 products) an item runs when the
                               splits' sums of squared digits certify that no
                               partial sum can exceed 2^24 (Cauchy-Schwarz);
                               items that fail keep tc_chunk.  0: not used */
} mwmm_plan_desc;

/* Plan a product of an m x k by a k x n matrix mod p.
 * u = v = 0 picks the words automatically: FP64 form, the (u,v) of least
 * modelled cost u*v*(1 + 6/lambda) among (1,1),(1,2),(1,3),(1,4),(2,2),(2,3)
 * with lambda >= 1 (Sec. 3.3, Table 1); INT8 form, the fewest digits that
 * represent (p-1)/2; CRT form, the fewest moduli (u = v must be 0 there;
 * k <= 2^22).  MWMM_FORM_AUTO plans the INT8 form.  Explicit (u,v) are
 * validated (FP64: Prop. 3.3 must give lambda >= 1, else MWMM_ERR_BOUND;
 * INT8: u and v must be at least the fewest digits).  Pure host logic: makes no CUDA call and allocates no
 * device memory.  m, n, k >= 0; k may be 0 (C = 0).
 * Errors: MWMM_ERR_ARG, MWMM_ERR_PRIME, MWMM_ERR_BOUND. */
mwmm_status mwmm_plan(mwmm_plan_t *out, int64_t m, int64_t n, int64_t k, uint64_t p,
                      int u, int v, mwmm_form form, const mwmm_plan_opts *opts);

mwmm_status mwmm_plan_info(mwmm_plan_t plan, mwmm_plan_desc *out);

/* Autotuned plan (no counterpart in the paper's code; the paper picks (u,v)
 * from its cost model and measured crossovers, Sec. 3.3 and Table 4).
 * Times candidate configurations of this product on the current device and
 * returns a plan with the fastest: the form (when form = MWMM_FORM_AUTO:
 * FP64, INT8 or CRT; otherwise the given one), (u,v) among the FP64 variants whose block size
 * is >= 1 with concatenation on and off where it applies, the tcgen05 tile
 * variant (one CTA or CTA pairs) and the INT32 K-range.  Each
 * candidate runs once to warm up and twice timed (CUDA events on `stream`,
 * synchronised); candidates whose flop model exceeds 3x the best measured
 * time are skipped.  dA / dB (device, row-major, leading dimensions lda /
 * ldb) may be NULL: zero operands are used (run times do not depend on the
 * values).  Allocates scratch for C and one workspace for the call.
 * Results are cached per (form, bitsize of p, log2 buckets of m, n, k, SM
 * count); environment variable MWMM_AUTOTUNE_CACHE names a file that is read
 * at the first lookup and rewritten (one JSON object per line) after each
 * new entry.  mwmm_plan_info reports tuned_ms and tuned_tried.
 * Errors: those of mwmm_plan, MWMM_ERR_NOMEM, MWMM_ERR_CUDA. */
mwmm_status mwmm_plan_autotuned(mwmm_plan_t *out, int64_t m, int64_t n, int64_t k, uint64_t p,
                                mwmm_form form, const uint64_t *dA, int64_t lda, const uint64_t *dB,
                                int64_t ldb, void *stream);
/* The autotuner's cache: entries held in memory, clear, save to / load from
 * a file (JSON lines; load adds to the entries held). */
int64_t mwmm_autotune_cache_entries(void);
void mwmm_autotune_cache_clear(void);
mwmm_status mwmm_autotune_cache_save(const char *path);
mwmm_status mwmm_autotune_cache_load(const char *path);

/* Bytes of device workspace one mwmm_matmul call needs (0 for a NULL plan). */
size_t mwmm_workspace_size(mwmm_plan_t plan);

/* C = A B mod p with device pointers, asynchronously on `stream`.
 * workspace: device memory of at least mwmm_workspace_size(plan) bytes,
 * 256-byte aligned, owned by the caller; or NULL, in which case the plan
 * allocates its own on the first call and keeps it until destroyed.
 * Errors: MWMM_ERR_ARG, MWMM_ERR_NOMEM, MWMM_ERR_CUDA (launch failures). */
mwmm_status mwmm_matmul(mwmm_plan_t plan, const uint64_t *dA, int64_t lda,
                        const uint64_t *dB, int64_t ldb, uint64_t *dC, int64_t ldc,
                        void *workspace, size_t workspace_bytes, void *stream);

/* C = A B mod p reusing the words of A left in `workspace` by the most recent
 * mwmm_matmul (or mwmm_split of side 0 into workspace + A_off) with this
 * plan: only B is split.  For sequences of products with one fixed A, as in
 * the block-Wiedemann iterations of Sec. 4.1 where A's decomposition is
 * computed once.  A itself is not read; the caller keeps the workspace
 * (NULL: the plan's own) unchanged between the calls.
 * Errors: as mwmm_matmul. */
mwmm_status mwmm_matmul_reuse_a(mwmm_plan_t plan, const uint64_t *dB, int64_t ldb, uint64_t *dC, int64_t ldc,
                                void *workspace, size_t workspace_bytes, void *stream);

/* Same product with HOST matrices: copies A and B to plan-owned device
 * buffers, computes, copies C back and synchronises `stream`.  Device-side
 * errors are checked before returning.  When m >= 1024 (and per-phase timing
 * is off) the rows are processed in 2..8 blocks of at least 512 rows on
 * three plan-owned streams, so that copying the next block of A in and the
 * previous block of C out overlaps the current block's split, products and
 * recombination (the copies overlap only with page-locked host memory); the
 * plan then also owns a workspace for one block.  The work starts after
 * everything enqueued earlier on `stream`. */
mwmm_status mwmm_matmul_host(mwmm_plan_t plan, const uint64_t *hA, int64_t lda,
                             const uint64_t *hB, int64_t ldb, uint64_t *hC, int64_t ldc,
                             void *stream);

/* mwmm_matmul_host without the final synchronisation and error check: the
 * work is enqueued (ordered after earlier work on `stream`; `stream` is
 * ordered after its end) and the call returns.  hC is complete once `stream`
 * has been synchronised; mwmm_plan_check reports device-side errors.  Host
 * buffers must stay valid until then and must be page-locked for the copies
 * to be asynchronous.  Calls on different plans with different streams
 * overlap (copies of one product with the products of another); calls on one
 * plan must be ordered (the same stream, or synchronised between). */
mwmm_status mwmm_matmul_host_async(mwmm_plan_t plan, const uint64_t *hA, int64_t lda,
                                   const uint64_t *hB, int64_t ldb, uint64_t *hC, int64_t ldc,
                                   void *stream);

/* Synchronise `stream` and report device-side errors raised by this plan's
 * earlier calls (MWMM_ERR_RANGE, MWMM_ERR_TIMEOUT); clears them. */
mwmm_status mwmm_plan_check(mwmm_plan_t plan, void *stream);

void mwmm_plan_destroy(mwmm_plan_t plan);

/* The tensor form, MWMM_FORM_INT8 or MWMM_FORM_CRT8, that batches and the
 * serving loop use for this product under MWMM_FORM_AUTO: the smaller time
 * in the planner's cost model (word products at the tensor rate, plus the
 * split and the recombination or CRT reconstruction, calibrated on 4096^3
 * products on B300: at that size INT8 at 22-24 bits, CRT at 20-21 bits and
 * from 25 bits; small products INT8).  Host
 * only, no CUDA call.  MWMM_FORM_INT8 when the CRT form cannot be planned
 * (k > 2^22); MWMM_FORM_AUTO for arguments no form can plan. */
mwmm_form mwmm_tensor_form(int64_t m, int64_t n, int64_t k, uint64_t p);

/* ---- batched products (many independent problems, different shapes and primes) ----
 * A batch is planned once: every problem gets its own plan (FP64: (u,v) by
 * the cost model, lambda from Prop. 3.3; INT8: fewest digits; CRT: fewest
 * moduli), their words and sums share one device workspace owned by the
 * batch, the tcgen05 work items of all problems are spread over the SMs
 * (longest first, each to the least loaded SM), and the kernel launches are
 * captured once into a CUDA graph, whatever the count: 2 for the FP64 form;
 * for the tensor forms split, word products, then the INT8 recombination
 * and / or the CRT reconstruction (3 or 4).  INT8 and CRT problems may mix in
 * one batch (MWMM_FORM_AUTO); FP64 problems run in batches of their own.  The device
 * pointers of the problems are bound at creation: a run recomputes every C
 * from the current contents of its A and B.  The paper computes one product
 * at a time; its first perspective (Sec. 6) suggests batching. */
typedef struct {
    int64_t m, n, k;
    uint64_t p;               /* odd, 5 <= p < 2^52 */
    const uint64_t *A;        /* device, m x k, row-major, entries in [0, p) */
    int64_t lda;
    const uint64_t *B;        /* device, k x n */
    int64_t ldb;
    uint64_t *C;              /* device, m x n; must not overlap another problem's C */
    int64_t ldc;
} mwmm_problem;

typedef struct mwmm_batch_s *mwmm_batch_t;

typedef struct {
    int32_t count, form;
    int32_t ctas;             /* CTAs of the persistent tcgen05 launch (tensor forms) */
    int64_t items;            /* tcgen05 work items over all problems */
    int64_t launches;         /* kernel launches per run */
    uint64_t workspace_bytes, table_bytes;
    double flops_2mnk;        /* sum over problems of 2 m n k */
    double word_flops;        /* sum of 2 u v m n k (CRT: 2 s m n k), the word-product flops */
    int32_t tuned_groups;     /* opts.autotune: bitsize groups whose configuration was timed or cached */
    int32_t pad0;
    double tuned_ms;          /* sum over groups of the probe products' measured times */
} mwmm_batch_desc;

/* Plan and capture a batch (allocates the workspace and tables; makes CUDA
 * calls).  form: MWMM_FORM_FP64, MWMM_FORM_INT8 or MWMM_FORM_CRT8 for every
 * problem, or MWMM_FORM_AUTO for the tensor form of each problem (INT8 or
 * CRT, mwmm_tensor_form; per problem, since one bitsize can span a wide range
 * of sizes).  opts applies to every problem (lambda is ignored).  With
 * opts->autotune set, the problems are grouped by the bit length of p and
 * their form, and each group's (u,v), INT32 K-range and concatenation are
 * those mwmm_plan_autotuned picks in that form for the group's median-size
 * problem among the configurations the batched kernels run (one-CTA tcgen05
 * tiles, one FP64 K range); the choice is timed on zero operands of that
 * size, or taken from the autotuner's cache.  Errors: those
 * of mwmm_plan for any problem, MWMM_ERR_ARG, MWMM_ERR_NOMEM, MWMM_ERR_CUDA. */
mwmm_status mwmm_batch_create(mwmm_batch_t *out, const mwmm_problem *probs, int count, mwmm_form form,
                              const mwmm_plan_opts *opts);
/* Replay the captured graph on `stream` (asynchronous). */
mwmm_status mwmm_batch_run(mwmm_batch_t batch, void *stream);
/* Synchronise `stream`; report and clear device-side errors of the batch. */
mwmm_status mwmm_batch_check(mwmm_batch_t batch, void *stream);
mwmm_status mwmm_batch_info(mwmm_batch_t batch, mwmm_batch_desc *out);
/* The plan of problem `index` (words, block size, digits). */
mwmm_status mwmm_batch_problem_info(mwmm_batch_t batch, int index, mwmm_plan_desc *out);
void mwmm_batch_destroy(mwmm_batch_t batch);

/* One call for callers that keep a cache handle: creates (or re-creates, when
 * the problems differ from the cached ones) the batch in *cache and runs it.
 * cache == NULL: create, run, synchronise, destroy. */
mwmm_status mwmm_matmul_batched(const mwmm_problem *probs, int count, mwmm_form form, mwmm_batch_t *cache,
                                void *stream);

/* ---- serving: continuous batching of products as they arrive ----
 * A server owns a worker thread and a device-memory budget.  Clients submit
 * problems (device pointers; the operands stay on the device) from any
 * thread and get a ticket.  The worker forms a batch around the queued
 * request with the least work (or the oldest one, once it has waited several
 * times its estimated run time), adds queued requests of similar work in
 * arrival order as soon as their workspace fits in what is left of the
 * budget, and launches the batch on the next of max_inflight streams while
 * earlier batches still run.  Requests of at most 32 work items (output
 * tiles x word windows x K chunks) share the batched kernels of
 * mwmm_batch_create (without graph capture; at most 8192 items per batch);
 * larger ones run the single-product kernels of a plan on the same stream.
 * Finished batches return their memory and wake their waiters.  Latency = completion seen by the worker
 * minus arrival (submit time, or an earlier scheduled time the client gives).
 * The budget covers the per-request workspaces plus one 32 MiB table region
 * per stream; operands and outputs are the client's. */
typedef struct {
    int32_t max_batch;   /* requests per batch (0: 64) */
    int32_t form;        /* MWMM_FORM_AUTO: each request's tensor form (INT8 or
                            CRT, mwmm_tensor_form; a batch may mix them);
                            MWMM_FORM_INT8, MWMM_FORM_CRT8 or MWMM_FORM_FP64:
                            that form for every request */
    int32_t reserved[8];
} mwmm_serve_opts;

typedef struct {
    int64_t submitted, completed, rejected, batches;
    double mean_batch;             /* requests per launched batch */
    int64_t peak_queue, peak_inflight;
    uint64_t peak_bytes;           /* most workspace bytes in use at once */
    uint64_t budget_bytes;
    double flops_2mnk;             /* sum of 2 m n k over completed requests */
    double busy_s;                 /* first arrival to last completion */
    double gops;                   /* flops_2mnk / busy_s / 1e9 */
    double p50_ms, p99_ms, mean_ms, max_ms;
} mwmm_serve_report;

typedef struct mwmm_server_s *mwmm_server_t;

/* Errors: MWMM_ERR_BUDGET (budget below max_inflight x 32 MiB + 16 MiB),
 * MWMM_ERR_NOMEM, MWMM_ERR_CUDA. */
mwmm_status mwmm_serve_create(mwmm_server_t *out, size_t mem_budget_bytes, int max_inflight,
                              const mwmm_serve_opts *opts);
/* Seconds on the server's clock (0 at creation). */
double mwmm_serve_now(mwmm_server_t server);
/* Non-blocking.  t_arrival: scheduled arrival on the server clock, or < 0 for
 * "now".  Errors: those of mwmm_plan, MWMM_ERR_ARG, MWMM_ERR_BUDGET (the
 * request's workspace exceeds the whole budget; it is counted as rejected). */
mwmm_status mwmm_serve_submit(mwmm_server_t server, const mwmm_problem *prob, double t_arrival,
                              uint64_t *ticket);
/* MWMM_OK (or the request's error) once done, MWMM_ERR_BUSY while pending. */
mwmm_status mwmm_serve_poll(mwmm_server_t server, uint64_t ticket);
/* Block until done (timeout_ms < 0: no limit); MWMM_ERR_TIMEOUT on expiry. */
mwmm_status mwmm_serve_wait(mwmm_server_t server, uint64_t ticket, int timeout_ms);
/* Latency of a finished request in seconds. */
mwmm_status mwmm_serve_latency(mwmm_server_t server, uint64_t ticket, double *seconds);
mwmm_status mwmm_serve_stats(mwmm_server_t server, mwmm_serve_report *out);
/* Zero the counters and forget finished requests (their tickets). */
mwmm_status mwmm_serve_reset_stats(mwmm_server_t server);
/* Finish every submitted request, then release the server. */
void mwmm_serve_destroy(mwmm_server_t server);

/* The INT8-form product for callers that cannot allocate device memory
 * (their allocator belongs to another framework, or their device footprint
 * must stay fixed after start-up).  The paper has no counterpart: this is a
 * deployment variant of mwmm_matmul with default options.
 * The word matrices and diagonal sums live in a 64 MiB array that the
 * library reserves statically on each GPU where this code is loaded, held
 * until the process exits; the caller passes only A, B and C (device
 * pointers, same conventions as mwmm_matmul).  The first call on a device
 * looks up that array's address and caches it.
 * Every call shares the one array, so calls that overlap on the GPU race:
 * issue them one at a time per device.  Synchronous: returns once C is
 * written.  Calls no cudaMalloc/cudaFree or other allocating routine.
 * A product whose words and diagonal sums exceed the array runs the fused
 * form instead (tc_fused = 2 of mwmm_plan_opts, when n > 128: the sums stay
 * on the SM, so the scratch holds the words only).
 * Errors: MWMM_ERR_BUDGET when even the words exceed the array (about
 * m = n = k = 1500 at 52 bits; more for smaller primes), plus the errors of
 * mwmm_plan and mwmm_matmul, and MWMM_ERR_TIMEOUT. */
mwmm_status mwmm_matmul_noalloc(int64_t m, int64_t n, int64_t k, uint64_t p,
                                const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb,
                                uint64_t *dC, int64_t ldc, void *stream);

/* ---- step-level entry points (used to check single steps of the path) ---- */

/* Alg. 4 / INT8 digits: write the words of A (side 0, M is m x k) or of B
 * (side 1, M is k x n) into `words` using the plan's word layout (see
 * mwmm_plan_desc; `words` receives the X_off..X_off+size region only, i.e.
 * the first chunk lands at words + 0). */
mwmm_status mwmm_split(mwmm_plan_t plan, int side, const uint64_t *dM, int64_t ld,
                       void *words, void *stream);

/* Alg. 1 on the device: out[e] = x[e] mod p, for integer-valued doubles
 * 0 <= x[e] <= 2^51 p (Prop. 2.1), using q = fl(1/p).  5 <= p < 2^52. */
mwmm_status mwmm_fmod(const double *dx, int64_t count, uint64_t p, double *dout, void *stream);

/* Alg. 2 on the device: out[e] = x[e] y[e] mod p for integer-valued doubles
 * x, y in [0, p).  For p <= 2^52/3 this is Alg. 2 as printed (Prop. 2.2);
 * above, y is split as y_h 2^26 + y_l and two Alg. 2 calls are combined so
 * that each product stays within Prop. 2.2's bound. */
mwmm_status mwmm_mulmod(const double *dx, const double *dy, int64_t count, uint64_t p,
                        double *dout, void *stream);

/* Self-test of the bounded device waits (no counterpart in the paper).
 * Every wait of the product kernels on a shared-memory barrier gives up
 * after a fixed number of SM cycles (about two seconds), sets the plan's
 * error flag and lets the kernel return, so a stalled pipeline ends as
 * MWMM_ERR_TIMEOUT from mwmm_plan_check instead of a hung context.  This call
 * runs that same wait routine in a one-thread kernel on a barrier phase that
 * nothing completes, with a limit of `cycles` (1 .. 2^34), synchronises
 * `stream`, and returns MWMM_ERR_TIMEOUT when the wait gave up (the expected
 * outcome), MWMM_OK if it did not, MWMM_ERR_ARG for a limit out of range,
 * MWMM_ERR_NOMEM / MWMM_ERR_CUDA on a runtime failure.  It allocates and
 * frees a 4-byte flag; the device stays usable afterwards. */
mwmm_status mwmm_selftest_wait_timeout(int64_t cycles, void *stream);

/* Pipe-rate diagnostic (no counterpart in the paper): the FP64 fused
 * multiply-add rate of the current device, the roofline denominator of the
 * FP64 form.  Runs a kernel of sixteen independent DFMA chains per thread
 * (the FP64 word-product kernel's 4 x 4 accumulator block; one block of
 * 1024 threads per SM) for `iters` (1 .. 2^24) iterations after a short
 * warm-up, times it with CUDA events on `stream`, synchronises, and writes
 * 2 x 16 x iters x threads / time in GFLOP/s to *gflops.  Allocates nothing.
 * Errors: MWMM_ERR_ARG, MWMM_ERR_CUDA. */
mwmm_status mwmm_measure_fp64_rate(int64_t iters, double *gflops, void *stream);

/* Residency diagnostic (no counterpart in the paper): on the current device,
 * *sms = its SM count, *ctas = CTAs of the one-CTA word-product kernel that
 * can be resident at once (its persistent grid), *pair_clusters = clusters
 * of two CTAs of the pair kernel (tc_pair) that can be resident at once
 * (cudaOccupancyMaxActiveClusters: at most sms / 2, fewer where the device's
 * SMs do not all pair up).  Any pointer may be NULL.  Errors: MWMM_ERR_CUDA
 * (no device, or a query failed). */
mwmm_status mwmm_tc_residency(int32_t *sms, int32_t *ctas, int32_t *pair_clusters);

/* ---- per-phase timing (CUDA events on the call's stream) ----
 * When timing is on, every mwmm_matmul / mwmm_matmul_host call records events
 * around its phases: the split of A, the split of B (Alg. 4 or INT8 digits),
 * the word products (FP64 form: the fused kernel, which also reduces and
 * recombines; INT8 form: the tcgen05 kernel), and the recombination (INT8
 * form).  mwmm_plan_timing synchronises on the recorded events, returns the
 * times summed over the calls since the previous query, and resets them. */
typedef struct {
    double split_a_ms, split_b_ms, gemm_ms, recombine_ms, total_ms;
    int64_t calls;     /* products timed */
    int64_t launches;  /* kernels launched by those products */
} mwmm_timing;

mwmm_status mwmm_plan_set_timing(mwmm_plan_t plan, int on);
mwmm_status mwmm_plan_timing(mwmm_plan_t plan, mwmm_timing *out);

const char *mwmm_status_str(mwmm_status s);
const char *mwmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MWMM_H */
