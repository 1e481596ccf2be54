// Batched products: many independent C_i = A_i B_i mod p_i (different shapes
// and primes) run by one CUDA-graph replay of three table-driven kernels.
//
// The paper computes one product at a time; its first perspective (Sec. 6)
// suggests batching the block products.  Here a batch is planned once:
//   - each problem gets its own plan (words, lambda / digits, layout),
//   - all word matrices and diagonal sums share one device workspace,
//   - the split kernel walks a table of (problem, side, tile) blocks,
//   - INT8 and CRT forms (they may mix in one batch): the persistent tcgen05
//     kernel walks per-CTA lists of work items (tile, diagonal or modulus,
//     K-range) of all problems, assigned longest first to the least loaded
//     SM so every SM gets the same modelled work; the recombination kernel
//     (INT8 problems) and the CRT reconstruction kernel (CRT problems) walk
//     (problem, 8-row block) jobs,
//   - FP64 form: the fused kernel walks a table of (problem, 64 x 64 tile),
// and the launches are captured once into a CUDA graph; a run is one
// cudaGraphLaunch on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "mwmm_internal.h"

using mwmm::Plan;

struct mwmm_batch_s {
    int form = 0;
    std::vector<mwmm_problem> probs;
    std::vector<Plan> plans;
    uint8_t *ws = nullptr;        // words + sums of every problem
    uint8_t *tables = nullptr;    // kernel tables
    int *err = nullptr;           // error words
    uint64_t ws_bytes = 0, table_bytes = 0;
    int nsplit = 0, ntc_ctas = 0, nrec = 0, nf64 = 0;
    int cert = 0;  // some problem runs certified chunks
    int64_t nitems = 0;
    const void *d_split_jobs = nullptr;
    const int *d_split_blocks = nullptr;
    const mwmm::TcItem *d_items = nullptr;
    const int64_t *d_cta_off = nullptr;
    const void *d_rec = nullptr;
    const int *d_rec_jobs = nullptr;
    const void *d_f64 = nullptr;
    const int *d_f64_jobs = nullptr;
    const void *d_crt = nullptr;
    const int *d_crt_jobs = nullptr;
    int ncrt = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double flops_2mnk = 0, word_flops = 0;
    int64_t launches = 0;
    int tuned_groups = 0;
    double tuned_ms = 0;
    int chunk_blocks = mwmm::kTcMaxChunk / mwmm::kTcKB;
};

namespace mwmm {

// Claim order of the batch's items: the word-product kernel's CTAs take the
// items one by one from a counter in this order (list scheduling on the
// actual finish times).  Problems go largest first (by modelled cost), so the
// batch ends on the smallest; inside a problem the windows go heaviest first,
// every tile of a window in row order, so the ~148 items running at once
// mostly share one problem's word tiles in L2.  T.cta_off holds {0, N, 0}:
// the item range and the counter (zero; the launch clears it again).
static void claim_order(std::vector<mwmm::TcItem> &items, const std::vector<size_t> &prob_start,
                        std::vector<int64_t> &off) {
    const size_t P = prob_start.size();
    std::vector<int64_t> cost(P, 0);
    for (size_t p = 0; p < P; ++p) {
        const size_t e = p + 1 < P ? prob_start[p + 1] : items.size();
        for (size_t i = prob_start[p]; i < e; ++i) cost[p] += items[i].ni * items[i].nkbc + 2;  // +2: drain, store
    }
    std::vector<size_t> order(P);
    for (size_t p = 0; p < P; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    std::vector<mwmm::TcItem> out;
    out.reserve(items.size());
    for (size_t p : order) {
        const size_t e = p + 1 < P ? prob_start[p + 1] : items.size();
        out.insert(out.end(), items.begin() + (long)prob_start[p], items.begin() + (long)e);
    }
    items.swap(out);
    off.assign(3, 0);
    off[1] = (int64_t)items.size();
}

// Work items of one INT8- or CRT-form problem whose words start at Aw / Bw
// and whose sums start at S (see the plan layout and TcItem).  INT8: windows
// of tc_ndiag diagonals; CRT: one window per modulus i, the pair (i, i)
// (s0 = 2 i, so that B word s0 - i = i), its sums in plane i.
// Every item carries the problem's worst-case FP32 chunk (its digit width's:
// 9-bit digits 256 products, 8-bit digits and CRT residues 1024) and, for a
// plan with certified chunks, its squared-digit maxima (sqA, sqB).
static void tc_items(const Plan &pl, const uint8_t *Aw, const uint8_t *Bw, int32_t *S, std::vector<mwmm::TcItem> &items,
                     const uint32_t *sqA = nullptr, const uint32_t *sqB = nullptr) {
    const int64_t mtc = pl.A_rows / mwmm::kTcBM;
    const int64_t ntc = pl.tc_nb == mwmm::kTcBN ? pl.B_rows / mwmm::kTcBN : 1;
    const int64_t kcb = pl.kc / mwmm::kTcKB;
    const int64_t plane = (int64_t)pl.nkc * pl.A_rows * pl.B_rows;
    const bool crt = pl.form == MWMM_FORM_CRT8;
    const int nwin = crt ? pl.crt_s : (pl.nsums + pl.tc_ndiag - 1) / pl.tc_ndiag;
    // windows by decreasing number of word pairs (stable)
    std::vector<int> worder(nwin);
    std::vector<int> wni(nwin);
    for (int g = 0; g < nwin; ++g) {
        const int s0 = crt ? 2 * g : g * pl.tc_ndiag;
        const int nd = crt ? 1 : std::min(pl.tc_ndiag, pl.nsums - s0);
        wni[g] = crt ? 1 : std::min(s0 + nd - 1, pl.u - 1) - std::max(0, s0 - (pl.v - 1)) + 1;
        worder[g] = g;
    }
    std::stable_sort(worder.begin(), worder.end(), [&](int a, int b) { return wni[a] > wni[b]; });
    for (int g : worder) {
        const int s0 = crt ? 2 * g : g * pl.tc_ndiag;
        const int nd = crt ? 1 : std::min(pl.tc_ndiag, pl.nsums - s0);
        const int ilo = crt ? g : std::max(0, s0 - (pl.v - 1)), ihi = crt ? g : std::min(s0 + nd - 1, pl.u - 1);
        const int splane = crt ? g : s0;
        for (int kc = 0; kc < pl.nkc; ++kc)
            for (int64_t mt = 0; mt < mtc; ++mt)
                for (int64_t nt = 0; nt < ntc; ++nt) {
                    mwmm::TcItem it;
                    std::memset(&it, 0, sizeof(it));
                    it.Aw = Aw;
                    it.Bw = Bw;
                    it.S = S + (((int64_t)splane * pl.nkc + kc) * pl.A_rows + mt * mwmm::kTcBM) * pl.B_rows +
                           nt * mwmm::kTcBN;
                    it.A_rows = pl.A_rows;
                    it.B_rows = pl.B_rows;
                    it.nkb = pl.nkb;
                    it.kb0 = (int64_t)kc * kcb;
                    it.nkbc = std::min(kcb, pl.nkb - it.kb0);
                    it.mt = mt;
                    it.nt = nt;
                    it.plane = plane;
                    it.s0 = s0;
                    it.ndiag = nd;
                    it.nb = pl.tc_nb;
                    it.i0 = ilo;
                    it.ni = ihi - ilo + 1;
                    it.v = pl.v;
                    it.b_wpad = pl.B_wpad;
                    it.rv = (int32_t)std::min<int64_t>(mwmm::kTcBM, pl.m - mt * mwmm::kTcBM);
                    it.cv = (int32_t)std::min<int64_t>(pl.tc_nb, pl.n - nt * pl.tc_nb);
                    it.b_wstride = pl.B_wstride * mwmm::kTileBytes;
                    it.b_kstride = pl.B_kstride * mwmm::kTileBytes;
                    it.f16 = pl.form == MWMM_FORM_INT8 && pl.digit_bits == 9;
                    it.chunk = (int32_t)(pl.tc_chunk / mwmm::kTcKB);
                    it.sqA = nd == 1 ? sqA : nullptr;
                    it.sqB = nd == 1 ? sqB : nullptr;
                    items.push_back(it);
                }
    }
}

void build_batch_tables(const Plan *plans, const mwmm_problem *probs, uint8_t *const *ws_base, int count,
                        int *err, BatchTables &T) {
    T = BatchTables();
    T.split_jobs.resize(split_job_bytes() * 2 * (size_t)count);
    int nsj = 0;
    std::vector<size_t> prob_start;  // first item of each tensor-form problem
    for (int i = 0; i < count; ++i) {
        const Plan &pl = plans[i];
        const mwmm_problem &q = probs[i];
        if (pl.m == 0 || pl.n == 0 || pl.k == 0) continue;
        if (pl.form != MWMM_FORM_FP64) prob_start.push_back(T.items.size());
        uint8_t *w = ws_base[i];
        uint32_t *sqA = pl.form == MWMM_FORM_INT8 ? plan_sq(pl, w, 0) : nullptr;
        uint32_t *sqB = pl.form == MWMM_FORM_INT8 ? plan_sq(pl, w, 1) : nullptr;
        if (sqA) T.cert = 1;
        split_job(pl, 0, q.A, q.lda, w + pl.A_off, &T.split_jobs[split_job_bytes() * nsj], nsj, T.split_blocks, sqA);
        ++nsj;
        split_job(pl, 1, q.B, q.ldb, w + pl.B_off, &T.split_jobs[split_job_bytes() * nsj], nsj, T.split_blocks, sqB);
        ++nsj;
        if (pl.form == MWMM_FORM_FP64) {
            T.f64_recs.resize(T.f64_recs.size() + fp64_job_bytes());
            fp64_job(pl, w + pl.A_off, w + pl.B_off, q.C, q.ldc, err, &T.f64_recs[T.f64_recs.size() - fp64_job_bytes()],
                     (int)(T.f64_recs.size() / fp64_job_bytes()) - 1, T.f64_jobs);
        } else if (pl.form == MWMM_FORM_CRT8) {
            int32_t *S = reinterpret_cast<int32_t *>(w + pl.S_off);
            tc_items(pl, w + pl.A_off, w + pl.B_off, S, T.items);
            T.crt_recs.resize(T.crt_recs.size() + crt_job_bytes());
            crt_job(pl, S, q.C, q.ldc, &T.crt_recs[T.crt_recs.size() - crt_job_bytes()],
                    (int)(T.crt_recs.size() / crt_job_bytes()) - 1, T.crt_jobs);
        } else {
            int32_t *S = reinterpret_cast<int32_t *>(w + pl.S_off);
            tc_items(pl, w + pl.A_off, w + pl.B_off, S, T.items, sqA, sqB);
            T.rec_recs.resize(T.rec_recs.size() + recombine_job_bytes());
            recombine_job(pl, S, q.C, q.ldc, &T.rec_recs[T.rec_recs.size() - recombine_job_bytes()],
                          (int)(T.rec_recs.size() / recombine_job_bytes()) - 1, T.rec_jobs);
        }
    }
    T.split_jobs.resize(split_job_bytes() * nsj);
    if (!T.items.empty()) {
        T.ctas = (int)std::min<int64_t>((int64_t)T.items.size(), tc_sm_count());
        claim_order(T.items, prob_start, T.cta_off);
    }
    T.nsplit = (int)(T.split_blocks.size() / 4);
    T.nrec = (int)(T.rec_jobs.size() / 4);
    T.nf64 = (int)(T.f64_jobs.size() / 4);
    T.ncrt = (int)(T.crt_jobs.size() / 4);
}

int launch_product(const Plan &pl, const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb, uint64_t *dC,
                   int64_t ldc, uint8_t *ws, void *stream) {
    if (pl.m == 0 || pl.n == 0 || pl.k == 0) return 0;
    int e = launch_split(pl, 0, dA, lda, ws + pl.A_off, stream, plan_sq(pl, ws, 0));
    if (!e) e = launch_split(pl, 1, dB, ldb, ws + pl.B_off, stream, plan_sq(pl, ws, 1));
    if (e) return e;
    if (pl.form == MWMM_FORM_FP64)
        return launch_gemm_fp64(pl, ws + pl.A_off, ws + pl.B_off, dC, ldc, reinterpret_cast<uint64_t *>(ws + pl.S_off),
                                pl.err_dev, stream);
    return launch_tensor_products(pl, ws, dC, ldc, pl.err_dev, stream);
}

int launch_tensor_products(const Plan &pl, uint8_t *ws, uint64_t *C, int64_t ldc, int *err, void *stream) {
    if (pl.tc_fused)
        return launch_gemm_tc_fused(pl, ws + pl.A_off, ws + pl.B_off, C, ldc, reinterpret_cast<uint64_t *>(ws + pl.S_off),
                                    err, stream);
    int32_t *S = reinterpret_cast<int32_t *>(ws + pl.S_off);
    int e = launch_gemm_tc(pl, ws + pl.A_off, ws + pl.B_off, S, err, stream, plan_sq(pl, ws, 0), plan_sq(pl, ws, 1));
    if (!e) e = launch_recombine(pl, S, C, ldc, stream);
    return e;
}

int64_t batch_items(const Plan &pl) {
    if (pl.m == 0 || pl.n == 0 || pl.k == 0) return 0;
    if (pl.form == MWMM_FORM_FP64) return ((pl.m + 63) / 64) * ((pl.n + 63) / 64);
    const int64_t mtc = pl.A_rows / kTcBM, ntc = pl.tc_nb == kTcBN ? pl.B_rows / kTcBN : 1;
    const int64_t nwin = pl.form == MWMM_FORM_CRT8 ? pl.crt_s : (pl.nsums + pl.tc_ndiag - 1) / pl.tc_ndiag;
    return mtc * ntc * nwin * pl.nkc;
}

// Offsets and total size of the packed tables; with dst != nullptr (and the
// total <= capacity) the tables are copied there.
uint64_t pack_batch_tables_to(const BatchTables &T, uint8_t *dst, uint64_t capacity, uint64_t off[kBatchTables]) {
    const void *src[kBatchTables] = {T.split_jobs.data(), T.split_blocks.data(), T.items.data(), T.cta_off.data(),
                                     T.rec_recs.data(),   T.rec_jobs.data(),     T.f64_recs.data(), T.f64_jobs.data(),
                                     T.crt_recs.data(),   T.crt_jobs.data()};
    const uint64_t bytes[kBatchTables] = {T.split_jobs.size(), T.split_blocks.size() * sizeof(int),
                                          T.items.size() * sizeof(TcItem), T.cta_off.size() * sizeof(int64_t),
                                          T.rec_recs.size(), T.rec_jobs.size() * sizeof(int), T.f64_recs.size(),
                                          T.f64_jobs.size() * sizeof(int), T.crt_recs.size(),
                                          T.crt_jobs.size() * sizeof(int)};
    uint64_t tb = 0;
    for (int i = 0; i < kBatchTables; ++i) {
        off[i] = tb;
        tb = (tb + bytes[i] + 255) & ~uint64_t(255);
    }
    if (dst && tb <= capacity)
        for (int i = 0; i < kBatchTables; ++i)
            if (bytes[i]) std::memcpy(dst + off[i], src[i], bytes[i]);
    return tb;
}

uint64_t pack_batch_tables(const BatchTables &T, std::vector<uint8_t> &blob, uint64_t off[kBatchTables]) {
    const uint64_t tb = pack_batch_tables_to(T, nullptr, 0, off);
    blob.assign(tb, 0);
    return pack_batch_tables_to(T, blob.data(), tb, off);
}

int launch_batch_tables(const BatchTables &T, const uint8_t *dtables, const uint64_t off[kBatchTables], int fp64,
                        int chunk_blocks, int *err, void *stream) {
    int e = launch_split_batched(dtables + off[0], reinterpret_cast<const int *>(dtables + off[1]), T.nsplit, fp64,
                                 stream, T.cert);
    if (e) return e;
    if (fp64) return launch_gemm_fp64_batched(dtables + off[6], reinterpret_cast<const int *>(dtables + off[7]),
                                              T.nf64, stream);
    e = launch_gemm_tc_table(reinterpret_cast<const TcItem *>(dtables + off[2]),
                             const_cast<int64_t *>(reinterpret_cast<const int64_t *>(dtables + off[3])),
                             (int64_t)T.items.size(), T.ctas, chunk_blocks, err, stream, T.cert);
    if (e) return e;
    e = launch_recombine_batched(dtables + off[4], reinterpret_cast<const int *>(dtables + off[5]), T.nrec, stream);
    if (e) return e;
    return launch_crt_batched(dtables + off[8], reinterpret_cast<const int *>(dtables + off[9]), T.ncrt, stream);
}

}  // namespace mwmm

namespace {

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

mwmm_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return MWMM_OK;
    return e == cudaErrorMemoryAllocation ? MWMM_ERR_NOMEM : MWMM_ERR_CUDA;
}

void free_batch(mwmm_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ws) cudaFree(b->ws);
    if (b->tables) cudaFree(b->tables);
    if (b->err) cudaFree(b->err);
    delete b;
}

mwmm_status record(mwmm_batch_s *b, cudaStream_t s) {
    const int fp64 = b->form == MWMM_FORM_FP64;
    int e = mwmm::launch_split_batched(b->d_split_jobs, b->d_split_blocks, b->nsplit, fp64, s, b->cert);
    if (e) return cuda_st((cudaError_t)e);
    if (fp64) {
        e = mwmm::launch_gemm_fp64_batched(b->d_f64, b->d_f64_jobs, b->nf64, s);
        return cuda_st((cudaError_t)e);
    }
    e = mwmm::launch_gemm_tc_table(b->d_items, const_cast<int64_t *>(b->d_cta_off), b->nitems, b->ntc_ctas,
                                   b->chunk_blocks, b->err, s, b->cert);
    if (e) return cuda_st((cudaError_t)e);
    e = mwmm::launch_recombine_batched(b->d_rec, b->d_rec_jobs, b->nrec, s);
    if (e) return cuda_st((cudaError_t)e);
    e = mwmm::launch_crt_batched(b->d_crt, b->d_crt_jobs, b->ncrt, s);
    return cuda_st((cudaError_t)e);
}

bool same_problems(const mwmm_batch_s *b, const mwmm_problem *probs, int count, int form) {
    if (!b || b->form != form || (int)b->probs.size() != count) return false;
    return std::memcmp(b->probs.data(), probs, sizeof(mwmm_problem) * (size_t)count) == 0;
}

}  // namespace

extern "C" {

mwmm_status mwmm_batch_create(mwmm_batch_t *out, const mwmm_problem *probs, int count, mwmm_form form,
                              const mwmm_plan_opts *opts) {
    if (!out || count < 0 || (count > 0 && !probs)) return MWMM_ERR_ARG;
    *out = nullptr;
    if (form != MWMM_FORM_AUTO && form != MWMM_FORM_FP64 && form != MWMM_FORM_INT8 && form != MWMM_FORM_CRT8)
        return MWMM_ERR_ARG;
    mwmm_batch_s *b = new (std::nothrow) mwmm_batch_s();
    if (!b) return MWMM_ERR_NOMEM;
    b->form = form;
    if (opts && opts->tc_chunk) b->chunk_blocks = opts->tc_chunk / mwmm::kTcKB;
    b->probs.assign(probs, probs + count);
    b->plans.resize(count);
    // ---- form of each problem: the requested one, or under AUTO the tensor
    // form of the planner's cost model (per problem: the sizes of one bitsize
    // group span a wide range, and measured on the 512-instance batch this
    // beats one timed form per group)
    std::vector<int> pform(count);
    for (int i = 0; i < count; ++i)
        pform[i] = form != MWMM_FORM_AUTO ? (int)form
                                          : mwmm::choose_tensor_form(probs[i].m, probs[i].n, probs[i].k, probs[i].p);
    // ---- autotuning: one configuration per (bitsize, form) group, timed on
    // the group's median-size problem (or taken from the autotuner's cache)
    struct Tuned { bool ok = false; int form = 0, u = 0, v = 0; mwmm_plan_opts o{}; };
    auto gkey = [](int bits, int f) { return bits * 4 + (f & 3); };
    std::vector<Tuned> tuned(65 * 4);
    if (opts && opts->autotune) {
        std::vector<std::vector<int>> groups(65 * 4);
        for (int i = 0; i < count; ++i) {
            int bits = 0;
            for (uint64_t x = probs[i].p; x; x >>= 1) ++bits;
            if (probs[i].m > 0 && probs[i].n > 0 && probs[i].k > 0 && bits <= 64)
                groups[gkey(bits, pform[i])].push_back(i);
        }
        cudaStream_t ts = nullptr;
        if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return MWMM_ERR_CUDA;
        }
        for (int gi = 0; gi < 65 * 4; ++gi) {
            std::vector<int> &g = groups[gi];
            if (g.empty()) continue;
            std::sort(g.begin(), g.end(), [&](int a, int c) {
                return (double)probs[a].m * probs[a].n * probs[a].k < (double)probs[c].m * probs[c].n * probs[c].k;
            });
            const mwmm_problem &q = probs[g[g.size() / 2]];
            int f = 0, tried = 0;
            double ms = 0;
            Tuned t;
            if (mwmm::autotune(gi & 3, q.m, q.n, q.k, q.p, nullptr, 0, nullptr, 0, true, ts, &f, &t.u, &t.v, &t.o,
                               &ms, &tried) == MWMM_OK) {
                t.ok = true;
                t.form = f;
                tuned[gi] = t;
                b->tuned_groups += 1;
                b->tuned_ms += ms;
            }
        }
        cudaStreamSynchronize(ts);
        cudaStreamDestroy(ts);
    }
    // ---- plans and workspace layout
    std::vector<uint64_t> base(count);
    uint64_t total = 0;
    for (int i = 0; i < count; ++i) {
        const mwmm_problem &q = probs[i];
        mwmm_plan_opts o;
        std::memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        int u = 0, v = 0;
        int bits = 0;
        for (uint64_t x = q.p; x; x >>= 1) ++bits;
        const int pf = pform[i];
        if (bits <= 64 && tuned[gkey(bits, pf)].ok) {  // the group's configuration; the caller's checks and chunk stay
            const Tuned &t = tuned[gkey(bits, pf)];
            const mwmm_plan_opts user = o;
            o = t.o;
            o.validate = user.validate;
            if (user.tc_chunk) o.tc_chunk = user.tc_chunk;
            u = t.u;
            v = t.v;
        }
        o.lambda = 0;      // per-problem block sizes: always the bound
        o.tc_pair = -1;    // table items are one-CTA tiles
        o.tc_fused = 1;    // table items write diagonal sums for the batched recombination
        o.ksplit = 1;      // batched FP64 tiles run the whole K range
        o.tc_fill = 1;     // the batch's many items fill the SMs; no K ranges for that
        mwmm_status st = mwmm::make_plan(&b->plans[i], q.m, q.n, q.k, q.p, u, v, pf, &o);
        if (st != MWMM_OK && (u || v || o.kc)) {  // the group's words do not fit this prime: plan it alone
            o.kc = 0;
            o.f64_concat = 0;
            st = mwmm::make_plan(&b->plans[i], q.m, q.n, q.k, q.p, 0, 0, pf, &o);
        }
        if (st != MWMM_OK) {
            delete b;
            return st;
        }
        const Plan &pl = b->plans[i];
        if (pl.m > 0 && pl.n > 0 && (!q.C || q.ldc < pl.n || (pl.k > 0 && (!q.A || !q.B || q.lda < pl.k ||
                                                                       q.ldb < pl.n)))) {
            delete b;
            return MWMM_ERR_ARG;
        }
        base[i] = total;
        total = align256(total + pl.ws_bytes);
        b->flops_2mnk += 2.0 * pl.m * pl.n * pl.k;
        const double prods = pl.form == MWMM_FORM_CRT8 ? (double)pl.crt_s : (double)pl.u * pl.v;
        b->word_flops += 2.0 * prods * pl.m * pl.n * pl.k;
    }
    b->ws_bytes = total;
    cudaError_t ce = cudaMalloc(&b->err, 256);
    if (ce == cudaSuccess) ce = cudaMemset(b->err, 0, 256);
    if (ce == cudaSuccess && total) ce = cudaMalloc(&b->ws, total);
    if (ce != cudaSuccess) {
        mwmm_status st = cuda_st(ce);
        free_batch(b);
        return st;
    }
    // ---- tables
    std::vector<uint8_t *> wsb(count);
    for (int i = 0; i < count; ++i) {
        b->plans[i].err_dev = b->err;
        wsb[i] = b->ws + base[i];
    }
    mwmm::BatchTables T;
    mwmm::build_batch_tables(b->plans.data(), probs, wsb.data(), count, b->err, T);
    b->nitems = (int64_t)T.items.size();
    b->nsplit = T.nsplit;
    b->nrec = T.nrec;
    b->nf64 = T.nf64;
    b->ncrt = T.ncrt;
    b->ntc_ctas = T.ctas;
    b->cert = T.cert;
    std::vector<uint8_t> blob;
    uint64_t off[mwmm::kBatchTables];
    const uint64_t tb = mwmm::pack_batch_tables(T, blob, off);
    b->table_bytes = tb;
    if (tb) {
        ce = cudaMalloc(&b->tables, tb);
        if (ce == cudaSuccess) ce = cudaMemcpy(b->tables, blob.data(), tb, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            mwmm_status st = cuda_st(ce);
            free_batch(b);
            return st;
        }
    }
    struct { uint64_t off; } pieces[mwmm::kBatchTables];
    for (int i = 0; i < mwmm::kBatchTables; ++i) pieces[i].off = off[i];
    b->d_split_jobs = b->tables + pieces[0].off;
    b->d_split_blocks = reinterpret_cast<const int *>(b->tables + pieces[1].off);
    b->d_items = reinterpret_cast<const mwmm::TcItem *>(b->tables + pieces[2].off);
    b->d_cta_off = reinterpret_cast<const int64_t *>(b->tables + pieces[3].off);
    b->d_rec = b->tables + pieces[4].off;
    b->d_rec_jobs = reinterpret_cast<const int *>(b->tables + pieces[5].off);
    b->d_f64 = b->tables + pieces[6].off;
    b->d_f64_jobs = reinterpret_cast<const int *>(b->tables + pieces[7].off);
    b->d_crt = b->tables + pieces[8].off;
    b->d_crt_jobs = reinterpret_cast<const int *>(b->tables + pieces[9].off);
    b->launches = (b->nsplit > 0) + (form == MWMM_FORM_FP64 ? (b->nf64 > 0)
                                                            : (b->ntc_ctas > 0) + (b->nrec > 0) + (b->ncrt > 0));
    // ---- capture the launches once; zero outputs of empty-k problems are set per run
    if (mwmm::prepare_kernel_attributes() != 0) {
        free_batch(b);
        return MWMM_ERR_CUDA;
    }
    cudaStream_t cs;
    ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        free_batch(b);
        return MWMM_ERR_CUDA;
    }
    ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    mwmm_status st = MWMM_OK;
    if (ce == cudaSuccess) {
        for (int i = 0; i < count; ++i) {  // k = 0: C = 0
            const Plan &pl = b->plans[i];
            if (pl.m > 0 && pl.n > 0 && pl.k == 0)
                cudaMemset2DAsync(probs[i].C, (size_t)probs[i].ldc * 8, 0, (size_t)pl.n * 8, (size_t)pl.m, cs);
        }
        st = record(b, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (st == MWMM_OK && e2 != cudaSuccess) st = MWMM_ERR_CUDA;
        b->graph = g;
        if (st == MWMM_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = MWMM_ERR_CUDA;
    } else {
        st = MWMM_ERR_CUDA;
    }
    cudaStreamDestroy(cs);
    if (st != MWMM_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return MWMM_OK;
}

mwmm_status mwmm_batch_run(mwmm_batch_t b, void *stream) {
    if (!b) return MWMM_ERR_ARG;
    if (!b->exec) return MWMM_OK;
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? MWMM_OK : MWMM_ERR_CUDA;
}

mwmm_status mwmm_batch_check(mwmm_batch_t b, void *stream) {
    if (!b) return MWMM_ERR_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MWMM_ERR_CUDA;
    int flags[2] = {0, 0};
    if (cudaMemcpy(flags, b->err, sizeof(flags), cudaMemcpyDeviceToHost) != cudaSuccess) return MWMM_ERR_CUDA;
    if (flags[0] || flags[1]) cudaMemset(b->err, 0, sizeof(flags));
    if (flags[0]) return MWMM_ERR_TIMEOUT;
    if (flags[1]) return MWMM_ERR_RANGE;
    return MWMM_OK;
}

mwmm_status mwmm_batch_info(mwmm_batch_t b, mwmm_batch_desc *d) {
    if (!b || !d) return MWMM_ERR_ARG;
    std::memset(d, 0, sizeof(*d));
    d->count = (int32_t)b->probs.size();
    d->form = b->form;
    d->items = b->nitems;
    d->ctas = b->ntc_ctas;
    d->launches = b->launches;
    d->workspace_bytes = b->ws_bytes;
    d->table_bytes = b->table_bytes;
    d->flops_2mnk = b->flops_2mnk;
    d->word_flops = b->word_flops;
    d->tuned_groups = b->tuned_groups;
    d->tuned_ms = b->tuned_ms;
    return MWMM_OK;
}

mwmm_status mwmm_batch_problem_info(mwmm_batch_t b, int index, mwmm_plan_desc *d) {
    if (!b || !d || index < 0 || index >= (int)b->plans.size()) return MWMM_ERR_ARG;
    mwmm::describe_plan(b->plans[index], d);
    return MWMM_OK;
}

void mwmm_batch_destroy(mwmm_batch_t b) {
    if (!b) return;
    free_batch(b);
}

mwmm_status mwmm_matmul_batched(const mwmm_problem *probs, int count, mwmm_form form, mwmm_batch_t *cache,
                                void *stream) {
    mwmm_batch_t b = cache ? *cache : nullptr;
    if (!same_problems(b, probs, count, (int)form)) {
        if (b) {
            cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
            mwmm_batch_destroy(b);
        }
        b = nullptr;
        mwmm_status st = mwmm_batch_create(&b, probs, count, form, nullptr);
        if (cache) *cache = b;
        if (st != MWMM_OK) return st;
    }
    mwmm_status st = mwmm_batch_run(b, stream);
    if (!cache) {
        if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && st == MWMM_OK)
            st = MWMM_ERR_CUDA;
        mwmm_batch_destroy(b);
    }
    return st;
}

}  // extern "C"
