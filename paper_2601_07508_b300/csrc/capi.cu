// C ABI of libmwmm (declared in include/mwmm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "mwmm_internal.h"

using mwmm::Plan;

// Row-block pipeline of mwmm_matmul_host: rows of C depend only on the same
// rows of A, so the product runs as R row blocks (sub-plans sharing B's
// words) while copies stream on their own engines.
struct HostPipe {
    int R = 0;        // row blocks
    int64_t mb = 0;   // rows per block (the last one may be shorter)
    Plan sub, tail;   // plans of an mb-row block and of the last block
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev;  // start, B in, end, then A-in / C-ready per block
    void *ws = nullptr;
    uint64_t A_off = 0, B_off = 0, S_off = 0, ws_bytes = 0;
    ~HostPipe() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (s_in) cudaStreamDestroy(s_in);
        if (s_comp) cudaStreamDestroy(s_comp);
        if (s_out) cudaStreamDestroy(s_out);
        if (ws) cudaFree(ws);
    }
};

struct mwmm_plan_s {
    Plan pl;
    HostPipe *pipe = nullptr;  // created by the first pipelined mwmm_matmul_host
    // per-phase timing: one set of 5 events per timed call
    bool timing = false;
    std::vector<cudaEvent_t> pool;     // free events
    std::vector<cudaEvent_t> pending;  // 5 per timed call, in record order
    int64_t pending_launches = 0;
};

namespace {

mwmm_status cuda_status(int e) {
    if (e == 0) return MWMM_OK;
    if (e == (int)cudaErrorMemoryAllocation) return MWMM_ERR_NOMEM;
    return MWMM_ERR_CUDA;
}

// Device resources every call needs: the error flags (allocated on the first
// device call, on the device current at that time).
mwmm_status ensure_device(Plan &pl) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MWMM_ERR_CUDA;
    if (pl.err_dev) return dev == pl.device ? MWMM_OK : MWMM_ERR_ARG;  // the plan's state lives on pl.device
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, 256);
    if (e != cudaSuccess) return cuda_status((int)e);
    e = cudaMemset(p, 0, 256);
    if (e != cudaSuccess) {
        cudaFree(p);
        return MWMM_ERR_CUDA;
    }
    pl.err_dev = static_cast<int *>(p);
    pl.device = dev;
    return MWMM_OK;
}

mwmm_status ensure_own_ws(Plan &pl) {
    if (pl.own_ws_bytes >= pl.ws_bytes && (pl.own_ws || pl.ws_bytes == 0)) return MWMM_OK;
    if (pl.own_ws) cudaFree(pl.own_ws);
    pl.own_ws = nullptr;
    pl.own_ws_bytes = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, pl.ws_bytes);
    if (e != cudaSuccess) return cuda_status((int)e);
    pl.own_ws = p;
    pl.own_ws_bytes = pl.ws_bytes;
    return MWMM_OK;
}

bool valid_ld(const Plan &pl, int64_t lda, int64_t ldb, int64_t ldc) {
    return lda >= (pl.k > 0 ? pl.k : 1) && ldb >= (pl.n > 0 ? pl.n : 1) && ldc >= (pl.n > 0 ? pl.n : 1);
}

// Events for one timed call (5 of them), or nulls when timing is off.
struct PhaseEvents {
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

mwmm_status take_events(mwmm_plan_s *h, PhaseEvents &pe) {
    if (!h->timing) return MWMM_OK;
    for (int i = 0; i < 5; ++i) {
        if (h->pool.empty()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return MWMM_ERR_CUDA;
            h->pool.push_back(e);
        }
        pe.ev[i] = h->pool.back();
        h->pool.pop_back();
        h->pending.push_back(pe.ev[i]);
    }
    return MWMM_OK;
}

inline void rec(cudaEvent_t e, cudaStream_t s) {
    if (e) cudaEventRecord(e, s);
}

// Run the product on device pointers with a given workspace (dA == NULL:
// the A words already in the workspace are used).
mwmm_status run_product(mwmm_plan_s *h, const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb,
                        uint64_t *dC, int64_t ldc, uint8_t *ws, void *stream) {
    Plan &pl = h->pl;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pl.m == 0 || pl.n == 0) return MWMM_OK;
    if (pl.k == 0)  // empty sum: C = 0
        return cuda_status((int)cudaMemset2DAsync(dC, (size_t)ldc * 8, 0, (size_t)pl.n * 8, (size_t)pl.m, s));
    PhaseEvents pe;
    mwmm_status st = take_events(h, pe);
    if (st != MWMM_OK) return st;
    rec(pe.ev[0], s);
    int e = dA ? mwmm::launch_split(pl, 0, dA, lda, ws + pl.A_off, stream, mwmm::plan_sq(pl, ws, 0)) : 0;
    if (e) return cuda_status(e);
    rec(pe.ev[1], s);
    e = mwmm::launch_split(pl, 1, dB, ldb, ws + pl.B_off, stream, mwmm::plan_sq(pl, ws, 1));
    if (e) return cuda_status(e);
    rec(pe.ev[2], s);
    if (pl.form == MWMM_FORM_FP64) {
        e = mwmm::launch_gemm_fp64(pl, ws + pl.A_off, ws + pl.B_off, dC, ldc,
                                   reinterpret_cast<uint64_t *>(ws + pl.S_off), pl.err_dev, stream);
        rec(pe.ev[3], s);
        rec(pe.ev[4], s);
        if (h->timing) h->pending_launches += (dA ? 3 : 2) + (pl.ksplit > 1 ? 1 : 0);
        return cuda_status(e);
    }
    if (pl.tc_fused) {  // products, reduction and recombination in one kernel (+ the K-part sum)
        e = mwmm::launch_gemm_tc_fused(pl, ws + pl.A_off, ws + pl.B_off, dC, ldc,
                                       reinterpret_cast<uint64_t *>(ws + pl.S_off), pl.err_dev, stream);
        rec(pe.ev[3], s);
        rec(pe.ev[4], s);
        if (h->timing) h->pending_launches += (dA ? 3 : 2) + (pl.ksplit > 1 ? 1 : 0);
        return cuda_status(e);
    }
    int32_t *S = reinterpret_cast<int32_t *>(ws + pl.S_off);
    e = mwmm::launch_gemm_tc(pl, ws + pl.A_off, ws + pl.B_off, S, pl.err_dev, stream, mwmm::plan_sq(pl, ws, 0),
                             mwmm::plan_sq(pl, ws, 1));
    if (e) return cuda_status(e);
    rec(pe.ev[3], s);
    e = mwmm::launch_recombine(pl, S, dC, ldc, stream);
    rec(pe.ev[4], s);
    if (h->timing) h->pending_launches += dA ? 4 : 3;
    return cuda_status(e);
}

uint64_t align256u(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Rows per block: at least 512 (several waves of the word-product kernels
// per block), at most 8 blocks; R = 1 means no pipeline.
void choose_blocks(const Plan &pl, int *R, int64_t *mb) {
    const int64_t quantum = pl.form == MWMM_FORM_FP64 ? 64 : 256;
    int r = (int)std::min<int64_t>(8, pl.m / 512);
    if (r < 2 || pl.k == 0) {
        *R = 1;
        *mb = pl.m;
        return;
    }
    int64_t b = (pl.m + r - 1) / r;
    b = (b + quantum - 1) / quantum * quantum;
    *R = (int)((pl.m + b - 1) / b);
    *mb = b;
}

mwmm_status make_sub_plan(const Plan &pl, int64_t rows, Plan *out) {
    mwmm_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    o.validate = pl.validate;
    if (pl.form == MWMM_FORM_FP64) {
        o.lambda = pl.lambda;
        o.f64_concat = pl.f64_concat ? 2 : 1;
    } else {
        o.tc_chunk = (int32_t)pl.tc_chunk;
        o.kc = pl.tc_fused ? 0 : pl.kc;
        o.tc_pair = pl.tc_pair ? 1 : -1;  // the parent's tile kernel
        o.tc_fused = pl.tc_fused ? 2 : 1;  // every row block in the parent's layout of B's words
        o.tc_seg = pl.tc_seg;
        o.tc_digit_bits = pl.digit_bits;
    }
    const bool crt = pl.form == MWMM_FORM_CRT8;  // its words follow from p and k
    mwmm_status st = mwmm::make_plan(out, rows, pl.n, pl.k, pl.p, crt ? 0 : pl.u, crt ? 0 : pl.v, pl.form, &o);
    if (st != MWMM_OK) return st;
    out->tc_cert_chunk = 0;  // row blocks share one workspace laid out by the pipeline: worst-case chunks
    out->err_dev = pl.err_dev;  // shared flags (owned by the full plan)
    out->device = pl.device;
    return MWMM_OK;
}

mwmm_status ensure_pipe(mwmm_plan_s *h) {
    if (h->pipe) return MWMM_OK;
    Plan &pl = h->pl;
    std::unique_ptr<HostPipe> hp(new (std::nothrow) HostPipe());
    if (!hp) return MWMM_ERR_NOMEM;
    choose_blocks(pl, &hp->R, &hp->mb);
    mwmm_status st = make_sub_plan(pl, hp->mb, &hp->sub);
    if (st == MWMM_OK) st = make_sub_plan(pl, pl.m - (int64_t)(hp->R - 1) * hp->mb, &hp->tail);
    if (st != MWMM_OK) return st;
    // one workspace for every block: A words (mb rows), B words, then the
    // larger of the two plans' sums / partial results
    const Plan &a = hp->sub, &t = hp->tail;
    const uint64_t sreg = std::max(a.ws_bytes - a.S_off, t.ws_bytes > t.S_off ? t.ws_bytes - t.S_off : 0);
    hp->A_off = 0;
    hp->B_off = align256u(a.B_off);
    hp->S_off = align256u(hp->B_off + (a.S_off - a.B_off));
    hp->ws_bytes = align256u(hp->S_off + sreg);
    cudaError_t e = cudaMalloc(&hp->ws, hp->ws_bytes);
    if (e != cudaSuccess) return cuda_status((int)e);
    for (cudaStream_t *sp : {&hp->s_in, &hp->s_comp, &hp->s_out})
        if (cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking) != cudaSuccess) return MWMM_ERR_CUDA;
    hp->ev.resize(3 + 2 * (size_t)hp->R, nullptr);
    for (cudaEvent_t &ev : hp->ev)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return MWMM_ERR_CUDA;
    h->pipe = hp.release();
    return MWMM_OK;
}

// One row block: split its A rows, multiply by B's words, recombine into C.
int run_rows(const Plan &sub, const uint64_t *dA, int64_t lda, uint8_t *ws, const HostPipe &hp, uint64_t *dC,
             int64_t ldc, cudaStream_t s) {
    uint8_t *Aw = ws + hp.A_off, *Bw = ws + hp.B_off, *Sr = ws + hp.S_off;
    int e = mwmm::launch_split(sub, 0, dA, lda, Aw, s);
    if (e) return e;
    if (sub.form == MWMM_FORM_FP64)
        return mwmm::launch_gemm_fp64(sub, Aw, Bw, dC, ldc, reinterpret_cast<uint64_t *>(Sr), sub.err_dev, s);
    if (sub.tc_fused)
        return mwmm::launch_gemm_tc_fused(sub, Aw, Bw, dC, ldc, reinterpret_cast<uint64_t *>(Sr), sub.err_dev, s);
    e = mwmm::launch_gemm_tc(sub, Aw, Bw, reinterpret_cast<int32_t *>(Sr), sub.err_dev, s);
    if (e) return e;
    return mwmm::launch_recombine(sub, reinterpret_cast<int32_t *>(Sr), dC, ldc, s);
}

// Pipelined host product: B in, then per row block A_r in (copy stream) ->
// split, products, recombination (compute stream) -> C_r out (copy stream).
mwmm_status host_pipelined(mwmm_plan_s *h, const uint64_t *hA, int64_t lda, const uint64_t *hB, int64_t ldb,
                           uint64_t *hC, int64_t ldc, uint64_t *dA, uint64_t *dB, uint64_t *dC, cudaStream_t s) {
    Plan &pl = h->pl;
    HostPipe &hp = *h->pipe;
    cudaEvent_t *ev = hp.ev.data();
    uint8_t *ws = static_cast<uint8_t *>(hp.ws);
    cudaError_t e = cudaEventRecord(ev[0], s);  // after the caller's earlier work on `s`
    for (cudaStream_t q : {hp.s_in, hp.s_comp, hp.s_out})
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q, ev[0], 0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(dB, (size_t)pl.n * 8, hB, (size_t)ldb * 8, (size_t)pl.n * 8, (size_t)pl.k,
                              cudaMemcpyHostToDevice, hp.s_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], hp.s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.s_comp, ev[1], 0);
    if (e != cudaSuccess) return MWMM_ERR_CUDA;
    int ke = mwmm::launch_split(hp.sub, 1, dB, pl.n, ws + hp.B_off, hp.s_comp);
    if (ke) return cuda_status(ke);
    for (int r = 0; r < hp.R; ++r) {
        const int64_t r0 = (int64_t)r * hp.mb;
        const Plan &sub = r + 1 < hp.R ? hp.sub : hp.tail;
        cudaEvent_t a_in = ev[3 + 2 * r], c_ready = ev[4 + 2 * r];
        e = cudaMemcpy2DAsync(dA + r0 * pl.k, (size_t)pl.k * 8, hA + r0 * lda, (size_t)lda * 8, (size_t)pl.k * 8,
                              (size_t)sub.m, cudaMemcpyHostToDevice, hp.s_in);
        if (e == cudaSuccess) e = cudaEventRecord(a_in, hp.s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.s_comp, a_in, 0);
        if (e != cudaSuccess) return MWMM_ERR_CUDA;
        ke = run_rows(sub, dA + r0 * pl.k, pl.k, ws, hp, dC + r0 * pl.n, pl.n, hp.s_comp);
        if (ke) return cuda_status(ke);
        e = cudaEventRecord(c_ready, hp.s_comp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.s_out, c_ready, 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(hC + r0 * ldc, (size_t)ldc * 8, dC + r0 * pl.n, (size_t)pl.n * 8,
                                  (size_t)pl.n * 8, (size_t)sub.m, cudaMemcpyDeviceToHost, hp.s_out);
        if (e != cudaSuccess) return MWMM_ERR_CUDA;
    }
    e = cudaEventRecord(ev[2], hp.s_out);  // the last copy out follows every block
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[2], 0);
    return e == cudaSuccess ? MWMM_OK : MWMM_ERR_CUDA;
}

}  // namespace

extern "C" {

const char *mwmm_version(void) { return "mwmm 0.1 (sm_103a)"; }

mwmm_status mwmm_selftest_wait_timeout(int64_t cycles, void *stream) {
    if (cycles < 1 || cycles > ((int64_t)1 << 34)) return MWMM_ERR_ARG;  // at most ~9 s
    int *flag = nullptr;
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e != cudaSuccess) return cuda_status((int)e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int host = 0;
    e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = (cudaError_t)mwmm::launch_wait_probe(cycles, flag, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_status((int)e);
    return host ? MWMM_ERR_TIMEOUT : MWMM_OK;
}

const char *mwmm_status_str(mwmm_status s) {
    switch (s) {
        case MWMM_OK: return "ok";
        case MWMM_ERR_ARG: return "invalid argument";
        case MWMM_ERR_PRIME: return "p must be odd with 5 <= p < 2^52";
        case MWMM_ERR_BOUND: return "no block size >= 1 for this (u,v) and p";
        case MWMM_ERR_RANGE: return "an input entry is >= p";
        case MWMM_ERR_NOMEM: return "device allocation failed";
        case MWMM_ERR_BUDGET: return "request exceeds the memory budget";
        case MWMM_ERR_CUDA: return "CUDA runtime error";
        case MWMM_ERR_TIMEOUT: return "a bounded device wait expired";
        case MWMM_ERR_BUSY: return "busy";
        case MWMM_ERR_UNSUPPORTED: return "unsupported on this device";
    }
    return "unknown status";
}

mwmm_status mwmm_plan(mwmm_plan_t *out, int64_t m, int64_t n, int64_t k, uint64_t p, int u, int v,
                      mwmm_form form, const mwmm_plan_opts *opts) {
    if (!out) return MWMM_ERR_ARG;
    *out = nullptr;
    mwmm_plan_s *h = new (std::nothrow) mwmm_plan_s();
    if (!h) return MWMM_ERR_NOMEM;
    mwmm_status st = mwmm::make_plan(&h->pl, m, n, k, p, u, v, (int)form, opts);
    if (st != MWMM_OK) {
        delete h;
        return st;
    }
    *out = h;
    return MWMM_OK;
}

mwmm_status mwmm_plan_info(mwmm_plan_t plan, mwmm_plan_desc *d) {
    if (!plan || !d) return MWMM_ERR_ARG;
    mwmm::describe_plan(plan->pl, d);
    return MWMM_OK;
}

mwmm_form mwmm_tensor_form(int64_t m, int64_t n, int64_t k, uint64_t p) {
    mwmm::Plan pl;
    mwmm_plan_opts z;
    std::memset(&z, 0, sizeof(z));
    if (mwmm::make_plan(&pl, m, n, k, p, 0, 0, MWMM_FORM_INT8, &z) != MWMM_OK) return MWMM_FORM_AUTO;
    return (mwmm_form)mwmm::choose_tensor_form(m, n, k, p);
}

mwmm_status mwmm_plan_autotuned(mwmm_plan_t *out, int64_t m, int64_t n, int64_t k, uint64_t p, mwmm_form form,
                                const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb, void *stream) {
    if (!out) return MWMM_ERR_ARG;
    *out = nullptr;
    if ((dA && lda < std::max<int64_t>(k, 1)) || (dB && ldb < n)) return MWMM_ERR_ARG;
    // validate p and the shape first (same errors as mwmm_plan)
    Plan probe;
    mwmm_status st = mwmm::make_plan(&probe, m, n, k, p, 0, 0, form == MWMM_FORM_FP64 ? MWMM_FORM_FP64 : MWMM_FORM_INT8,
                                     nullptr);
    if (st != MWMM_OK && form != MWMM_FORM_AUTO) return st;
    if (m == 0 || n == 0 || k == 0) return mwmm_plan(out, m, n, k, p, 0, 0, form, nullptr);  // nothing to time
    int f = 0, u = 0, v = 0, tried = 0;
    double ms = 0;
    mwmm_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    st = mwmm::autotune((int)form, m, n, k, p, dA, lda, dB, ldb, false, stream, &f, &u, &v, &o, &ms, &tried);
    if (st != MWMM_OK) return st;
    st = mwmm_plan(out, m, n, k, p, u, v, (mwmm_form)f, &o);
    if (st != MWMM_OK) return st;
    (*out)->pl.tuned_ms = ms;
    (*out)->pl.tuned_tried = tried;
    return MWMM_OK;
}

}  // extern "C"

namespace mwmm {

void describe_plan(const Plan &P, mwmm_plan_desc *d) {
    std::memset(d, 0, sizeof(*d));
    d->m = P.m; d->n = P.n; d->k = P.k; d->p = P.p;
    d->form = P.form; d->u = P.u; d->v = P.v;
    d->alpha = P.alpha; d->beta = P.beta;
    d->lambda = P.lambda; d->lambda_max = P.lambda_max;
    d->tc_chunk = P.tc_chunk; d->kc = P.kc; d->nkc = P.nkc; d->nsums = P.nsums; d->tc_pair = P.tc_pair;
    d->f64_concat = P.f64_concat; d->ksplit = P.ksplit;
    d->q = P.q;
    d->kb_elems = P.kb_elems; d->nkb = P.nkb; d->A_rows = P.A_rows; d->B_rows = P.B_rows;
    d->B_wpad = P.B_wpad;
    d->tc_fused = P.tc_fused;
    d->tc_seg = P.tc_seg;
    d->A_off = P.A_off; d->B_off = P.B_off; d->S_off = P.S_off;
    d->workspace_bytes = P.ws_bytes;
    d->tuned_ms = P.tuned_ms;
    d->tuned_tried = P.tuned_tried;
    for (int i = 0; i < P.crt_s && i < 24; ++i) d->crt_m[i] = P.crt_m[i];
    d->tc_digit_bits = P.form == MWMM_FORM_CRT8 || P.form == MWMM_FORM_FP64 ? 0 : P.digit_bits;
    d->tc_cert_chunk = P.tc_cert_chunk;
}

}  // namespace mwmm

extern "C" {

size_t mwmm_workspace_size(mwmm_plan_t plan) { return plan ? (size_t)plan->pl.ws_bytes : 0; }

mwmm_status mwmm_matmul(mwmm_plan_t plan, const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb,
                        uint64_t *dC, int64_t ldc, void *workspace, size_t workspace_bytes, void *stream) {
    if (!plan) return MWMM_ERR_ARG;
    Plan &pl = plan->pl;
    if (pl.m == 0 || pl.n == 0) return MWMM_OK;
    if (!dC || (pl.k > 0 && (!dA || !dB)) || !valid_ld(pl, lda, ldb, ldc)) return MWMM_ERR_ARG;
    if (workspace && (workspace_bytes < pl.ws_bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)))
        return MWMM_ERR_ARG;
    mwmm_status st = ensure_device(pl);
    if (st != MWMM_OK) return st;
    if (!workspace) {
        st = ensure_own_ws(pl);
        if (st != MWMM_OK) return st;
        workspace = pl.own_ws;
    }
    return run_product(plan, dA, lda, dB, ldb, dC, ldc, static_cast<uint8_t *>(workspace), stream);
}

mwmm_status mwmm_matmul_reuse_a(mwmm_plan_t plan, const uint64_t *dB, int64_t ldb, uint64_t *dC, int64_t ldc,
                                void *workspace, size_t workspace_bytes, void *stream) {
    if (!plan) return MWMM_ERR_ARG;
    Plan &pl = plan->pl;
    if (pl.m == 0 || pl.n == 0) return MWMM_OK;
    if (!dC || (pl.k > 0 && !dB) || !valid_ld(pl, pl.k > 0 ? pl.k : 1, ldb, ldc)) return MWMM_ERR_ARG;
    if (workspace && (workspace_bytes < pl.ws_bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)))
        return MWMM_ERR_ARG;
    mwmm_status st = ensure_device(pl);
    if (st != MWMM_OK) return st;
    if (!workspace) {
        if (!pl.own_ws && pl.ws_bytes) return MWMM_ERR_ARG;  // no words of A to reuse yet
        workspace = pl.own_ws;
    }
    return run_product(plan, nullptr, 0, dB, ldb, dC, ldc, static_cast<uint8_t *>(workspace), stream);
}

mwmm_status mwmm_plan_check(mwmm_plan_t plan, void *stream) {
    if (!plan) return MWMM_ERR_ARG;
    Plan &pl = plan->pl;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return MWMM_ERR_CUDA;
    if (!pl.err_dev) return MWMM_OK;
    int flags[2] = {0, 0};
    e = cudaMemcpy(flags, pl.err_dev, sizeof(flags), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return MWMM_ERR_CUDA;
    if (flags[0] || flags[1]) {
        e = cudaMemset(pl.err_dev, 0, sizeof(flags));
        if (e != cudaSuccess) return MWMM_ERR_CUDA;
    }
    if (flags[0]) return MWMM_ERR_TIMEOUT;
    if (flags[1]) return MWMM_ERR_RANGE;
    return MWMM_OK;
}

mwmm_status mwmm_matmul_host_async(mwmm_plan_t plan, const uint64_t *hA, int64_t lda, const uint64_t *hB,
                                   int64_t ldb, uint64_t *hC, int64_t ldc, void *stream) {
    if (!plan) return MWMM_ERR_ARG;
    Plan &pl = plan->pl;
    if (pl.m == 0 || pl.n == 0) return MWMM_OK;
    if (!hC || (pl.k > 0 && (!hA || !hB)) || !valid_ld(pl, lda, ldb, ldc)) return MWMM_ERR_ARG;
    mwmm_status st = ensure_device(pl);
    if (st != MWMM_OK) return st;
    const uint64_t abytes = (uint64_t)pl.m * pl.k * 8, bbytes = (uint64_t)pl.k * pl.n * 8,
                   cbytes = (uint64_t)pl.m * pl.n * 8;
    const uint64_t need = ((abytes + 255) & ~uint64_t(255)) + ((bbytes + 255) & ~uint64_t(255)) + cbytes;
    if (pl.hostbuf_bytes < need) {
        if (pl.hostbuf_dev) cudaFree(pl.hostbuf_dev);
        pl.hostbuf_dev = nullptr;
        pl.hostbuf_bytes = 0;
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) return cuda_status((int)e);
        pl.hostbuf_dev = static_cast<uint64_t *>(p);
        pl.hostbuf_bytes = need;
    }
    uint8_t *base = reinterpret_cast<uint8_t *>(pl.hostbuf_dev);
    uint64_t *dA = reinterpret_cast<uint64_t *>(base);
    uint64_t *dB = reinterpret_cast<uint64_t *>(base + ((abytes + 255) & ~uint64_t(255)));
    uint64_t *dC = reinterpret_cast<uint64_t *>(base + ((abytes + 255) & ~uint64_t(255)) +
                                                ((bbytes + 255) & ~uint64_t(255)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int R = 1;
    int64_t mb = pl.m;
    choose_blocks(pl, &R, &mb);
    if (R > 1 && !plan->timing) {  // per-phase timing needs the one-stream order
        st = ensure_pipe(plan);
        if (st == MWMM_OK) st = host_pipelined(plan, hA, lda, hB, ldb, hC, ldc, dA, dB, dC, s);
        return st;
    }
    cudaError_t e = cudaSuccess;
    if (pl.k > 0) {
        e = cudaMemcpy2DAsync(dA, (size_t)pl.k * 8, hA, (size_t)lda * 8, (size_t)pl.k * 8, (size_t)pl.m,
                              cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dB, (size_t)pl.n * 8, hB, (size_t)ldb * 8, (size_t)pl.n * 8, (size_t)pl.k,
                                  cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return MWMM_ERR_CUDA;
    }
    st = ensure_own_ws(pl);
    if (st != MWMM_OK) return st;
    st = run_product(plan, dA, pl.k > 0 ? pl.k : 1, dB, pl.n, dC, pl.n, static_cast<uint8_t *>(pl.own_ws), stream);
    if (st != MWMM_OK) return st;
    e = cudaMemcpy2DAsync(hC, (size_t)ldc * 8, dC, (size_t)pl.n * 8, (size_t)pl.n * 8, (size_t)pl.m,
                          cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return MWMM_ERR_CUDA;
    return MWMM_OK;
}

mwmm_status mwmm_matmul_host(mwmm_plan_t plan, const uint64_t *hA, int64_t lda, const uint64_t *hB, int64_t ldb,
                             uint64_t *hC, int64_t ldc, void *stream) {
    mwmm_status st = mwmm_matmul_host_async(plan, hA, lda, hB, ldb, hC, ldc, stream);
    if (st != MWMM_OK || !plan || plan->pl.m == 0 || plan->pl.n == 0) return st;
    return mwmm_plan_check(plan, stream);
}

mwmm_status mwmm_plan_set_timing(mwmm_plan_t plan, int on) {
    if (!plan) return MWMM_ERR_ARG;
    plan->timing = on != 0;
    return MWMM_OK;
}

mwmm_status mwmm_plan_timing(mwmm_plan_t plan, mwmm_timing *out) {
    if (!plan || !out) return MWMM_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    mwmm_status st = MWMM_OK;
    if (!plan->pending.empty() && cudaEventSynchronize(plan->pending.back()) != cudaSuccess) st = MWMM_ERR_CUDA;
    for (size_t c = 0; st == MWMM_OK && c + 5 <= plan->pending.size(); c += 5) {
        float t[4];
        cudaEvent_t *e = &plan->pending[c];
        for (int i = 0; i < 4; ++i)
            if (cudaEventElapsedTime(&t[i], e[i], e[i + 1]) != cudaSuccess) st = MWMM_ERR_CUDA;
        out->split_a_ms += t[0];
        out->split_b_ms += t[1];
        out->gemm_ms += t[2];
        out->recombine_ms += t[3];
        out->total_ms += t[0] + t[1] + t[2] + t[3];
        out->calls += 1;
    }
    out->launches = plan->pending_launches;
    for (cudaEvent_t e : plan->pending) plan->pool.push_back(e);
    plan->pending.clear();
    plan->pending_launches = 0;
    return st;
}

void mwmm_plan_destroy(mwmm_plan_t plan) {
    if (!plan) return;
    for (cudaEvent_t e : plan->pool) cudaEventDestroy(e);
    for (cudaEvent_t e : plan->pending) cudaEventDestroy(e);
    delete plan->pipe;
    Plan &pl = plan->pl;
    if (pl.own_ws) cudaFree(pl.own_ws);
    if (pl.hostbuf_dev) cudaFree(pl.hostbuf_dev);
    if (pl.err_dev) cudaFree(pl.err_dev);
    delete plan;
}

mwmm_status mwmm_split(mwmm_plan_t plan, int side, const uint64_t *dM, int64_t ld, void *words, void *stream) {
    if (!plan || (side != 0 && side != 1) || !words) return MWMM_ERR_ARG;
    Plan &pl = plan->pl;
    const int64_t rowlen = side == 0 ? pl.k : pl.n;
    if (ld < (rowlen > 0 ? rowlen : 1) || (!dM && pl.k > 0 && (side == 0 ? pl.m : pl.n) > 0)) return MWMM_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(words) & 15) return MWMM_ERR_ARG;
    mwmm_status st = ensure_device(pl);
    if (st != MWMM_OK) return st;
    return cuda_status(mwmm::launch_split(pl, side, dM, ld, words, stream));
}

mwmm_status mwmm_fmod(const double *dx, int64_t count, uint64_t p, double *dout, void *stream) {
    if (count < 0 || (count > 0 && (!dx || !dout))) return MWMM_ERR_ARG;
    if (p < 5 || (p & 1) == 0 || p >= (uint64_t(1) << 52)) return MWMM_ERR_PRIME;
    return cuda_status(mwmm::launch_fmod(dx, count, p, dout, stream));
}

mwmm_status mwmm_mulmod(const double *dx, const double *dy, int64_t count, uint64_t p, double *dout,
                        void *stream) {
    if (count < 0 || (count > 0 && (!dx || !dy || !dout))) return MWMM_ERR_ARG;
    if (p < 5 || (p & 1) == 0 || p >= (uint64_t(1) << 52)) return MWMM_ERR_PRIME;
    return cuda_status(mwmm::launch_mulmod(dx, dy, count, p, dout, stream));
}

}  // extern "C"
