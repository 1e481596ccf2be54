// Autotuner: picks the configuration of a product (form, words (u,v), tile
// variant, K-range lengths) by timing candidates on the device.
//
// The paper selects (u,v) from its cost model and from measured crossovers
// (Sec. 3.3, Table 4) and notes that the best variant depends on the machine.
// Here the choice is measured on the GPU that will run the product:
//   - FP64 form: every (u,v) of (1,1) (1,2) (1,3) (1,4) (2,2) (2,3) whose
//     block size lambda >= 1 (Prop. 3.3); concatenation (Alg. 6) on and off
//     when it applies; K ranges automatic, or one range in batch mode;
//   - INT8-word form: the tcgen05 tile variant (128 x 256 one-CTA, clusters of
//     two sharing B, 256 x 256 CTA pairs; one-CTA only in batch mode) and the
//     INT32 K-range kc (the largest the bound allows, and half of k when that
//     splits the k loop), within twice the default workspace;
//   - the multimodular CRT form of Sec. 5.2 (one-CTA and, for single
//     products, pair tiles) when asked for, and for MWMM_FORM_AUTO: single
//     products try every form; a batch tries the two tensor forms (INT8 and
//     CRT), which share its word-product kernel.
// Candidates are ordered by a flop model; each is run once to warm up and
// timed twice (CUDA events, the faster run counts); a candidate whose model
// time exceeds 3x the best measured time is skipped.  The kernels' run time
// does not depend on the operand values, so zero operands serve when the
// caller passes none.
//
// Results are cached per (form, bitsize of p, log2 buckets of m, n, k, batch
// mode, SM count); with MWMM_AUTOTUNE_CACHE set, the cache is read from that
// file at the first lookup and rewritten (JSON lines) after each new entry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mwmm_internal.h"

namespace mwmm {

namespace {

struct Entry {
    int form = 0, u = 0, v = 0;
    mwmm_plan_opts o{};
    double ms = 0;
    int tried = 0;
};

std::mutex g_mu;
std::map<std::string, Entry> g_cache;
bool g_loaded = false;

int log2_bucket(int64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

int bit_length(uint64_t p) {
    int b = 0;
    while (p) {
        p >>= 1;
        ++b;
    }
    return b;
}

std::string make_key(int form, int64_t m, int64_t n, int64_t k, uint64_t p, bool batch) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "f%d.b%d.m%d.n%d.k%d.%s.sm%d", form, bit_length(p), log2_bucket(m),
                  log2_bucket(n), log2_bucket(k), batch ? "batch" : "single", tc_sm_count());
    return buf;
}

// One JSON object per line; the fields are written and read in this order.
const char *kLineFmt =
    "{\"key\": \"%[^\"]\", \"form\": %d, \"u\": %d, \"v\": %d, \"tc_chunk\": %d, \"kc\": %lld, \"tc_pair\": %d, "
    "\"tc_digit_bits\": %d, \"f64_concat\": %d, \"ksplit\": %d, \"ms\": %lf, \"tried\": %d}";

bool parse_line(const char *line, std::string *key, Entry *e) {
    char k[160];
    long long kc = 0;
    int n = std::sscanf(line, kLineFmt, k, &e->form, &e->u, &e->v, &e->o.tc_chunk, &kc, &e->o.tc_pair,
                        &e->o.tc_digit_bits, &e->o.f64_concat, &e->o.ksplit, &e->ms, &e->tried);
    if (n != 12) return false;
    e->o.kc = kc;
    *key = k;
    return true;
}

int load_file(const char *path) {
    FILE *f = std::fopen(path, "r");
    if (!f) return -1;
    char line[512];
    int count = 0;
    while (std::fgets(line, sizeof(line), f)) {
        std::string key;
        Entry e;
        std::memset(&e.o, 0, sizeof(e.o));
        if (parse_line(line, &key, &e)) {
            g_cache[key] = e;
            ++count;
        }
    }
    std::fclose(f);
    return count;
}

int save_file(const char *path) {
    FILE *f = std::fopen(path, "w");
    if (!f) return -1;
    for (const auto &kv : g_cache) {
        const Entry &e = kv.second;
        std::fprintf(f,
                     "{\"key\": \"%s\", \"form\": %d, \"u\": %d, \"v\": %d, \"tc_chunk\": %d, \"kc\": %lld, "
                     "\"tc_pair\": %d, \"tc_digit_bits\": %d, \"f64_concat\": %d, \"ksplit\": %d, \"ms\": %.6f, "
                     "\"tried\": %d}\n",
                     kv.first.c_str(), e.form, e.u, e.v, e.o.tc_chunk, (long long)e.o.kc, e.o.tc_pair,
                     e.o.tc_digit_bits, e.o.f64_concat, e.o.ksplit, e.ms, e.tried);
    }
    return std::fclose(f) == 0 ? 0 : -1;
}

void ensure_loaded() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("MWMM_AUTOTUNE_CACHE");
    if (path && *path) load_file(path);
}

struct Cand {
    Entry e;
    Plan pl;
    double model_ms = 0;
};

void add(std::vector<Cand> &out, int form, int u, int v, const mwmm_plan_opts &o, int64_t m, int64_t n,
         int64_t k, uint64_t p) {
    Cand c;
    c.e.form = form;
    c.e.u = u;
    c.e.v = v;
    c.e.o = o;
    if (make_plan(&c.pl, m, n, k, p, u, v, form, &o) != MWMM_OK) return;
    const double mnk2 = 2.0 * (double)m * (double)n * (double)std::max<int64_t>(k, 1);
    const double uv = (double)c.pl.u * c.pl.v;
    if (form == MWMM_FORM_FP64) {
        const double lam = (double)std::min<int64_t>(c.pl.lambda, std::max<int64_t>(k, 1));
        c.model_ms = uv * mnk2 * (1.0 + 3.0 / lam) / 1.0e12 * 1e3;  // FP64 pipe ~1 TFLOP/s
    } else {
        const double prods = form == MWMM_FORM_CRT8 ? (double)c.pl.crt_s : uv;  // one product per modulus
        c.model_ms = prods * mnk2 / 1.4e15 * 1e3 + (double)c.pl.ws_bytes / 5.0e12 * 1e3;
    }
    out.push_back(c);
}

void candidates(int form_req, int64_t m, int64_t n, int64_t k, uint64_t p, bool batch, std::vector<Cand> &out) {
    // A batch runs either FP64 problems or tensor-form (INT8 / CRT) problems,
    // so a batch's AUTO choice is between the two tensor forms.
    const bool want_int8 = form_req == MWMM_FORM_AUTO || form_req == MWMM_FORM_INT8;
    const bool want_crt = form_req == MWMM_FORM_AUTO || form_req == MWMM_FORM_CRT8;
    const bool want_fp64 = (form_req == MWMM_FORM_AUTO && !batch) || form_req == MWMM_FORM_FP64;
    mwmm_plan_opts z;
    std::memset(&z, 0, sizeof(z));
    z.tc_fill = batch ? 1 : 0;  // a batch's items fill the SMs together
    if (want_crt) {
        Plan crt;
        if (make_plan(&crt, m, n, k, p, 0, 0, MWMM_FORM_CRT8, &z) == MWMM_OK) {
            mwmm_plan_opts o = z;
            add(out, MWMM_FORM_CRT8, 0, 0, o, m, n, k, p);
            if (!batch && m > kTcBM && n > kTcBN / 2) {
                o.tc_pair = 1;
                add(out, MWMM_FORM_CRT8, 0, 0, o, m, n, k, p);
            }
        }
    }
    if (want_int8) {
        Plan base;
        if (make_plan(&base, m, n, k, p, 0, 0, MWMM_FORM_INT8, &z) == MWMM_OK) {
            std::vector<int64_t> kcs = {0};
            const int64_t half = (k / 2 + kTcKB - 1) / kTcKB * kTcKB;
            if (base.nkc == 1 && k >= 2048 && half < base.kc) kcs.push_back(half);
            std::vector<int> pairs = {-1};  // one-CTA tiles; the two-CTA kernel where it applies
            if (!batch && m > kTcBM && n > kTcBN / 2) pairs.push_back(1);
            for (int64_t kc : kcs)
                for (int pair : pairs) {
                    mwmm_plan_opts o = z;
                    o.kc = kc;
                    o.tc_pair = pair;
                    o.tc_digit_bits = base.digit_bits;  // the words base.u, base.v are of this width
                    const size_t before = out.size();
                    add(out, MWMM_FORM_INT8, base.u, base.v, o, m, n, k, p);
                    if (out.size() > before && out.back().pl.ws_bytes > 2 * base.ws_bytes + (64u << 20))
                        out.pop_back();  // more than twice the default workspace
                }
        }
    }
    if (want_fp64) {
        static const int uvs[6][2] = {{1, 1}, {1, 2}, {1, 3}, {1, 4}, {2, 2}, {2, 3}};
        for (const auto &uv : uvs) {
            if (block_size(p, uv[0], uv[1]) < 1) continue;
            mwmm_plan_opts o = z;
            o.ksplit = batch ? 1 : 0;
            add(out, MWMM_FORM_FP64, uv[0], uv[1], o, m, n, k, p);
            if (uv[1] >= 2 && uv[1] <= 4 && n < kF64BN) {  // concatenation applies: also try without
                o.f64_concat = 1;
                add(out, MWMM_FORM_FP64, uv[0], uv[1], o, m, n, k, p);
            }
        }
    }
    std::stable_sort(out.begin(), out.end(), [](const Cand &a, const Cand &b) { return a.model_ms < b.model_ms; });
}

// Time one candidate: warm-up, then the faster of two runs.  < 0: failed.
double time_candidate(const Cand &c, const uint64_t *dA, int64_t lda, const uint64_t *dB, int64_t ldb,
                      uint64_t *dC, void *ws, uint64_t ws_bytes, cudaStream_t s) {
    mwmm_plan_t h = nullptr;
    if (mwmm_plan(&h, c.pl.m, c.pl.n, c.pl.k, c.pl.p, c.e.u, c.e.v, (mwmm_form)c.e.form, &c.e.o) != MWMM_OK)
        return -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = -1;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        bool ok = mwmm_matmul(h, dA, lda, dB, ldb, dC, c.pl.n, ws, ws_bytes, s) == MWMM_OK;
        for (int r = 0; ok && r < 2; ++r) {
            ok = cudaEventRecord(e0, s) == cudaSuccess &&
                 mwmm_matmul(h, dA, lda, dB, ldb, dC, c.pl.n, ws, ws_bytes, s) == MWMM_OK &&
                 cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = best < 0 ? ms : std::min(best, (double)ms);
        }
        if (mwmm_plan_check(h, s) != MWMM_OK) best = -1;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    mwmm_plan_destroy(h);
    return best;
}

}  // namespace

mwmm_status autotune(int form_req, int64_t m, int64_t n, int64_t k, uint64_t p, const uint64_t *dA, int64_t lda,
                     const uint64_t *dB, int64_t ldb, bool batch, void *stream, int *form, int *u, int *v,
                     mwmm_plan_opts *opts, double *ms, int *tried) {
    if (m <= 0 || n <= 0 || k < 0) return MWMM_ERR_ARG;
    if (form_req != MWMM_FORM_AUTO && form_req != MWMM_FORM_FP64 && form_req != MWMM_FORM_INT8 &&
        form_req != MWMM_FORM_CRT8)
        return MWMM_ERR_ARG;
    const std::string key = make_key(form_req, m, n, k, p, batch);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        ensure_loaded();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            Plan check;  // a cached entry must still plan for this exact problem
            if (make_plan(&check, m, n, k, p, it->second.u, it->second.v, it->second.form, &it->second.o) == MWMM_OK) {
                *form = it->second.form;
                *u = it->second.u;
                *v = it->second.v;
                *opts = it->second.o;
                *ms = it->second.ms;
                *tried = 0;  // from the cache
                return MWMM_OK;
            }
        }
    }
    std::vector<Cand> cands;
    candidates(form_req, m, n, k, p, batch, cands);
    if (cands.empty()) return MWMM_ERR_BOUND;
    // scratch: C, the largest workspace, and zero operands when none are given
    uint64_t ws_bytes = 0;
    for (const Cand &c : cands) ws_bytes = std::max(ws_bytes, c.pl.ws_bytes);
    const uint64_t cbytes = (uint64_t)m * n * 8;
    const uint64_t abytes = dA ? 0 : (uint64_t)m * std::max<int64_t>(k, 1) * 8;
    const uint64_t bbytes = dB ? 0 : (uint64_t)std::max<int64_t>(k, 1) * n * 8;
    auto al = [](uint64_t x) { return (x + 255) & ~uint64_t(255); };
    uint8_t *scratch = nullptr;
    cudaError_t ce = cudaMalloc(&scratch, al(cbytes) + al(abytes) + al(bbytes) + std::max<uint64_t>(ws_bytes, 256));
    if (ce != cudaSuccess) return ce == cudaErrorMemoryAllocation ? MWMM_ERR_NOMEM : MWMM_ERR_CUDA;
    uint64_t *dC = reinterpret_cast<uint64_t *>(scratch);
    uint8_t *zone = scratch + al(cbytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!dA) {
        dA = reinterpret_cast<const uint64_t *>(zone);
        lda = std::max<int64_t>(k, 1);
        zone += al(abytes);
    }
    if (!dB) {
        dB = reinterpret_cast<const uint64_t *>(zone);
        ldb = n;
        zone += al(bbytes);
    }
    void *ws = zone;
    if (abytes + bbytes) ce = cudaMemsetAsync(scratch + al(cbytes), 0, al(abytes) + al(bbytes), s);
    double best = -1;
    int bi = -1, tried_n = 0;
    for (size_t i = 0; ce == cudaSuccess && i < cands.size(); ++i) {
        if (best > 0 && cands[i].model_ms > 3.0 * best) continue;
        const double t = time_candidate(cands[i], dA, lda, dB, ldb, dC, ws, ws_bytes, s);
        ++tried_n;
        if (t > 0 && (best < 0 || t < best)) {
            best = t;
            bi = (int)i;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (ce != cudaSuccess) return MWMM_ERR_CUDA;
    if (bi < 0) return MWMM_ERR_CUDA;
    Entry e = cands[bi].e;
    e.ms = best;
    e.tried = tried_n;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_cache[key] = e;
        const char *path = std::getenv("MWMM_AUTOTUNE_CACHE");
        if (path && *path) save_file(path);
    }
    *form = e.form;
    *u = e.u;
    *v = e.v;
    *opts = e.o;
    *ms = best;
    *tried = tried_n;
    return MWMM_OK;
}

}  // namespace mwmm

extern "C" {

int64_t mwmm_autotune_cache_entries(void) {
    std::lock_guard<std::mutex> lock(mwmm::g_mu);
    mwmm::ensure_loaded();
    return (int64_t)mwmm::g_cache.size();
}

void mwmm_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lock(mwmm::g_mu);
    mwmm::g_cache.clear();
    mwmm::g_loaded = true;  // do not reload the file behind the caller's back
}

mwmm_status mwmm_autotune_cache_save(const char *path) {
    if (!path) return MWMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(mwmm::g_mu);
    return mwmm::save_file(path) == 0 ? MWMM_OK : MWMM_ERR_ARG;
}

mwmm_status mwmm_autotune_cache_load(const char *path) {
    if (!path) return MWMM_ERR_ARG;
    std::lock_guard<std::mutex> lock(mwmm::g_mu);
    mwmm::g_loaded = true;
    return mwmm::load_file(path) >= 0 ? MWMM_OK : MWMM_ERR_ARG;
}

}  // extern "C"
