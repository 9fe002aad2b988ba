// C ABI of the decoding library: code objects, parameter validation, workspace and
// dispatch to the flooding / layered kernels, the multi-stream host path (Sec. III-C)
// and per-kernel event timing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ldpc_internal.h"
#include "layered_pairs.h"

namespace {

thread_local std::string g_err;

ldpc_status fail(ldpc_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
ldpc_status fail(ldpc_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

ldpc_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(LDPC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------------- profiling state

std::atomic<int64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct Pending {
    int family;
    cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;
int64_t g_fam_launches[ldpc::F_COUNT];
double g_fam_ms[ldpc::F_COUNT];

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_pending()
{
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_fam_launches[p.family]++;
            g_fam_ms[p.family] += ms;
        }
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

namespace ldpc {

void set_error(const char *msg) { g_err = msg; }

LaunchScope::LaunchScope(int fam, cudaStream_t s) : family(fam), stream(s), on(false)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_prof_on.load(std::memory_order_relaxed)) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        ev[0] = take_event();
        ev[1] = take_event();
        if (ev[0] && ev[1] && cudaEventRecord(ev[0], s) == cudaSuccess) on = true;
    }
}

LaunchScope::~LaunchScope()
{
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (cudaEventRecord(ev[1], stream) == cudaSuccess) g_pending.push_back({family, ev[0], ev[1]});
    if (g_pending.size() > 4096) drain_pending();
}

// One input status word per device, allocated with the first code created on it and kept
// for the life of the process (codes embed its address in their device tables).
namespace {
std::mutex g_status_mu;
unsigned int *g_status[64];
}  // namespace

cudaError_t device_status_word(int dev, unsigned int **out)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status[dev]) {
        unsigned int *w = nullptr;  // [0] the status word, [1] the value last taken from it
        cudaError_t e = cudaMalloc(&w, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(w, 0, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            if (w) cudaFree(w);
            return e;
        }
        g_status[dev] = w;
    }
    *out = g_status[dev];
    return cudaSuccess;
}

// Swap the status word for zero in stream order (kernels of other streams may set bits at
// any time; an exchange loses none of them).
__global__ void k_take_status(unsigned int *w) { w[1] = atomicExch(w, 0u); }

}  // namespace ldpc

using ldpc::CodeDev;

extern "C" {

const char *ldpc_last_error(void) { return g_err.c_str(); }

ldpc_status ldpc_default_params(ldpc_decode_params *p)
{
    if (!p) return fail(LDPC_EINVAL, "params is NULL");
    memset(p, 0, sizeof *p);
    p->sched = LDPC_SCHED_FLOODING;
    p->algo = LDPC_ALGO_SPA;
    p->msg = LDPC_MSG_F32;
    p->max_iter = 20;
    p->early_exit = 1;
    p->phi_clamp = 80.0f;
    p->nms_alpha_num = 3;
    p->nms_alpha_shift = 2;
    p->msg_sat = 31;
    p->app_sat = 127;
    p->llr_scale = 2.0f;
    p->impl = LDPC_IMPL_AUTO;
    return LDPC_OK;
}

ldpc_status ldpc_code_create(const int32_t *base, int32_t mb, int32_t nb, int32_t Z, ldpc_code **out)
{
    if (!base || !out) return fail(LDPC_EINVAL, "base or out is NULL");
    if (mb < 1 || nb <= mb || mb > ldpc::MB_MAX || nb > ldpc::NB_MAX)
        return fail(LDPC_EINVAL, "need 1 <= mb < nb, mb <= %d, nb <= %d (got %d x %d)", ldpc::MB_MAX, ldpc::NB_MAX,
                    mb, nb);
    if (Z < 1 || Z > ldpc::Z_MAX) return fail(LDPC_EINVAL, "Z must be in [1, %d] (got %d)", ldpc::Z_MAX, Z);
    ldpc_code *c = new (std::nothrow) ldpc_code;
    if (!c) return fail(LDPC_ENOMEM, "host allocation failed");
    memset(&c->host, 0, sizeof c->host);
    c->dev = nullptr;
    c->tuned_flood[0] = c->tuned_flood[1] = SCHED_UNTUNED;
    c->tuned_layered = SCHED_UNTUNED;
    CodeDev &h = c->host;
    h.mb = mb;
    h.nb = nb;
    h.Z = Z;
    int nnz = 0;
    std::vector<int> coldeg(nb, 0);
    for (int l = 0; l < mb; l++) {
        h.rowptr[l] = nnz;
        int deg = 0;
        for (int j = 0; j < nb; j++) {
            const int s = base[l * nb + j];
            if (s < -1 || s >= Z) {
                delete c;
                return fail(LDPC_EINVAL, "base[%d][%d] = %d outside [-1, Z=%d)", l, j, s, Z);
            }
            if (s < 0) continue;
            if (nnz >= ldpc::NNZ_MAX) {
                delete c;
                return fail(LDPC_EINVAL, "more than %d nonzero blocks", ldpc::NNZ_MAX);
            }
            h.ent[nnz++] = (j << 16) | s;
            deg++;
            coldeg[j]++;
        }
        if (deg < 2) {
            delete c;
            return fail(LDPC_EINVAL, "block row %d has %d nonzero blocks (need >= 2)", l, deg);
        }
        if (deg > h.dc_max) h.dc_max = deg;
    }
    h.rowptr[mb] = nnz;
    int k = 0;
    for (int j = 0; j < nb; j++) {
        if (coldeg[j] < 1) {
            delete c;
            return fail(LDPC_EINVAL, "block column %d is empty", j);
        }
        if (coldeg[j] > h.dv_max) h.dv_max = coldeg[j];
        h.colptr[j] = k;
        for (int b = 0; b < nnz; b++)
            if ((h.ent[b] >> 16) == j) h.colent[k++] = (b << 16) | (h.ent[b] & 0xffff);
    }
    h.colptr[nb] = k;
    {
        int n = 0;
        for (int d = 2; d <= 9; d++) {
            h.dbeg[d - 2] = n;
            for (int l = 0; l < mb; l++) {
                const int dl = h.rowptr[l + 1] - h.rowptr[l];
                if (d < 9 ? dl == d : dl > 8) h.rord[n++] = l;
            }
        }
        h.dbeg[8] = n;
    }
    h.nnz = nnz;
    h.N = nb * Z;
    h.M = mb * Z;
    h.K = h.N - h.M;
    h.E = nnz * Z;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = ldpc::device_status_word(c->device, &h.status);
    if (e == cudaSuccess) e = cudaMalloc(&c->dev, sizeof(CodeDev));
    if (e == cudaSuccess) e = cudaMemcpy(c->dev, &h, sizeof(CodeDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "device code tables");
    }
    *out = c;
    return LDPC_OK;
}

void ldpc_code_destroy(ldpc_code *c)
{
    if (!c) return;
    if (c->dev) cudaFree(c->dev);
    delete c;
}

ldpc_status ldpc_code_info(const ldpc_code *c, int32_t *N, int32_t *K, int32_t *M, int64_t *E)
{
    if (!c) return fail(LDPC_EINVAL, "code is NULL");
    if (N) *N = c->host.N;
    if (K) *K = c->host.K;
    if (M) *M = c->host.M;
    if (E) *E = c->host.E;
    return LDPC_OK;
}

static ldpc_status check_params(const ldpc_code *c, const ldpc_decode_params *p, int llr_type)
{
    if (!c || !p) return fail(LDPC_EINVAL, "code or params is NULL");
    if (p->max_iter < 1 || p->max_iter > 10000) return fail(LDPC_EINVAL, "max_iter must be in [1, 10000]");
    if (p->early_exit != 0 && p->early_exit != 1) return fail(LDPC_EINVAL, "early_exit must be 0 or 1");
    for (int i = 0; i < 4; i++)
        if (p->reserved[i] != 0) return fail(LDPC_EINVAL, "reserved fields must be zero");
    if (p->impl != LDPC_IMPL_AUTO && p->impl != LDPC_IMPL_PLAIN && p->impl != LDPC_IMPL_STREAMING &&
        p->impl != LDPC_IMPL_CLUSTER)
        return fail(LDPC_EINVAL, "bad impl");
    if (p->sched == LDPC_SCHED_FLOODING && p->algo == LDPC_ALGO_SPA) {
        if (p->msg != LDPC_MSG_F32 && p->msg != LDPC_MSG_F16)
            return fail(LDPC_ENOTSUP, "flooding SPA stores messages as F32 or F16");
        if (!(p->phi_clamp > 1.0f) || !(p->phi_clamp <= 87.0f))
            return fail(LDPC_EINVAL, "phi_clamp must be in (1, 87] so that phi(X) is a normal fp32 value");
        if (llr_type != LDPC_LLR_F32) return fail(LDPC_EINVAL, "flooding SPA takes fp32 LLRs");
        if (p->impl == LDPC_IMPL_PLAIN && p->msg != LDPC_MSG_F32)
            return fail(LDPC_ENOTSUP, "the plain comparator stores F32 messages");
        if (p->impl == LDPC_IMPL_CLUSTER && !ldpc::cluster_supported(c->host, p->msg))
            return fail(LDPC_ENOTSUP, "code does not fit the cluster decoder");
        if (c->host.dc_max > 32) return fail(LDPC_ENOTSUP, "check degree %d > 32", c->host.dc_max);
        return LDPC_OK;
    }
    if (p->sched == LDPC_SCHED_LAYERED && p->algo == LDPC_ALGO_SPA) {
        if (p->msg != LDPC_MSG_F32 && p->msg != LDPC_MSG_F16)
            return fail(LDPC_ENOTSUP, "layered SPA stores messages as F32 or F16");
        if (!(p->phi_clamp > 1.0f) || !(p->phi_clamp <= 87.0f))
            return fail(LDPC_EINVAL, "phi_clamp must be in (1, 87] so that phi(X) is a normal fp32 value");
        if (llr_type != LDPC_LLR_F32) return fail(LDPC_EINVAL, "layered SPA takes fp32 LLRs");
        if (p->impl != LDPC_IMPL_AUTO) return fail(LDPC_ENOTSUP, "layered SPA has only the on-chip slot decoder");
        if (ldpc::layered_spa_slots_per_cta(c->host, p->msg) < 1)
            return fail(LDPC_ENOTSUP, "code too large for on-chip layered SPA (N=%d, E=%d, dc_max=%d)", c->host.N,
                        c->host.E, c->host.dc_max);
        return LDPC_OK;
    }
    if (p->sched == LDPC_SCHED_LAYERED && p->algo == LDPC_ALGO_NMS) {
        if (p->msg != LDPC_MSG_I8) return fail(LDPC_ENOTSUP, "layered min-sum stores I8 messages");
        if (p->impl == LDPC_IMPL_PLAIN || p->impl == LDPC_IMPL_CLUSTER)
            return fail(LDPC_ENOTSUP, "layered min-sum runs on the slot decoders");
        if (p->msg_sat < 1 || p->msg_sat > 127 || p->app_sat < p->msg_sat || p->app_sat > 127)
            return fail(LDPC_EINVAL, "need 1 <= msg_sat <= app_sat <= 127");
        if (p->nms_alpha_num < 1 || p->nms_alpha_shift < 0 || p->nms_alpha_shift > 16 ||
            ((int64_t)p->nms_alpha_num * p->msg_sat >> p->nms_alpha_shift) > 127)
            return fail(LDPC_EINVAL, "min-sum scaling must keep |R| <= 127");
        if (llr_type == LDPC_LLR_F32 && !(p->llr_scale > 0.0f && isfinite(p->llr_scale)))
            return fail(LDPC_EINVAL, "llr_scale must be positive");
        if (llr_type != LDPC_LLR_F32 && llr_type != LDPC_LLR_I8) return fail(LDPC_EINVAL, "bad llr_type");
        if (!ldpc::layered_supported(c->host))
            return fail(LDPC_ENOTSUP, "code too large for on-chip layered decoding (Z=%d, dc_max=%d)", c->host.Z,
                        c->host.dc_max);
        return LDPC_OK;
    }
    return fail(LDPC_ENOTSUP, "unsupported sched/algo combination (%d, %d)", p->sched, p->algo);
}

// The on-chip slot decoder serves the flooding forms whenever one codeword's state fits in
// a CTA's shared memory; LDPC_IMPL_STREAMING and the plain comparator use the HBM layout.
static bool use_slots(const ldpc_code *c, const ldpc_decode_params *p)
{
    return p->sched == LDPC_SCHED_FLOODING && p->impl == LDPC_IMPL_AUTO && ldpc::slots_supported(c->host, p->msg) &&
           c->tuned_flood[p->msg == LDPC_MSG_F16 ? 1 : 0] != SCHED_STREAMING;
}

// The cluster decoder serves flooding codes whose codeword does not fit one CTA (AUTO), or
// any code that fits its split when asked for.
static bool use_cluster(const ldpc_code *c, const ldpc_decode_params *p)
{
    if (p->sched != LDPC_SCHED_FLOODING) return false;
    if (p->impl == LDPC_IMPL_CLUSTER) return true;
    return p->impl == LDPC_IMPL_AUTO && !ldpc::slots_supported(c->host, p->msg) &&
           ldpc::cluster_supported(c->host, p->msg) && c->tuned_flood[p->msg == LDPC_MSG_F16 ? 1 : 0] != SCHED_STREAMING;
}

// The layered min-sum runs as persistent slots (work counter in the workspace) unless
// LDPC_IMPL_STREAMING asks for the one-CTA-per-group kernel, which needs no workspace.
static bool use_layered_slots(const ldpc_code *c, const ldpc_decode_params *p)
{
    return p->sched == LDPC_SCHED_LAYERED && p->algo == LDPC_ALGO_NMS && p->impl == LDPC_IMPL_AUTO &&
           ldpc::layered_slots_per_cta(c->host) > 0 && c->tuned_layered != SCHED_STREAMING;
}

// The layered min-sum's persistent slots carry two codewords per thread in packed half
// precision where that is exact for the parameters, unless tuning picked one per thread.
#ifndef LDPC_LAYERED_PAIRS
#define LDPC_LAYERED_PAIRS 1  // 0: the min-sum slots always carry one codeword per thread
#endif
static bool use_layered_pairs(const ldpc_code *c, const ldpc_decode_params *p)
{
    return LDPC_LAYERED_PAIRS && c->tuned_layered != SCHED_SLOTS_V1 && ldpc::layered_pairs_exact(*p) &&
           ldpc::layered_pairs_per_cta(c->host) > 0;
}
static cudaError_t layered_slots_any(const ldpc_code *c, const ldpc_decode_params &p, const void *llr, int llr_type,
                                     int64_t n_cw, uint8_t *bits, int32_t *iters, float *app, void *ws,
                                     cudaStream_t s)
{
    const ldpc::HostReq rq = {c, llr, n_cw, bits, iters, app};
    return use_layered_pairs(c, &p) ? ldpc::layered_pairs_decode(c->host, c->dev, p, &rq, 1, llr_type, ws, s)
                                    : ldpc::layered_slots_decode(c->host, c->dev, p, &rq, 1, llr_type, ws, s);
}

// The layered sum-product always runs as persistent slots (check_params admits only codes
// whose slot fits a CTA).
static bool use_layered_spa(const ldpc_decode_params *p)
{
    return p->sched == LDPC_SCHED_LAYERED && p->algo == LDPC_ALGO_SPA;
}

static size_t ws_bytes(const ldpc_code *c, const ldpc_decode_params *p, int64_t n_cw)
{
    if (n_cw == 0) return 0;
    if (use_layered_slots(c, p) || use_layered_spa(p) || use_cluster(c, p)) return ldpc::SLOTS_WS_BYTES;
    if (p->sched == LDPC_SCHED_LAYERED) return 0;
    if (use_slots(c, p)) return ldpc::SLOTS_WS_BYTES;
    return ldpc::flood_ws_layout(c->host, n_cw, p->msg, nullptr, nullptr);
}

ldpc_status ldpc_workspace_size(const ldpc_code *c, const ldpc_decode_params *p, int64_t n_cw, size_t *bytes)
{
    if (!bytes) return fail(LDPC_EINVAL, "bytes is NULL");
    ldpc_status st =
        check_params(c, p, p && p->sched == LDPC_SCHED_LAYERED && p->algo == LDPC_ALGO_NMS ? LDPC_LLR_I8 : LDPC_LLR_F32);
    if (st != LDPC_OK) return st;
    if (n_cw < 0) return fail(LDPC_EINVAL, "n_cw < 0");
    *bytes = ws_bytes(c, p, n_cw);
    return LDPC_OK;
}

ldpc_status ldpc_decode_batch(const ldpc_code *c, const ldpc_decode_params *p, const void *llr, int32_t llr_type,
                              int64_t n_cw, uint8_t *bits, int32_t *iters, float *app, void *workspace,
                              size_t workspace_bytes, void *stream)
{
    ldpc_status st = check_params(c, p, llr_type);
    if (st != LDPC_OK) return st;
    if (n_cw < 0 || n_cw > ((int64_t)1 << 31)) return fail(LDPC_EINVAL, "n_cw must be in [0, 2^31]");
    if (n_cw == 0) return LDPC_OK;
    if (!llr || !bits || !iters) return fail(LDPC_EINVAL, "llr, bits and iters must be non-NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (p->sched == LDPC_SCHED_LAYERED && p->algo == LDPC_ALGO_NMS && !use_layered_slots(c, p)) {
        e = ldpc::layered_decode(c->host, c->dev, *p, llr, llr_type, n_cw, bits, iters, app, s);
        return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "layered decode launch");
    }
    const size_t need = ws_bytes(c, p, n_cw);
    void *ws = workspace;
    bool own = false;
    if (ws) {
        if (workspace_bytes < need)
            return fail(LDPC_ENOMEM, "workspace of %zu bytes < %zu needed", workspace_bytes, need);
        if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(LDPC_EINVAL, "workspace must be 256-byte aligned");
    } else {
        e = cudaMallocAsync(&ws, need, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LDPC_ENOMEM, "workspace allocation of %zu bytes failed: %s", need, cudaGetErrorString(e));
        }
        own = true;
    }
    if (use_layered_spa(p)) {
        e = ldpc::layered_spa_decode(c->host, c->dev, *p, static_cast<const float *>(llr), n_cw, bits, iters, app, ws,
                                     s);
    } else if (use_layered_slots(c, p)) {
        e = layered_slots_any(c, *p, llr, llr_type, n_cw, bits, iters, app, ws, s);
    } else if (use_slots(c, p)) {
        const ldpc::HostReq rq = {c, llr, n_cw, bits, iters, app};
        e = ldpc::flood_multi_decode(&rq, 1, *p, ws, s);
    } else if (use_cluster(c, p)) {
        const ldpc::HostReq rq = {c, llr, n_cw, bits, iters, app};
        e = ldpc::flood_cluster_decode(c->host, c->dev, *p, &rq, 1, ws, s);
    } else {
        ldpc::FloodWs w;
        ldpc::flood_ws_layout(c->host, n_cw, p->msg, &w, static_cast<char *>(ws));
        e = ldpc::flood_decode(c->host, c->dev, *p, static_cast<const float *>(llr), n_cw, bits, iters, app, w, s);
    }
    if (own) {
        cudaError_t e2 = cudaFreeAsync(ws, s);
        if (e == cudaSuccess) e = e2;
    }
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "flooding decode launch");
}

ldpc_status ldpc_decode_multi(const ldpc_request *reqs, int32_t n_req, const ldpc_decode_params *p, int32_t llr_type,
                              void *workspace, size_t workspace_bytes, void *stream)
{
    if (!reqs || n_req < 0 || n_req > ldpc::MULTI_MAX_REQS)
        return fail(LDPC_EINVAL, "need 0 <= n_req <= %d and a request array", ldpc::MULTI_MAX_REQS);
    if (!p) return fail(LDPC_EINVAL, "params is NULL");
    if (p->impl != LDPC_IMPL_AUTO) return fail(LDPC_ENOTSUP, "mixed-code launches use the slot decoders (impl AUTO)");
    ldpc::HostReq hr[ldpc::MULTI_MAX_REQS];
    const ldpc_code *seen[ldpc::MULTI_MAX_GROUPS];
    int ncodes = 0, live = 0;
    for (int i = 0; i < n_req; i++) {
        const ldpc_request &q = reqs[i];
        ldpc_status st = check_params(q.code, p, llr_type);
        if (st != LDPC_OK) return st;
        if (q.n_cw < 0 || q.n_cw > ((int64_t)1 << 31)) return fail(LDPC_EINVAL, "request %d: bad n_cw", i);
        if (q.n_cw > 0 && (!q.llr_dev || !q.bits_dev || !q.iters_dev))
            return fail(LDPC_EINVAL, "request %d: llr, bits and iters must be non-NULL", i);
        const bool fits = p->sched == LDPC_SCHED_FLOODING ? (use_slots(q.code, p) || use_cluster(q.code, p))
                          : use_layered_spa(p)               ? true
                                                             : use_layered_slots(q.code, p);
        if (!fits) return fail(LDPC_ENOTSUP, "request %d: code too large for the slot decoders", i);
        int g = 0;
        while (g < ncodes && seen[g] != q.code) g++;
        if (g == ncodes) {
            if (ncodes == ldpc::MULTI_MAX_GROUPS)
                return fail(LDPC_EINVAL, "more than %d distinct codes in one launch", ldpc::MULTI_MAX_GROUPS);
            seen[ncodes++] = q.code;
        }
        hr[i] = {q.code, q.llr_dev, q.n_cw, q.bits_dev, q.iters_dev, q.app_dev};
        live += q.n_cw > 0;
    }
    if (!live) return LDPC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *ws = workspace;
    bool own = false;
    cudaError_t e;
    if (ws) {
        if (workspace_bytes < ldpc::SLOTS_WS_BYTES)
            return fail(LDPC_ENOMEM, "workspace of %zu bytes < %zu needed", workspace_bytes, ldpc::SLOTS_WS_BYTES);
        if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(LDPC_EINVAL, "workspace must be 256-byte aligned");
    } else {
        e = cudaMallocAsync(&ws, ldpc::SLOTS_WS_BYTES, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LDPC_ENOMEM, "workspace allocation failed: %s", cudaGetErrorString(e));
        }
        own = true;
    }
    if (p->sched == LDPC_SCHED_FLOODING) {
        // slot-sized codes share one persistent launch; a code that needs a cluster per
        // codeword gets its own cluster launch (stream-ordered: the work counter is reused)
        ldpc::HostReq small[ldpc::MULTI_MAX_REQS];
        int ns = 0;
        for (int i = 0; i < n_req; i++)
            if (hr[i].n_cw > 0 && use_slots(hr[i].code, p)) small[ns++] = hr[i];
        e = ns ? ldpc::flood_multi_decode(small, ns, *p, ws, s) : cudaSuccess;
        // cluster-sized codes: one launch per code over all its requests
        bool done_req[ldpc::MULTI_MAX_REQS] = {};
        for (int i = 0; i < n_req && e == cudaSuccess; i++) {
            if (done_req[i] || hr[i].n_cw <= 0 || use_slots(hr[i].code, p)) continue;
            ldpc::HostReq same[ldpc::MULTI_MAX_REQS];
            int nsame = 0;
            for (int k = i; k < n_req; k++)
                if (!done_req[k] && hr[k].n_cw > 0 && hr[k].code == hr[i].code) {
                    same[nsame++] = hr[k];
                    done_req[k] = true;
                }
            e = ldpc::flood_cluster_decode(hr[i].code->host, hr[i].code->dev, *p, same, nsame, ws, s);
        }
    } else {
        e = cudaSuccess;
        // the min-sum decodes all requests of one code in one launch (one work sequence); the
        // layered sum-product gives every request a launch of its own (stream-ordered: the work
        // counter is reused)
        bool done_req[ldpc::MULTI_MAX_REQS] = {};
        if (!use_layered_spa(p))
            for (int i = 0; i < n_req && e == cudaSuccess; i++) {
                if (done_req[i] || hr[i].n_cw <= 0) continue;
                ldpc::HostReq same[ldpc::MULTI_MAX_REQS];
                int ns = 0;
                for (int k = i; k < n_req; k++)
                    if (!done_req[k] && hr[k].n_cw > 0 && hr[k].code == hr[i].code) {
                        same[ns++] = hr[k];
                        done_req[k] = true;
                    }
                const ldpc_code *c = hr[i].code;
                e = use_layered_pairs(c, p) ? ldpc::layered_pairs_decode(c->host, c->dev, *p, same, ns, llr_type, ws, s)
                                            : ldpc::layered_slots_decode(c->host, c->dev, *p, same, ns, llr_type, ws, s);
            }
        for (int i = 0; i < n_req && e == cudaSuccess; i++)
            if (hr[i].n_cw > 0 && !done_req[i])
                e = ldpc::layered_spa_decode(hr[i].code->host, hr[i].code->dev, *p,
                                             static_cast<const float *>(hr[i].llr), hr[i].n_cw, hr[i].bits,
                                             hr[i].iters, hr[i].app, ws, s);
    }
    if (own) {
        cudaError_t e2 = cudaFreeAsync(ws, s);
        if (e == cudaSuccess) e = e2;
    }
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "multi-request decode launch");
}

ldpc_status ldpc_autotune(ldpc_code *c, const ldpc_decode_params *p, const void *llr, int32_t llr_type, int64_t n_cw,
                          void *stream, int32_t *choice, float *ms)
{
    if (p && p->impl != LDPC_IMPL_AUTO) return fail(LDPC_EINVAL, "autotuning chooses the AUTO schedule (impl AUTO)");
    ldpc_status st = check_params(c, p, llr_type);
    if (st != LDPC_OK) return st;
    if (use_layered_spa(p)) return fail(LDPC_ENOTSUP, "layered SPA has a single schedule: nothing to tune");
    if (n_cw < 1 || !llr) return fail(LDPC_EINVAL, "autotuning needs a non-empty sample of LLRs");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *slot = p->sched == LDPC_SCHED_FLOODING ? &c->tuned_flood[p->msg == LDPC_MSG_F16 ? 1 : 0] : &c->tuned_layered;
    int cand[3], nc = 0;
    if (p->sched == LDPC_SCHED_FLOODING) {
        if (ldpc::slots_supported(c->host, p->msg)) {
            cand[nc++] = SCHED_SLOTS_V1;
            if (ldpc::slots_pairable(c->host, p->msg)) cand[nc++] = SCHED_SLOTS_V2;
        } else if (ldpc::cluster_supported(c->host, p->msg)) {
            cand[nc++] = SCHED_SLOTS_V1;  // the cluster decoder
        }
    } else if (ldpc::layered_slots_per_cta(c->host) > 0) {
        cand[nc++] = SCHED_SLOTS_V1;
        if (ldpc::layered_pairs_exact(*p) && ldpc::layered_pairs_per_cta(c->host) > 0) cand[nc++] = SCHED_SLOTS_V2;
    }
    cand[nc++] = SCHED_STREAMING;
    uint8_t *bits = nullptr;
    int32_t *it = nullptr;
    void *ws = nullptr;
    size_t wsb = 0;
    {
        const int saved = *slot;
        *slot = SCHED_STREAMING;
        wsb = ws_bytes(c, p, n_cw);
        *slot = saved;
        if (wsb < ldpc::SLOTS_WS_BYTES) wsb = ldpc::SLOTS_WS_BYTES;
    }
    cudaError_t e = cudaMalloc(&bits, (size_t)n_cw * c->host.N);
    if (e == cudaSuccess) e = cudaMalloc(&it, (size_t)n_cw * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&ws, wsb);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    int pick = SCHED_UNTUNED;
    for (int i = 0; i < nc && e == cudaSuccess; i++) {
        *slot = cand[i];
        float tmin = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
            if (rep) e = cudaEventRecord(e0, s);
            st = ldpc_decode_batch(c, p, llr, llr_type, n_cw, bits, it, nullptr, ws, wsb, stream);
            if (st != LDPC_OK) e = cudaErrorUnknown;
            if (rep && e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (rep && e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (rep && e == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && t < tmin) tmin = t;
        }
        if (ms) ms[i] = tmin;
        if (tmin < best) {
            best = tmin;
            pick = cand[i];
        }
    }
    if (ms)
        for (int i = nc; i < 3; i++) ms[i] = -1.0f;
    *slot = e == cudaSuccess ? pick : SCHED_UNTUNED;
    if (choice) *choice = *slot;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(bits);
    cudaFree(it);
    cudaFree(ws);
    if (st != LDPC_OK) return st;
    return e == cudaSuccess ? LDPC_OK : cuda_fail(e, "autotune");
}

ldpc_status ldpc_stream_check(void *stream, uint32_t *flags)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned int *w = nullptr;
    if (e == cudaSuccess) e = ldpc::device_status_word(dev, &w);
    unsigned int v = 0;
    if (e == cudaSuccess) {
        ldpc::k_take_status<<<1, 1, 0, s>>>(w);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, w + 1, sizeof v, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream check");
    if (flags) *flags = v;
    if (v)
        return fail(LDPC_EINVAL, "decoded input held %s%s%s", (v & ldpc::IN_NONFINITE) ? "non-finite fp32 LLRs" : "",
                    (v & ldpc::IN_NONFINITE) && (v & ldpc::IN_I8_RANGE) ? " and " : "",
                    (v & ldpc::IN_I8_RANGE) ? "int8 LLRs outside [-msg_sat, msg_sat]" : "");
    return LDPC_OK;
}

ldpc_status ldpc_multi_workspace_size(size_t *bytes)
{
    if (!bytes) return fail(LDPC_EINVAL, "bytes is NULL");
    *bytes = ldpc::SLOTS_WS_BYTES;
    return LDPC_OK;
}

// ---------------------------------------------------------------- multi-stream host path

namespace {
struct HostSlot {
    cudaStream_t s = nullptr;
    float *llr = nullptr;
    uint8_t *bits = nullptr;
    int32_t *iters = nullptr;
    void *ws = nullptr;
    int64_t cap_cw = 0;
    int N = 0;
    size_t ws_cap = 0;
    int device = -1;
};
thread_local std::vector<HostSlot> t_slots;

void free_slot(HostSlot &h)
{
    if (h.llr) cudaFree(h.llr);
    if (h.bits) cudaFree(h.bits);
    if (h.iters) cudaFree(h.iters);
    if (h.ws) cudaFree(h.ws);
    if (h.s) cudaStreamDestroy(h.s);
    h = HostSlot();
}
}  // namespace

void ldpc_release_host_buffers(void)
{
    for (auto &h : t_slots) {
        if (h.s) cudaStreamSynchronize(h.s);
        free_slot(h);
    }
    t_slots.clear();
}

ldpc_status ldpc_decode_host(const ldpc_code *c, const ldpc_decode_params *p, const float *llr_host, int64_t n_cw,
                             uint8_t *bits_host, int32_t *iters_host, int32_t W, int64_t chunk_cw)
{
    ldpc_status st = check_params(c, p, LDPC_LLR_F32);
    if (st != LDPC_OK) return st;
    if (n_cw < 0) return fail(LDPC_EINVAL, "n_cw < 0");
    if (n_cw == 0) return LDPC_OK;
    if (!llr_host || !bits_host) return fail(LDPC_EINVAL, "llr_host and bits_host must be non-NULL");
    if (W < 1 || W > 64) return fail(LDPC_EINVAL, "n_streams must be in [1, 64]");
    if (chunk_cw <= 0) chunk_cw = (n_cw + W - 1) / W;
    const int N = c->host.N;
    int dev = 0;
    cudaGetDevice(&dev);
    if ((int)t_slots.size() < W) t_slots.resize(W);
    const size_t wsb = ws_bytes(c, p, chunk_cw);
    for (int w = 0; w < W; w++) {
        HostSlot &h = t_slots[w];
        if (h.device != dev || h.cap_cw < chunk_cw || h.N < N || h.ws_cap < wsb) {
            if (h.s) cudaStreamSynchronize(h.s);
            free_slot(h);
            h.device = dev;
            cudaError_t e = cudaStreamCreateWithFlags(&h.s, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaMalloc(&h.llr, (size_t)chunk_cw * N * sizeof(float));
            if (e == cudaSuccess) e = cudaMalloc(&h.bits, (size_t)chunk_cw * N);
            if (e == cudaSuccess) e = cudaMalloc(&h.iters, (size_t)chunk_cw * sizeof(int32_t));
            if (e == cudaSuccess && wsb) e = cudaMalloc(&h.ws, wsb);
            if (e != cudaSuccess) {
                cudaGetLastError();
                free_slot(h);
                return fail(LDPC_ENOMEM, "multi-stream buffers: %s", cudaGetErrorString(e));
            }
            h.cap_cw = chunk_cw;
            h.N = N;
            h.ws_cap = wsb;
        }
    }
    int64_t done = 0;
    for (int64_t i = 0; done < n_cw; i++) {
        HostSlot &h = t_slots[i % W];
        const int64_t cnt = (n_cw - done) < chunk_cw ? (n_cw - done) : chunk_cw;
        cudaError_t e = cudaMemcpyAsync(h.llr, llr_host + done * N, (size_t)cnt * N * sizeof(float),
                                        cudaMemcpyHostToDevice, h.s);
        if (e != cudaSuccess) return cuda_fail(e, "H2D copy");
        st = ldpc_decode_batch(c, p, h.llr, LDPC_LLR_F32, cnt, h.bits, h.iters, nullptr, h.ws, h.ws_cap, h.s);
        if (st != LDPC_OK) return st;
        e = cudaMemcpyAsync(bits_host + done * N, h.bits, (size_t)cnt * N, cudaMemcpyDeviceToHost, h.s);
        if (e == cudaSuccess && iters_host)
            e = cudaMemcpyAsync(iters_host + done, h.iters, (size_t)cnt * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                h.s);
        if (e != cudaSuccess) return cuda_fail(e, "D2H copy");
        done += cnt;
    }
    for (int w = 0; w < W; w++) {
        cudaError_t e = cudaStreamSynchronize(t_slots[w].s);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    }
    return LDPC_OK;
}

// ---------------------------------------------------------------- profiling

ldpc_status ldpc_profile_enable(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on.store(on ? 1 : 0);
    return LDPC_OK;
}

ldpc_status ldpc_profile_read(int32_t family, int64_t *launches, double *ms)
{
    if (family < 0 || family >= ldpc::F_COUNT) return fail(LDPC_EINVAL, "bad kernel family %d", family);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending();
    if (launches) *launches = g_fam_launches[family];
    if (ms) *ms = g_fam_ms[family];
    return LDPC_OK;
}

ldpc_status ldpc_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending();
    for (int i = 0; i < ldpc::F_COUNT; i++) {
        g_fam_launches[i] = 0;
        g_fam_ms[i] = 0.0;
    }
    return LDPC_OK;
}

int64_t ldpc_launch_count(void) { return g_launches.load(); }
void ldpc_launch_count_reset(void) { g_launches.store(0); }

}  // extern "C"
