// ldpc_decode_batch_static: the flooding decode with its scratch in a fixed device array,
// for callers that must not allocate device memory while decoding (see ldpc.h).
#include <stdio.h>

#include <mutex>

#include "ldpc_internal.h"

namespace {

// The scratch of every call: LDPC_STATIC_SCRATCH_BYTES of device memory, reserved on each
// GPU that loads this part of the library, for the life of the process (with lazy module
// loading that happens at the address lookup of the first call on the device).  In host
// code this name is only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[LDPC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_dev[kMaxDevices];  // device address of g_scratch per device (null = not looked up yet)

ldpc_status say(ldpc_status st, const char *fmt, long long a = 0, long long b = 0, long long c = 0)
{
    char buf[384];
    snprintf(buf, sizeof buf, fmt, a, b, c);
    ldpc::set_error(buf);
    return st;
}

}  // namespace

extern "C" ldpc_status ldpc_decode_batch_static(const ldpc_code *code, const ldpc_decode_params *p,
                                                const float *llr_dev, int64_t n_cw, uint8_t *bits_dev,
                                                int32_t *iters_dev, float *app_dev, void *stream)
{
    if (!code || !p) return say(LDPC_EINVAL, "code or params is NULL");
    if (p->sched != LDPC_SCHED_FLOODING || p->algo != LDPC_ALGO_SPA)
        return say(LDPC_ENOTSUP, "the static-scratch entry point runs the flooding SPA forms only "
                                 "(the layered form needs no scratch: use ldpc_decode_batch)");
    size_t need = 0;
    ldpc_status st = ldpc_workspace_size(code, p, n_cw, &need);
    if (st != LDPC_OK) return st;
    if (need > LDPC_STATIC_SCRATCH_BYTES)
        return say(LDPC_ENOMEM, "n_cw = %lld needs %lld bytes of scratch but the static array holds %lld bytes",
                   (long long)n_cw, (long long)need, (long long)LDPC_STATIC_SCRATCH_BYTES);
    if (n_cw == 0) return LDPC_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return say(LDPC_ECUDA, "cudaGetDevice failed (%lld)", (long long)e);
    if (dev < 0 || dev >= kMaxDevices) return say(LDPC_ENOTSUP, "device %lld beyond the supported count", dev);
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_dev[dev]) {
            // once per device, with that device current
            e = cudaGetSymbolAddress(&g_scratch_dev[dev], g_scratch);
            if (e != cudaSuccess) {
                g_scratch_dev[dev] = nullptr;
                cudaGetLastError();
                return say(LDPC_ECUDA, "cudaGetSymbolAddress of the static scratch failed (error %lld)", (long long)e);
            }
        }
        scratch = g_scratch_dev[dev];
    }
    return ldpc_decode_batch(code, p, llr_dev, LDPC_LLR_F32, n_cw, bits_dev, iters_dev, app_dev, scratch,
                             LDPC_STATIC_SCRATCH_BYTES, stream);
}
