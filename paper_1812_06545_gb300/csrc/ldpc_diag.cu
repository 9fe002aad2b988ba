// Special-function throughput of the device (the ceiling of the sum-product check rule,
// whose phi evaluations need exponentials and logarithms): independent ex2.approx /
// lg2.approx chains on every SM, timed with CUDA events.
#include "ldpc_internal.h"

namespace {

template <int OP>
__global__ void __launch_bounds__(512) k_sfu(float *out, int iters, float seed)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = seed + threadIdx.x * 1e-6f + i * 1e-3f;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            float y;
            if (OP == 0)
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
            else
                asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
            a[i] = fmaf(y, 0.5f, 0.75f);  // stays in (0.75, 2): finite for both functions
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; i++) s += a[i];
    if (s == -1.0f) out[0] = s;  // never true; keeps the chains live
}

template <int OP>
float time_sfu(float *scratch, cudaStream_t st, int sms, double *ops_per_s)
{
    const int iters = 2048, blocks = sms * 4, threads = 512;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
        cudaEventRecord(e0, st);
        k_sfu<OP><<<blocks, threads, 0, st>>>(scratch, iters, 0.1f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep && ms < best) best = ms;  // first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ops_per_s = (double)blocks * threads * iters * 8 / (best * 1e-3);
    return best;
}

}  // namespace

extern "C" ldpc_status ldpc_sfu_throughput(double *ex2_per_s, double *lg2_per_s, void *stream)
{
    if (!ex2_per_s || !lg2_per_s) {
        ldpc::set_error("outputs must be non-NULL");
        return LDPC_EINVAL;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *scratch = nullptr;
    if (cudaMalloc(&scratch, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        ldpc::set_error("scratch allocation failed");
        return LDPC_ENOMEM;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    time_sfu<0>(scratch, st, sms, ex2_per_s);
    time_sfu<1>(scratch, st, sms, lg2_per_s);
    cudaError_t e = cudaGetLastError();
    cudaFree(scratch);
    if (e != cudaSuccess) {
        ldpc::set_error(cudaGetErrorString(e));
        return LDPC_ECUDA;
    }
    return LDPC_OK;
}
