// Flooding sum-product decoding with the decoder state on chip: the slot decoder.
//
// A persistent grid of one CTA per SM.  Each CTA holds C codeword "slots"; a slot keeps
// its posterior APP [N] (fp32) and its check-to-variable messages R [E] (fp32 or fp16) in
// shared memory for the whole decode of one codeword, so HBM/L2 traffic per iteration is
// the codeword's channel LLRs only (re-read from the caller's buffer, L2-resident while
// the slot is busy).  Thread (c, r) of the CTA owns row r of every block row (the Z checks
// of a QC block row touch disjoint variables) and column r of every block column of slot c.
//
// One round of the CTA (Sec. II two-phase message passing, Algorithm 1 loop order):
//   check-node phase   every busy slot: Q = APP - R, R' from the phi rule (k_flood_cn's
//                      arithmetic), written in place; the parity of the hard decisions
//                      (APP sign bits) over each check marks a slot whose previous
//                      iteration left an unsatisfied check
//   barrier
//   decision           a slot with >= 1 iteration done and no unsatisfied check has
//                      converged: its APP (from that iteration) is final
//   variable-node phase other busy slots: APP = L + sum of the new R (column order = block
//                      row order, deterministic); a slot reaching max_iter is final
//   output             final slots write bits / APP / iteration count; one thread per slot
//                      takes the next codeword index from the global work counter
//   barrier
//   refill             a slot given a new codeword loads APP = L and clears its R
//   barrier (with the CTA-wide "any slot busy" vote)
// Codewords therefore leave as soon as they converge and free slots are refilled at once:
// early exit saves whole rounds of work instead of idling lanes of a tile.
#include "ldpc_internal.h"

namespace ldpc {

// phi in the two specialised forms of the streaming kernels (see flood_kernels.cu).
__device__ __forceinline__ float s_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float s_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float s_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kSLog2e = 1.4426950408889634f;
constexpr float kSLn2 = 0.6931471805599453f;

__device__ __forceinline__ float s_psi_in(float x)
{
    const float t = s_ex2(-x * kSLog2e);
    const float big = t * fmaf(t * t, (2.0f / 3.0f) * kSLog2e, 2.0f * kSLog2e);
    const float mid = s_lg2((1.0f + t) * s_rcp(1.0f - t));
    return x > 3.0f ? big : mid;
}

__device__ __forceinline__ float s_phi_out(float s2)
{
    const float t = s_ex2(-s2);
    const float S = s2 * kSLn2;
    const float den = S < 0.0625f ? S * fmaf(S, fmaf(S, 1.0f / 6.0f, -0.5f), 1.0f) : 1.0f - t;
    return s_lg2((1.0f + t) * s_rcp(den)) * kSLn2;
}

template <typename T>
__device__ __forceinline__ float msg_ld(const T *p);
template <>
__device__ __forceinline__ float msg_ld<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float msg_ld<__half>(const __half *p) { return __half2float(*p); }
template <typename T>
__device__ __forceinline__ void msg_st(T *p, float v);
template <>
__device__ __forceinline__ void msg_st<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void msg_st<__half>(__half *p, float v) { *p = __float2half_rn(v); }

struct SlotArgs {
    const float *llr;
    int64_t n_cw;
    int C;             // slots per CTA
    int strideA;       // floats per slot APP row (N rounded up)
    int strideR;       // messages per slot R row (E rounded up)
    int max_iter, early_exit;
    float X;
    uint8_t *bits;
    int32_t *iters;
    float *app_out;
    unsigned long long *next;  // work counter, zero at launch
};

// shared-memory footprint: tables + per-slot APP and R + slot bookkeeping
__host__ __device__ inline size_t slot_tables_bytes(const CodeDev &h)
{
    return (size_t)(2 * h.nnz + h.mb + 1 + h.nb + 1) * sizeof(int32_t);
}

template <int DMAX, typename MsgT>
__global__ void __launch_bounds__(1024, 1) k_flood_slots(const CodeDev *__restrict__ cd, SlotArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = cd->N, Z = cd->Z, mb = cd->mb, nb = cd->nb, nnz = cd->nnz;
    const int C = a.C;
    float *APPs = reinterpret_cast<float *>(smem);
    MsgT *Rs = reinterpret_cast<MsgT *>(APPs + (size_t)C * a.strideA);
    int32_t *t_ent = reinterpret_cast<int32_t *>(Rs + (size_t)C * a.strideR);
    int32_t *t_colent = t_ent + nnz;
    int32_t *t_rowptr = t_colent + nnz;
    int32_t *t_colptr = t_rowptr + mb + 1;
    int32_t *bad = t_colptr + nb + 1;     // [C] an unsatisfied check was seen this round
    int64_t *fresh = reinterpret_cast<int64_t *>(((uintptr_t)(bad + C) + 7) & ~(uintptr_t)7);  // [C] next codeword

    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < nnz; i += nth) {
        t_ent[i] = cd->ent[i];
        t_colent[i] = cd->colent[i];
    }
    for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
    for (int i = tid; i <= nb; i += nth) t_colptr[i] = cd->colptr[i];
    const int c = tid / Z, r = tid - (tid / Z) * Z;
    const bool mine = c < C;
    if (mine && r == 0) {
        const unsigned long long k = atomicAdd(a.next, 1ull);
        fresh[c] = k < (unsigned long long)a.n_cw ? (int64_t)k : -1;
        bad[c] = 0;
    }
    __syncthreads();

    float *A = APPs + (size_t)(mine ? c : 0) * a.strideA;
    MsgT *Rc = Rs + (size_t)(mine ? c : 0) * a.strideR;
    const float X = a.X, Xb = a.X * kSLog2e;
    constexpr uint32_t kSign = 0x80000000u;
    int64_t cw = -1;  // codeword in this thread's slot (identical across the slot's threads)
    int t = 0;        // iterations completed on it

    // load a new codeword into this thread's columns: APP = L (+0 for -0), R = 0
    auto refill = [&](int64_t k) {
        const float *Lr = a.llr + k * N;
        for (int j0 = 0; j0 < nb; j0 += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (j0 + u < nb) v[u] = __ldg(Lr + (j0 + u) * Z + r);
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (j0 + u < nb) A[(j0 + u) * Z + r] = v[u] + 0.0f;
        }
        for (int b = 0; b < nnz; b++) msg_st<MsgT>(Rc + b * Z + r, 0.0f);
    };

    if (mine) {
        cw = fresh[c];
        if (cw >= 0) refill(cw);
    }
    if (!__syncthreads_or(mine && cw >= 0)) return;

    for (;;) {
        const bool busy = mine && cw >= 0;
        // ---------------- check-node phase
        if (busy) {
            uint32_t parity_bad = 0;
            for (int l = 0; l < mb; l++) {
                const int b0 = t_rowptr[l], dc = t_rowptr[l + 1] - b0;
                float av[DMAX];
                float S = 0.0f, amax = 0.0f;
                uint32_t sg = 0, par = 0;
#pragma unroll
                for (int k = 0; k < DMAX; k++) {
                    if (k < dc) {
                        const int ent = t_ent[b0 + k];
                        int x = r + (ent & 0xffff);
                        x -= (x >= Z) ? Z : 0;
                        const float ap = A[(ent >> 16) * Z + x];
                        const float q = ap - msg_ld<MsgT>(Rc + (b0 + k) * Z + r);
                        par ^= __float_as_uint(ap);
                        const float mag = fminf(s_psi_in(fminf(fabsf(q), X)), Xb);
                        S += mag;
                        amax = fmaxf(amax, mag);
                        const uint32_t qs = __float_as_uint(q) & kSign;
                        sg ^= qs;
                        av[k] = __uint_as_float(__float_as_uint(mag) | qs);
                    }
                }
                float Sx = 0.0f;
#pragma unroll
                for (int k = 0; k < DMAX; k++)
                    if (k < dc) Sx += (fabsf(av[k]) == amax) ? 0.0f : fabsf(av[k]);
                const float sx = (amax > 0.5f * S) ? Sx : S - amax;
#pragma unroll
                for (int k = 0; k < DMAX; k++) {
                    if (k < dc) {
                        const float ak = fabsf(av[k]);
                        const float ex = (ak == amax) ? sx : S - ak;
                        const float mag = fminf(s_phi_out(ex), X);
                        const float rn = __uint_as_float(__float_as_uint(mag) | ((__float_as_uint(av[k]) ^ sg) & kSign));
                        msg_st<MsgT>(Rc + (b0 + k) * Z + r, rn);
                    }
                }
                parity_bad |= par;
            }
            if (parity_bad & kSign) bad[c] = 1;
        }
        __syncthreads();

        // ---------------- decision, variable-node phase, output
        bool done = false;
        if (busy) {
            const bool converged = t >= 1 && a.early_exit && bad[c] == 0;
            if (!converged) {
                const float *Lr = a.llr + cw * N;
                for (int j0 = 0; j0 < nb; j0 += 8) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        if (j0 + u < nb) v[u] = __ldg(Lr + (j0 + u) * Z + r);
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int j = j0 + u;
                        if (j < nb) {
                            float s = v[u];
                            const int i1 = t_colptr[j + 1];
                            for (int i = t_colptr[j]; i < i1; i++) {
                                const int ce = t_colent[i];
                                int rr = r - (ce & 0xffff);
                                rr += (rr < 0) ? Z : 0;
                                s += msg_ld<MsgT>(Rc + (ce >> 16) * Z + rr);
                            }
                            A[j * Z + r] = s + 0.0f;  // -0 -> +0: the sign bit is the hard decision
                        }
                    }
                }
                t++;
            }
            done = converged || t >= a.max_iter;
            if (done) {
                uint8_t *Bo = a.bits + cw * N;
                float *Ao = a.app_out ? a.app_out + cw * N : nullptr;
                for (int j = 0; j < nb; j++) {
                    const float v = A[j * Z + r];
                    Bo[j * Z + r] = v < 0.0f ? 1 : 0;
                    if (Ao) Ao[j * Z + r] = v;
                }
                if (r == 0) {
                    a.iters[cw] = t;
                    const unsigned long long k = atomicAdd(a.next, 1ull);
                    fresh[c] = k < (unsigned long long)a.n_cw ? (int64_t)k : -1;
                }
            }
        }
        __syncthreads();

        // ---------------- refill finished slots
        if (busy) {
            if (r == 0) bad[c] = 0;
            if (done) {
                cw = fresh[c];
                t = 0;
                if (cw >= 0) refill(cw);
            }
        }
        if (!__syncthreads_or(mine && cw >= 0)) break;
    }
}

// ------------------------------------------------------------------ host side

static int g_sm_count[64];

static int sm_count()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    if (!g_sm_count[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sm_count[dev] = n > 0 ? n : 1;
    }
    return g_sm_count[dev];
}

static int max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 227 * 1024;
}

static size_t slot_bytes(const CodeDev &h, int msg)
{
    const size_t sa = (size_t)((h.N + 3) & ~3) * sizeof(float);
    const size_t sr = (size_t)((h.E + 7) & ~7) * (msg == LDPC_MSG_F16 ? sizeof(__half) : sizeof(float));
    return sa + sr + sizeof(int32_t) + sizeof(int64_t);
}

static size_t slots_smem(const CodeDev &h, int msg, int C)
{
    return (size_t)C * slot_bytes(h, msg) + slot_tables_bytes(h) + 64;
}

// slots per CTA (0 if one slot does not fit on chip)
int slots_per_cta(const CodeDev &h, int msg, size_t smem_limit)
{
    if (h.dc_max > 32) return 0;
    int C = (int)(1024 / h.Z);
    while (C > 0 && slots_smem(h, msg, C) > smem_limit) C--;
    return C;
}

int slots_supported(const CodeDev &h, int msg) { return slots_per_cta(h, msg, 227 * 1024) > 0; }

template <int DMAX, typename MsgT>
static cudaError_t launch_slots(const CodeDev &h, const CodeDev *d, SlotArgs a, cudaStream_t s)
{
    const size_t sm = slots_smem(h, sizeof(MsgT) == 2 ? LDPC_MSG_F16 : LDPC_MSG_F32, a.C);
    cudaError_t e = cudaFuncSetAttribute(k_flood_slots<DMAX, MsgT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    const int threads = ((a.C * h.Z + 31) / 32) * 32;
    int64_t ctas = sm_count();
    const int64_t need = (a.n_cw + a.C - 1) / a.C;
    if (need < ctas) ctas = need;
    LaunchScope ls(F_SLOTS, s);
    k_flood_slots<DMAX, MsgT><<<(unsigned)ctas, threads, sm, s>>>(d, a);
    return cudaGetLastError();
}

cudaError_t slots_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const float *llr,
                         int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, void *counter, cudaStream_t s)
{
    const bool f16 = p.msg == LDPC_MSG_F16;
    SlotArgs a;
    a.llr = llr;
    a.n_cw = n_cw;
    a.C = slots_per_cta(h, p.msg, (size_t)max_smem_optin());
    if (a.C < 1) return cudaErrorInvalidValue;
    a.strideA = (h.N + 3) & ~3;
    a.strideR = (h.E + 7) & ~7;
    a.max_iter = p.max_iter;
    a.early_exit = p.early_exit;
    a.X = p.phi_clamp;
    a.bits = bits;
    a.iters = iters;
    a.app_out = app_out;
    a.next = static_cast<unsigned long long *>(counter);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (h.dc_max <= 8) return f16 ? launch_slots<8, __half>(h, d, a, s) : launch_slots<8, float>(h, d, a, s);
    if (h.dc_max <= 16) return f16 ? launch_slots<16, __half>(h, d, a, s) : launch_slots<16, float>(h, d, a, s);
    return f16 ? launch_slots<32, __half>(h, d, a, s) : launch_slots<32, float>(h, d, a, s);
}

}  // namespace ldpc
