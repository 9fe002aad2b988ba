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

// V consecutive slots share each shared-memory element group: APP and R are laid out
// [slot group][node][V], so one 64-bit (V = 2) shared access serves both codewords of a
// thread and the index arithmetic of an edge is paid once for V codewords.
template <typename T, int V>
struct SMsg;
template <>
struct SMsg<float, 1> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[1]) { x[0] = *p; }
    static __device__ __forceinline__ void st(float *p, const float (&x)[1]) { *p = x[0]; }
};
template <>
struct SMsg<float, 2> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[2])
    {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        x[0] = v.x;
        x[1] = v.y;
    }
    static __device__ __forceinline__ void st(float *p, const float (&x)[2])
    {
        *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
    }
};
template <>
struct SMsg<__half, 1> {
    static __device__ __forceinline__ void ld(const __half *p, float (&x)[1]) { x[0] = __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, const float (&x)[1]) { *p = __float2half_rn(x[0]); }
};
template <>
struct SMsg<__half, 2> {
    static __device__ __forceinline__ void ld(const __half *p, float (&x)[2])
    {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        x[0] = v.x;
        x[1] = v.y;
    }
    static __device__ __forceinline__ void st(__half *p, const float (&x)[2])
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(x[0], x[1]);
    }
};

// Degree dispatch: the checks of one block row all have the same degree, so every lane of
// a warp takes the same branch.  Degrees up to 8 get an exact, guard-free body; larger
// degrees share buckets of four (edges past the degree are skipped under a uniform guard).
__host__ __device__ constexpr int next_degree(int d) { return d < 8 ? d + 1 : d + 4; }

// One check of row r for V slots: Q = APP - R over its edges, phi rule, messages written
// in place (at the variable's position), parity of the APP sign bits accumulated in pbad.
template <int D, bool EXACT, int V, typename MsgT>
__device__ __forceinline__ void slot_check(int dc, const int32_t *__restrict__ ent, int bZ, const float *A, MsgT *Rc,
                                           int r, int Z, float X, float Xb, uint32_t (&pbad)[V])
{
    constexpr uint32_t kSign = 0x80000000u;
    float av[D][V];
    int xo[D];
    uint32_t sg[V], par[V];
#pragma unroll
    for (int v = 0; v < V; v++) sg[v] = par[v] = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        if (EXACT || k < dc) {
            const int e = ent[k];
            int x = r + (e >> 16);
            x -= (x >= Z) ? Z : 0;
            xo[k] = x;
            float ap[V], rv[V];
            SMsg<float, V>::ld(A + ((e & 0xffff) + x) * V, ap);
            SMsg<MsgT, V>::ld(Rc + (bZ + k * Z + x) * V, rv);
#pragma unroll
            for (int v = 0; v < V; v++) {
                const float q = ap[v] - rv[v];
                par[v] ^= __float_as_uint(ap[v]);
                const float mag = fminf(s_psi_in(fminf(fabsf(q), X)), Xb);
                const uint32_t qs = __float_as_uint(q) & kSign;
                sg[v] ^= qs;
                av[k][v] = __uint_as_float(__float_as_uint(mag) | qs);
            }
        }
    }
    // exclusive sums from suffix and prefix sums of |a| (no cancellation)
    float sf[D + 1][V];
#pragma unroll
    for (int v = 0; v < V; v++) sf[D][v] = 0.0f;
#pragma unroll
    for (int k = D - 1; k >= 0; k--)
#pragma unroll
        for (int v = 0; v < V; v++) sf[k][v] = (EXACT || k < dc) ? sf[k + 1][v] + fabsf(av[k][v]) : 0.0f;
    float pre[V];
#pragma unroll
    for (int v = 0; v < V; v++) pre[v] = 0.0f;
#pragma unroll
    for (int k = 0; k < D; k++) {
        if (EXACT || k < dc) {
            float out[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const float mag = fminf(s_phi_out(pre[v] + sf[k + 1][v]), X);
                pre[v] += fabsf(av[k][v]);
                out[v] = __uint_as_float(__float_as_uint(mag) | ((__float_as_uint(av[k][v]) ^ sg[v]) & kSign));
            }
            SMsg<MsgT, V>::st(Rc + (bZ + k * Z + xo[k]) * V, out);
        }
    }
#pragma unroll
    for (int v = 0; v < V; v++) pbad[v] |= par[v];
}

template <int D, int DMAX, int V, typename MsgT>
__device__ __forceinline__ void slot_check_dispatch(int dc, const int32_t *__restrict__ ent, int bZ, const float *A,
                                                    MsgT *Rc, int r, int Z, float X, float Xb, uint32_t (&pbad)[V])
{
    if constexpr (D >= DMAX) {
        slot_check<DMAX, false, V, MsgT>(dc, ent, bZ, A, Rc, r, Z, X, Xb, pbad);
    } else if constexpr (D <= 8) {
        if (dc == D)
            slot_check<D, true, V, MsgT>(dc, ent, bZ, A, Rc, r, Z, X, Xb, pbad);
        else
            slot_check_dispatch<next_degree(D), DMAX, V, MsgT>(dc, ent, bZ, A, Rc, r, Z, X, Xb, pbad);
    } else {
        if (dc <= D)
            slot_check<D, false, V, MsgT>(dc, ent, bZ, A, Rc, r, Z, X, Xb, pbad);
        else
            slot_check_dispatch<next_degree(D), DMAX, V, MsgT>(dc, ent, bZ, A, Rc, r, Z, X, Xb, pbad);
    }
}

struct SlotArgs {
    const float *llr;
    int64_t n_cw;
    int C;             // slots per CTA (a multiple of V)
    int strideA;       // nodes per slot-group APP block (N rounded up)
    int strideR;       // edges per slot-group R block (E rounded up)
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

template <int V>
constexpr int slot_threads_max() { return V == 2 ? 512 : 640; }

template <int DMAX, int V, typename MsgT>
__global__ void __launch_bounds__(slot_threads_max<V>(), 1) k_flood_slots(const CodeDev *__restrict__ cd, SlotArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = cd->N, Z = cd->Z, mb = cd->mb, nb = cd->nb, nnz = cd->nnz;
    const int C = a.C, G = a.C / V;
    float *APPs = reinterpret_cast<float *>(smem);
    MsgT *Rs = reinterpret_cast<MsgT *>(APPs + (size_t)G * a.strideA * V);
    int32_t *t_ent = reinterpret_cast<int32_t *>(Rs + (size_t)G * a.strideR * V);
    int32_t *t_colent = t_ent + nnz;
    int32_t *t_rowptr = t_colent + nnz;
    int32_t *t_colptr = t_rowptr + mb + 1;
    int32_t *bad = t_colptr + nb + 1;     // [C] an unsatisfied check was seen this round
    int64_t *fresh = reinterpret_cast<int64_t *>(((uintptr_t)(bad + C) + 7) & ~(uintptr_t)7);  // [C] next codeword

    // tables, pre-scaled: t_ent[b] = (s << 16) | (j * Z) for block b; t_colent[i] = b * Z
    // for the i-th block of the column lists.  Messages are stored at the variable's
    // position inside its block: edge (b, r) of check row r lives at b * Z + (r + s) mod Z,
    // so the check-node phase computes the wrap once for both addresses and the
    // variable-node phase, summing column position r of block column j, reads b * Z + r.
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < nnz; i += nth) {
        const int e = cd->ent[i];
        t_ent[i] = ((e & 0xffff) << 16) | ((e >> 16) * Z);
        t_colent[i] = (cd->colent[i] >> 16) * Z;
    }
    for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
    for (int i = tid; i <= nb; i += nth) t_colptr[i] = cd->colptr[i];
    const int g = tid / Z, r = tid - (tid / Z) * Z;
    const bool mine = g < G;
    if (mine && r == 0) {
#pragma unroll
        for (int v = 0; v < V; v++) {
            const unsigned long long k = atomicAdd(a.next, 1ull);
            fresh[g * V + v] = k < (unsigned long long)a.n_cw ? (int64_t)k : -1;
            bad[g * V + v] = 0;
        }
    }
    __syncthreads();

    float *A = APPs + (size_t)(mine ? g : 0) * a.strideA * V;
    MsgT *Rc = Rs + (size_t)(mine ? g : 0) * a.strideR * V;
    const float X = a.X, Xb = a.X * kSLog2e;
    constexpr uint32_t kSign = 0x80000000u;
    int64_t cw[V];  // codeword in each of this thread's slots (identical across the slot group's threads)
    int t[V];       // iterations completed on it

    // load a new codeword into slot v, this thread's columns: APP = L (+0 for -0), R = 0
    auto refill = [&](int v, int64_t k) {
        const float *Lr = a.llr + k * N;
        for (int j0 = 0; j0 < nb; j0 += 8) {
            float x[8];
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (j0 + u < nb) x[u] = __ldg(Lr + (j0 + u) * Z + r);
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (j0 + u < nb) A[((j0 + u) * Z + r) * V + v] = x[u] + 0.0f;
        }
        for (int b = 0; b < nnz; b++) {
            if constexpr (sizeof(MsgT) == 2)
                Rc[(b * Z + r) * V + v] = __float2half_rn(0.0f);
            else
                Rc[(b * Z + r) * V + v] = 0.0f;
        }
    };

    bool any = false;
#pragma unroll
    for (int v = 0; v < V; v++) {
        cw[v] = mine ? fresh[g * V + v] : -1;
        t[v] = 0;
        if (cw[v] >= 0) refill(v, cw[v]);
        any |= cw[v] >= 0;
    }
    if (!__syncthreads_or(any)) return;

    for (;;) {
        // ---------------- check-node phase: row r of every block row, all V slots at once
        if (any) {
            uint32_t pbad[V];
#pragma unroll
            for (int v = 0; v < V; v++) pbad[v] = 0;
            for (int l = 0; l < mb; l++) {
                const int b0 = t_rowptr[l], dc = t_rowptr[l + 1] - b0;
                slot_check_dispatch<2, DMAX, V, MsgT>(dc, t_ent + b0, b0 * Z, A, Rc, r, Z, X, Xb, pbad);
            }
#pragma unroll
            for (int v = 0; v < V; v++)
                if (cw[v] >= 0 && (pbad[v] & kSign)) bad[g * V + v] = 1;
        }
        __syncthreads();

        // ---------------- decision, variable-node phase, output
        bool done[V];
        if (any) {
            bool act[V];
            bool anyact = false;
#pragma unroll
            for (int v = 0; v < V; v++) {
                const bool conv = cw[v] >= 0 && t[v] >= 1 && a.early_exit && bad[g * V + v] == 0;
                act[v] = cw[v] >= 0 && !conv;
                done[v] = conv;
                anyact |= act[v];
            }
            if (anyact) {
                for (int j0 = 0; j0 < nb; j0 += 4) {
                    float lv[4][V];
#pragma unroll
                    for (int u = 0; u < 4; u++)
#pragma unroll
                        for (int v = 0; v < V; v++)
                            if (j0 + u < nb && act[v]) lv[u][v] = __ldg(a.llr + cw[v] * N + (j0 + u) * Z + r);
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int j = j0 + u;
                        if (j < nb) {
                            float sacc[V];
#pragma unroll
                            for (int v = 0; v < V; v++) sacc[v] = lv[u][v];
                            const int i1 = t_colptr[j + 1];
                            for (int i = t_colptr[j]; i < i1; i++) {
                                float rv[V];
                                SMsg<MsgT, V>::ld(Rc + (t_colent[i] + r) * V, rv);
#pragma unroll
                                for (int v = 0; v < V; v++) sacc[v] += rv[v];
                            }
#pragma unroll
                            for (int v = 0; v < V; v++)
                                if (act[v]) A[(j * Z + r) * V + v] = sacc[v] + 0.0f;  // -0 -> +0: sign bit = decision
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (act[v]) {
                    t[v]++;
                    done[v] = t[v] >= a.max_iter;
                }
                if (done[v]) {
                    uint8_t *Bo = a.bits + cw[v] * N;
                    float *Ao = a.app_out ? a.app_out + cw[v] * N : nullptr;
                    for (int j = 0; j < nb; j++) {
                        const float x = A[(j * Z + r) * V + v];
                        Bo[j * Z + r] = x < 0.0f ? 1 : 0;
                        if (Ao) Ao[j * Z + r] = x;
                    }
                    if (r == 0) {
                        a.iters[cw[v]] = t[v];
                        const unsigned long long k = atomicAdd(a.next, 1ull);
                        fresh[g * V + v] = k < (unsigned long long)a.n_cw ? (int64_t)k : -1;
                    }
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; v++) done[v] = false;
        }
        __syncthreads();

        // ---------------- refill finished slots
        any = false;
        if (mine) {
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (r == 0) bad[g * V + v] = 0;
                if (done[v]) {
                    cw[v] = fresh[g * V + v];
                    t[v] = 0;
                    if (cw[v] >= 0) refill(v, cw[v]);
                }
                any |= cw[v] >= 0;
            }
        }
        if (!__syncthreads_or(any)) break;
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

#ifndef LDPC_SLOTS_V
#define LDPC_SLOTS_V 2  // codewords per thread in the slot decoder (1 or 2)
#endif

static size_t slots_smem(const CodeDev &h, int msg, int C)
{
    return (size_t)C * slot_bytes(h, msg) + slot_tables_bytes(h) + 64;
}

// slots per CTA (0 if one slot does not fit on chip); *v gets the codewords per thread
int slots_per_cta(const CodeDev &h, int msg, size_t smem_limit, int *v = nullptr)
{
    if (h.dc_max > 32) return 0;
    // single slots: as many as fit; paired slots (two codewords per thread) when pairing
    // loses no slot
    int C1 = (int)(slot_threads_max<1>() / h.Z);
    while (C1 > 0 && slots_smem(h, msg, C1) > smem_limit) C1--;
    int C2 = (int)(slot_threads_max<2>() / h.Z) * 2;
    while (C2 > 0 && slots_smem(h, msg, C2) > smem_limit) C2--;
    C2 -= C2 % 2;
    const bool pair = LDPC_SLOTS_V == 2 && C2 >= 2 && C2 >= C1;
    if (v) *v = pair ? 2 : 1;
    return pair ? C2 : C1;
}

int slots_supported(const CodeDev &h, int msg) { return slots_per_cta(h, msg, 227 * 1024) > 0; }

template <int DMAX, int V, typename MsgT>
static cudaError_t launch_slots(const CodeDev &h, const CodeDev *d, SlotArgs a, cudaStream_t s)
{
    const size_t sm = slots_smem(h, sizeof(MsgT) == 2 ? LDPC_MSG_F16 : LDPC_MSG_F32, a.C);
    cudaError_t e = cudaFuncSetAttribute(k_flood_slots<DMAX, V, MsgT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    const int threads = ((a.C / V * h.Z + 31) / 32) * 32;
    int64_t ctas = sm_count();
    const int64_t need = (a.n_cw + a.C - 1) / a.C;
    if (need < ctas) ctas = need;
    LaunchScope ls(F_SLOTS, s);
    k_flood_slots<DMAX, V, MsgT><<<(unsigned)ctas, threads, sm, s>>>(d, a);
    return cudaGetLastError();
}

template <int DMAX, typename MsgT>
static cudaError_t launch_slots_v(const CodeDev &h, const CodeDev *d, SlotArgs a, int V, cudaStream_t s)
{
    if (V == 2) return launch_slots<DMAX, 2, MsgT>(h, d, a, s);
    return launch_slots<DMAX, 1, MsgT>(h, d, a, s);
}

cudaError_t slots_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const float *llr,
                         int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, void *counter, cudaStream_t s)
{
    const bool f16 = p.msg == LDPC_MSG_F16;
    SlotArgs a;
    a.llr = llr;
    a.n_cw = n_cw;
    int V = 1;
    a.C = slots_per_cta(h, p.msg, (size_t)max_smem_optin(), &V);
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
    if (h.dc_max <= 8) return f16 ? launch_slots_v<8, __half>(h, d, a, V, s) : launch_slots_v<8, float>(h, d, a, V, s);
    if (h.dc_max <= 16)
        return f16 ? launch_slots_v<16, __half>(h, d, a, V, s) : launch_slots_v<16, float>(h, d, a, V, s);
    return f16 ? launch_slots_v<32, __half>(h, d, a, V, s) : launch_slots_v<32, float>(h, d, a, V, s);
}

}  // namespace ldpc
