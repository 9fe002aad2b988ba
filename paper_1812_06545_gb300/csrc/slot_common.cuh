// Device code shared by the slot decoders: phi in the two specialised forms, shared-memory
// message access for one or two codewords per thread, and the degree-dispatched
// check-node update of one check row.
#pragma once

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

template <int V>
constexpr int slot_threads_max() { return V == 2 ? 512 : 640; }

}  // namespace ldpc
