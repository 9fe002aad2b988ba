// Device code shared by the decoders that keep a codeword on chip (flooding slots, two-SM
// clusters, layered sum-product): the check rule in the product (tanh) domain, shared-memory
// message access for one or two codewords per thread, and the degree-dispatched check-node
// update of one check row.
#pragma once

#include "ldpc_internal.h"

namespace ldpc {

// The approximate base-2 exponential and logarithm of the special-function units.
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
constexpr float kSLog2e = 1.4426950408889634f;
constexpr float kSLn2 = 0.6931471805599453f;

// phi(X) log2 e, the lower end [phi(X), X] of the clamp of |Q| in base-2 units (once per
// kernel): log2((1 + t)/(1 - t)) with t = e^-X, as two logarithms of opposite sign below
// X = 3 and from the series 2t + 2t^3/3 (relative accuracy) above.
__device__ __forceinline__ float s_phi_b2(float X)
{
    const float t = s_ex2(-X * kSLog2e);
    return X > 3.0f ? t * fmaf(t * t, (2.0f / 3.0f) * kSLog2e, 2.0f * kSLog2e) : s_lg2(1.0f + t) - s_lg2(1.0f - t);
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

// Edge descriptors of one check row (built once per code when a CTA loads its tables): for
// edge k of block b = (row l, column j, shift s), .x = byte offset of the posterior
// (j*Z + s) and .y of the message (b*Z + s), both scaled by the element size and V, and
// .z = Z - s.  Row r of the block row reaches variable position (r + s) mod Z, so the
// thread's offsets are .x and .y from its own bases (position r), less one block (ZA, ZR
// bytes) when r >= .z.
struct EdgeRef {
    int oa, orr;
};
__device__ __forceinline__ EdgeRef edge_ref(const int4 d, int r, int ZA, int ZR)
{
    const bool w = r >= d.z;
    return {d.x - (w ? ZA : 0), d.y - (w ? ZR : 0)};
}
template <typename T>
__device__ __forceinline__ const T *at(const char *base, int off) { return reinterpret_cast<const T *>(base + off); }
template <typename T>
__device__ __forceinline__ T *at(char *base, int off) { return reinterpret_cast<T *>(base + off); }

// Two floats as the operand of the packed FP32x2 instructions (FFMA2, FMUL2, FADD2).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// The check rule of the sum-product algorithm,
//   R'_k = prod_{j != k} sgn Q_j * min(X, phi(sum_{j != k} phi(a_j))),  a_j = |Q_j| clamped to [phi(X), X],
// in the product (tanh) domain.  With d_j = e^-a_j, tanh(a_j / 2) = (1 - d_j) / (1 + d_j), and
// the exclusive product P_k of the other edges' tanh gives R_k = ln((1 + P_k) / (1 - P_k)),
// which is phi(sum_{j != k} phi(a_j)) exactly (phi(x) = -ln tanh(x / 2) is its own inverse).
// With B = prod (1 + d_j) and A = prod (1 - d_j), the pair alpha = (B + A) / 2,
// beta = (B - A) / 2 gives (1 + P) / (1 - P) = alpha / beta, and one more factor d maps it
// to (alpha + d beta, beta + d alpha): every term is non-negative, so neither 1 - P nor the
// exclusion of edge k cancels (the exclusion combines prefix and suffix pairs as the product
// of the two maps).  Per edge this is one ex2 (of |Q|) and two lg2 (of alpha and beta).
// The clamp of a_j to [phi(X), X] is a clamp of the ex2 argument to [-Xb, -Pb]
// (Xb = X log2 e, Pb = phi(X) log2 e); the clamp min(X, .) of the result never binds, as
// phi(sum_{j != k} phi(a_j)) <= min_{j != k} a_j <= X, so it is not applied.
// B2: Q and R in base-2 units (LLR x log2 e), where neither the ex2 argument nor the lg2
// difference needs a scaling multiply; else natural units (FP16 messages, whose stored value
// is the natural one rounded to binary16).
template <bool B2>
__device__ __forceinline__ float tanh_d(float q, float Xb, float Pb)
{
    return s_ex2(fminf(fmaxf(B2 ? -fabsf(q) : fabsf(q) * -kSLog2e, -Xb), -Pb));
}
template <bool B2>
__device__ __forceinline__ float tanh_mag(float al, float be)
{
    const float l = s_lg2(al) - s_lg2(be);
    return B2 ? l : l * kSLn2;
}

// Rows up to degree 8, one codeword per thread: d and the sign held per edge.
__device__ __forceinline__ void tanh_combine(float pa, float pb, float sa, float sb, float &al, float &be)
{
    al = fmaf(pb, sb, pa * sa);
    be = fmaf(pb, sa, pa * sb);
}

template <int D, bool EXACT, bool B2, typename MsgT>
__device__ __forceinline__ void slot_check_tanh(int dc, const int4 *__restrict__ ed, const char *Ar, char *Rr, int r,
                                                int ZA, int ZR, float Xb, float Pb, uint32_t (&pbad)[1])
{
    constexpr uint32_t kSign = 0x80000000u;
    float d[D];
    uint32_t qs[D];
    int xo[D];
    uint32_t sg = 0, par = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        d[k] = 0.0f;  // a missing edge (k >= dc) is the identity map
        qs[k] = 0;
        xo[k] = 0;
        if (EXACT || k < dc) {
            const EdgeRef e = edge_ref(ed[k], r, ZA, ZR);
            xo[k] = e.orr;
            float ap[1], rv[1];
            SMsg<float, 1>::ld(at<float>(Ar, e.oa), ap);
            SMsg<MsgT, 1>::ld(at<MsgT>(Rr, e.orr), rv);
            const float q = B2 ? fmaf(ap[0], kSLog2e, -rv[0]) : ap[0] - rv[0];
            par ^= __float_as_uint(ap[0]);
            qs[k] = __float_as_uint(q) & kSign;
            sg ^= qs[k];
            d[k] = tanh_d<B2>(q, Xb, Pb);
        }
    }
    // suffix maps of edges k..D-1 applied to (1, 0)
    float sa[D + 1], sb[D + 1];
    sa[D] = 1.0f;
    sb[D] = 0.0f;
    sa[D - 1] = 1.0f;
    sb[D - 1] = d[D - 1];
#pragma unroll
    for (int k = D - 2; k >= 1; k--) {
        sa[k] = fmaf(d[k], sb[k + 1], sa[k + 1]);
        sb[k] = fmaf(d[k], sa[k + 1], sb[k + 1]);
    }
    float pa = 1.0f, pb = 0.0f;
#pragma unroll
    for (int k = 0; k < D; k++) {
        float al, be;
        if (k == 0) {
            al = sa[1];
            be = sb[1];
        } else if (k == D - 1) {
            al = pa;
            be = pb;
        } else {
            tanh_combine(pa, pb, sa[k + 1], sb[k + 1], al, be);
        }
        if (EXACT || k < dc) {
            float out[1] = {__uint_as_float(__float_as_uint(tanh_mag<B2>(al, be)) | (qs[k] ^ sg))};
            SMsg<MsgT, 1>::st(at<MsgT>(Rr, xo[k]), out);
        }
        if (k == 0) {
            pb = d[0];
        } else if (k < D - 1) {
            const float t = fmaf(d[k], pb, pa);
            pb = fmaf(d[k], pa, pb);
            pa = t;
        }
    }
    pbad[0] |= par;
}

// Two codewords per thread: the maps' multiplies and FMAs issue as packed pairs.
__device__ __forceinline__ void tanh_combine2(float2 pa, float2 pb, float2 sa, float2 sb, float2 &al, float2 &be)
{
    al = __ffma2_rn(pb, sb, __fmul2_rn(pa, sa));
    be = __ffma2_rn(pb, sa, __fmul2_rn(pa, sb));
}

template <int D, bool EXACT, bool B2, typename MsgT>
__device__ __forceinline__ void slot_check_tanh_pair(int dc, const int4 *__restrict__ ed, const char *Ar, char *Rr,
                                                     int r, int ZA, int ZR, float Xb, float Pb,
                                                     uint32_t (&pbad)[2])
{
    constexpr uint32_t kSign = 0x80000000u;
    float2 d[D];
    uint32_t qs0[D], qs1[D];
    int xo[D];
    uint32_t sg0 = 0, sg1 = 0, par0 = 0, par1 = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        d[k] = f2(0.0f, 0.0f);
        qs0[k] = qs1[k] = 0;
        xo[k] = 0;
        if (EXACT || k < dc) {
            const EdgeRef e = edge_ref(ed[k], r, ZA, ZR);
            xo[k] = e.orr;
            float ap[2], rv[2];
            SMsg<float, 2>::ld(at<float>(Ar, e.oa), ap);
            SMsg<MsgT, 2>::ld(at<MsgT>(Rr, e.orr), rv);
            const float2 q = B2 ? __ffma2_rn(f2(ap[0], ap[1]), f2(kSLog2e, kSLog2e), f2(-rv[0], -rv[1]))
                                : __ffma2_rn(f2(rv[0], rv[1]), f2(-1.0f, -1.0f), f2(ap[0], ap[1]));
            par0 ^= __float_as_uint(ap[0]);
            par1 ^= __float_as_uint(ap[1]);
            qs0[k] = __float_as_uint(q.x) & kSign;
            qs1[k] = __float_as_uint(q.y) & kSign;
            sg0 ^= qs0[k];
            sg1 ^= qs1[k];
            d[k] = f2(tanh_d<B2>(q.x, Xb, Pb), tanh_d<B2>(q.y, Xb, Pb));
        }
    }
    float2 sa[D + 1], sb[D + 1];
    sa[D] = f2(1.0f, 1.0f);
    sb[D] = f2(0.0f, 0.0f);
    sa[D - 1] = f2(1.0f, 1.0f);
    sb[D - 1] = d[D - 1];
#pragma unroll
    for (int k = D - 2; k >= 1; k--) {
        sa[k] = __ffma2_rn(d[k], sb[k + 1], sa[k + 1]);
        sb[k] = __ffma2_rn(d[k], sa[k + 1], sb[k + 1]);
    }
    float2 pa = f2(1.0f, 1.0f), pb = f2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < D; k++) {
        float2 al, be;
        if (k == 0) {
            al = sa[1];
            be = sb[1];
        } else if (k == D - 1) {
            al = pa;
            be = pb;
        } else {
            tanh_combine2(pa, pb, sa[k + 1], sb[k + 1], al, be);
        }
        if (EXACT || k < dc) {
            float2 mag = __fadd2_rn(f2(s_lg2(al.x), s_lg2(al.y)), f2(-s_lg2(be.x), -s_lg2(be.y)));
            if constexpr (!B2) mag = __fmul2_rn(mag, f2(kSLn2, kSLn2));
            float out[2] = {__uint_as_float(__float_as_uint(mag.x) | (qs0[k] ^ sg0)),
                            __uint_as_float(__float_as_uint(mag.y) | (qs1[k] ^ sg1))};
            SMsg<MsgT, 2>::st(at<MsgT>(Rr, xo[k]), out);
        }
        if (k == 0) {
            pb = d[0];
        } else if (k < D - 1) {
            const float2 t = __ffma2_rn(d[k], pb, pa);
            pb = __ffma2_rn(d[k], pa, pb);
            pa = t;
        }
    }
    pbad[0] |= par0;
    pbad[1] |= par1;
}

// The product-domain rule for a row of degree dc <= D with D > 8, in groups of 8 edges,
// holding no per-edge state between its two passes (the registers of D pairs would spill):
//   pass 1 forms every d_k and each group's pair (the product of its edges' maps);
//   pass 2, group by group, forms the group's d_k again, its suffix pairs, and a prefix
//   that starts from the product of the other groups' pairs.
// Every term stays non-negative, as in the prefix / suffix form of rows up to degree 8.
// qof(k, first) returns Q_k of edge k (`first`: pass 1, where the caller also takes what it
// needs once per edge); put(k, R, Q) writes the signed message R of edge k (Q: its Q_k).
__device__ __forceinline__ void pair_mul(float a1, float b1, float a2, float b2, float &a, float &b)
{
    a = fmaf(b1, b2, a1 * a2);
    b = fmaf(b1, a2, a1 * b2);
}

template <int D, bool B2, typename QF, typename PF>
__device__ __forceinline__ void tanh_check_wide(int dc, float Xb, float Pb, QF qof, PF put)
{
    constexpr uint32_t kSign = 0x80000000u;
    constexpr int G = (D + 7) / 8;
    float ga[G], gb[G];
    uint32_t sg = 0;
#pragma unroll
    for (int g = 0; g < G; g++) {
        ga[g] = 1.0f;
        gb[g] = 0.0f;
    }
    // the loops leave at the row's degree (a warp-uniform test) rather than predicate the
    // edges of the body past it
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (8 * g >= dc) break;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            {
                const float q = qof(k, true);
                sg ^= __float_as_uint(q);
                const float d = tanh_d<B2>(q, Xb, Pb);
                if (i == 0) {
                    gb[g] = d;
                } else {
                    const float t = fmaf(d, gb[g], ga[g]);
                    gb[g] = fmaf(d, ga[g], gb[g]);
                    ga[g] = t;
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (8 * g >= dc) break;
        // the other groups' product
        float pa = 1.0f, pb = 0.0f;
        bool first = true;
#pragma unroll
        for (int h = 0; h < G; h++) {
            if (h == g) continue;
            if (first) {
                pa = ga[h];
                pb = gb[h];
                first = false;
            } else {
                pair_mul(pa, pb, ga[h], gb[h], pa, pb);
            }
        }
        float d[8];
        uint32_t qb[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            d[i] = 0.0f;  // a missing edge is the identity map
            qb[i] = 0;
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            {
                const float q = qof(k, false);
                qb[i] = __float_as_uint(q);
                d[i] = tanh_d<B2>(q, Xb, Pb);
            }
        }
        float sa[9], sb[9];
        sa[8] = 1.0f;
        sb[8] = 0.0f;
        sa[7] = 1.0f;
        sb[7] = d[7];
#pragma unroll
        for (int i = 6; i >= 1; i--) {
            sa[i] = fmaf(d[i], sb[i + 1], sa[i + 1]);
            sb[i] = fmaf(d[i], sa[i + 1], sb[i + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            float al, be;
            if (i == 7)
                al = pa, be = pb;
            else
                pair_mul(pa, pb, sa[i + 1], sb[i + 1], al, be);
            {
                const float mag = tanh_mag<B2>(al, be);
                put(k, __uint_as_float(__float_as_uint(mag) | ((qb[i] ^ sg) & kSign)), __uint_as_float(qb[i]));
            }
            if (i < 7) {
                const float t = fmaf(d[i], pb, pa);
                pb = fmaf(d[i], pa, pb);
                pa = t;
            }
        }
    }
}

// The grouped rule holding each edge's factor between its two passes (d_k in a register,
// the sign of Q_k in d_k's own sign bit): pass 2 then needs no second load of the edge's
// operands and no second ex2.  put(k, R) writes the signed message of edge k.
template <int D, bool B2, typename QF, typename PF>
__device__ __forceinline__ void tanh_check_wide_held(int dc, float Xb, float Pb, QF qof, PF put)
{
    constexpr uint32_t kSign = 0x80000000u;
    constexpr int G = (D + 7) / 8;
    float ga[G], gb[G];
    uint32_t dq[D];  // d_k with the sign of Q_k
    uint32_t sg = 0;
#pragma unroll
    for (int g = 0; g < G; g++) {
        ga[g] = 1.0f;
        gb[g] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < D; k++) dq[k] = 0;
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (8 * g >= dc) break;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            const float q = qof(k);
            const uint32_t qs = __float_as_uint(q) & kSign;
            sg ^= qs;
            const float d = tanh_d<B2>(q, Xb, Pb);
            dq[k] = __float_as_uint(d) | qs;
            if (i == 0) {
                gb[g] = d;
            } else {
                const float t = fmaf(d, gb[g], ga[g]);
                gb[g] = fmaf(d, ga[g], gb[g]);
                ga[g] = t;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (8 * g >= dc) break;
        float pa = 1.0f, pb = 0.0f;
        bool first = true;
#pragma unroll
        for (int h = 0; h < G; h++) {
            if (h == g) continue;
            if (first) {
                pa = ga[h];
                pb = gb[h];
                first = false;
            } else {
                pair_mul(pa, pb, ga[h], gb[h], pa, pb);
            }
        }
        float d[8];
#pragma unroll
        for (int i = 0; i < 8; i++) d[i] = (8 * g + i < D) ? __uint_as_float(dq[8 * g + i] & ~kSign) : 0.0f;
        float sa[9], sb[9];
        sa[8] = 1.0f;
        sb[8] = 0.0f;
        sa[7] = 1.0f;
        sb[7] = d[7];
#pragma unroll
        for (int i = 6; i >= 1; i--) {
            sa[i] = fmaf(d[i], sb[i + 1], sa[i + 1]);
            sb[i] = fmaf(d[i], sa[i + 1], sb[i + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            float al, be;
            if (i == 7)
                al = pa, be = pb;
            else
                pair_mul(pa, pb, sa[i + 1], sb[i + 1], al, be);
            put(k, __uint_as_float(__float_as_uint(tanh_mag<B2>(al, be)) | ((dq[k] ^ sg) & kSign)));
            if (i < 7) {
                const float t = fmaf(d[i], pb, pa);
                pb = fmaf(d[i], pa, pb);
                pa = t;
            }
        }
    }
}

#ifndef LDPC_SLOTS_WIDE_HELD
#define LDPC_SLOTS_WIDE_HELD 16  // widest row body (one codeword per thread) that holds its factors
#endif

// Flooding slot decoder, one codeword per thread, rows above degree 8.
template <int D, bool B2, typename MsgT>
__device__ __forceinline__ void slot_check_tanh_wide(int dc, const int4 *__restrict__ ed, const char *Ar, char *Rr,
                                                     int r, int ZA, int ZR, float Xb, float Pb, uint32_t (&pbad)[1])
{
    uint32_t par = 0;
    auto qof = [&](int k, bool first) -> float {
        const EdgeRef e = edge_ref(ed[k], r, ZA, ZR);
        float ap[1], rv[1];
        SMsg<float, 1>::ld(at<float>(Ar, e.oa), ap);
        SMsg<MsgT, 1>::ld(at<MsgT>(Rr, e.orr), rv);
        if (first) par ^= __float_as_uint(ap[0]);
        return B2 ? fmaf(ap[0], kSLog2e, -rv[0]) : ap[0] - rv[0];
    };
    // the message offset is formed again at the store (holding it per edge costs D registers)
    auto put = [&](int k, float m, float) {
        const EdgeRef e = edge_ref(ed[k], r, ZA, ZR);
        float out[1] = {m};
        SMsg<MsgT, 1>::st(at<MsgT>(Rr, e.orr), out);
    };
    if constexpr (D <= LDPC_SLOTS_WIDE_HELD)
        tanh_check_wide_held<D, B2>(dc, Xb, Pb, [&](int k) { return qof(k, true); },
                                    [&](int k, float m) { put(k, m, 0.0f); });
    else
        tanh_check_wide<D, B2>(dc, Xb, Pb, qof, put);
    pbad[0] |= par;
}

// The grouped rule for two codewords per thread: the maps' multiplies and FMAs as packed
// pairs.  qof(k, first) returns both codewords' Q_k, put(k, R) writes both messages.
__device__ __forceinline__ void pair_mul2(float2 a1, float2 b1, float2 a2, float2 b2, float2 &a, float2 &b)
{
    a = __ffma2_rn(b1, b2, __fmul2_rn(a1, a2));
    b = __ffma2_rn(b1, a2, __fmul2_rn(a1, b2));
}

template <int D, bool B2, typename QF, typename PF>
__device__ __forceinline__ void tanh_check_wide2(int dc, float Xb, float Pb, QF qof, PF put)
{
    constexpr uint32_t kSign = 0x80000000u;
    constexpr int G = (D + 7) / 8;
    float2 ga[G], gb[G];
    uint32_t sg0 = 0, sg1 = 0;
#pragma unroll
    for (int g = 0; g < G; g++) {
        ga[g] = f2(1.0f, 1.0f);
        gb[g] = f2(0.0f, 0.0f);
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (8 * g >= dc) break;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            {
                const float2 q = qof(k, true);
                sg0 ^= __float_as_uint(q.x);
                sg1 ^= __float_as_uint(q.y);
                const float2 d = f2(tanh_d<B2>(q.x, Xb, Pb), tanh_d<B2>(q.y, Xb, Pb));
                if (i == 0) {
                    gb[g] = d;
                } else {
                    const float2 t = __ffma2_rn(d, gb[g], ga[g]);
                    gb[g] = __ffma2_rn(d, ga[g], gb[g]);
                    ga[g] = t;
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
        if (8 * g >= dc) break;
        float2 pa = f2(1.0f, 1.0f), pb = f2(0.0f, 0.0f);
        bool first = true;
#pragma unroll
        for (int h = 0; h < G; h++) {
            if (h == g) continue;
            if (first) {
                pa = ga[h];
                pb = gb[h];
                first = false;
            } else {
                pair_mul2(pa, pb, ga[h], gb[h], pa, pb);
            }
        }
        float2 d[8];
        uint32_t qb0[8], qb1[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            d[i] = f2(0.0f, 0.0f);
            qb0[i] = qb1[i] = 0;
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            {
                const float2 q = qof(k, false);
                qb0[i] = __float_as_uint(q.x);
                qb1[i] = __float_as_uint(q.y);
                d[i] = f2(tanh_d<B2>(q.x, Xb, Pb), tanh_d<B2>(q.y, Xb, Pb));
            }
        }
        float2 sa[9], sb[9];
        sa[8] = f2(1.0f, 1.0f);
        sb[8] = f2(0.0f, 0.0f);
        sa[7] = f2(1.0f, 1.0f);
        sb[7] = d[7];
#pragma unroll
        for (int i = 6; i >= 1; i--) {
            sa[i] = __ffma2_rn(d[i], sb[i + 1], sa[i + 1]);
            sb[i] = __ffma2_rn(d[i], sa[i + 1], sb[i + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = 8 * g + i;
            if (k >= D || k >= dc) break;
            float2 al, be;
            if (i == 7)
                al = pa, be = pb;
            else
                pair_mul2(pa, pb, sa[i + 1], sb[i + 1], al, be);
            {
                float2 mag = __fadd2_rn(f2(s_lg2(al.x), s_lg2(al.y)), f2(-s_lg2(be.x), -s_lg2(be.y)));
                if constexpr (!B2) mag = __fmul2_rn(mag, f2(kSLn2, kSLn2));
                put(k, f2(__uint_as_float(__float_as_uint(mag.x) | ((qb0[i] ^ sg0) & kSign)),
                          __uint_as_float(__float_as_uint(mag.y) | ((qb1[i] ^ sg1) & kSign))));
            }
            if (i < 7) {
                const float2 t = __ffma2_rn(d[i], pb, pa);
                pb = __ffma2_rn(d[i], pa, pb);
                pa = t;
            }
        }
    }
}

// Flooding slot decoder, two codewords per thread, rows above degree 8.
template <int D, bool B2, typename MsgT>
__device__ __forceinline__ void slot_check_tanh_pair_wide(int dc, const int4 *__restrict__ ed, const char *Ar,
                                                          char *Rr, int r, int ZA, int ZR, float Xb, float Pb,
                                                          uint32_t (&pbad)[2])
{
    uint32_t par0 = 0, par1 = 0;
    auto qof = [&](int k, bool first) -> float2 {
        const EdgeRef e = edge_ref(ed[k], r, ZA, ZR);
        float ap[2], rv[2];
        SMsg<float, 2>::ld(at<float>(Ar, e.oa), ap);
        SMsg<MsgT, 2>::ld(at<MsgT>(Rr, e.orr), rv);
        if (first) {
            par0 ^= __float_as_uint(ap[0]);
            par1 ^= __float_as_uint(ap[1]);
        }
        return B2 ? __ffma2_rn(f2(ap[0], ap[1]), f2(kSLog2e, kSLog2e), f2(-rv[0], -rv[1]))
                  : __ffma2_rn(f2(rv[0], rv[1]), f2(-1.0f, -1.0f), f2(ap[0], ap[1]));
    };
    auto put = [&](int k, float2 m) {
        const EdgeRef e = edge_ref(ed[k], r, ZA, ZR);
        float out[2] = {m.x, m.y};
        SMsg<MsgT, 2>::st(at<MsgT>(Rr, e.orr), out);
    };
    tanh_check_wide2<D, B2>(dc, Xb, Pb, qof, put);
    pbad[0] |= par0;
    pbad[1] |= par1;
}

// Whether the flooding slot decoder stores FP32 messages in base-2 units (R log2 e) while
// APP stays in natural units: Q in base-2 units is then one FMA (APP log2 e - R), the ex2
// argument and the lg2 difference need no scaling multiply, and the variable-node sum
// adds R ln 2 with an FMA; two multiplies fewer per edge update at no other cost.  (FP16
// messages stay natural: the stored binary16 value is the natural one rounded.)
#ifndef LDPC_SLOTS_B2
#define LDPC_SLOTS_B2 1
#endif
template <typename MsgT>
constexpr bool kSlotB2 = LDPC_SLOTS_B2 && sizeof(MsgT) == 4;

// One check of row r for V slots (V codewords per thread): Q = APP - R over its edges, the
// check rule, messages written in place (at the variable's position), parity of the APP sign
// bits accumulated in pbad.
template <int D, bool EXACT, int V, typename MsgT>
__device__ __forceinline__ void slot_check_v(int dc, const int4 *__restrict__ ed, const char *Ar, char *Rr, int r,
                                             int ZA, int ZR, float Xb, float Pb, uint32_t (&pbad)[V])
{
    constexpr bool B2 = kSlotB2<MsgT>;
    if constexpr (D <= 8 && V == 1)
        slot_check_tanh<D, EXACT, B2, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
    else if constexpr (D <= 8)
        slot_check_tanh_pair<D, EXACT, B2, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
    else if constexpr (V == 1)
        slot_check_tanh_wide<D, B2, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
    else
        slot_check_tanh_pair_wide<D, B2, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
}

template <int D, int DMAX, int V, typename MsgT>
__device__ __forceinline__ void slot_check_dispatch(int dc, const int4 *__restrict__ ed, const char *Ar, char *Rr,
                                                    int r, int ZA, int ZR, float Xb, float Pb, uint32_t (&pbad)[V])
{
    if constexpr (D >= DMAX) {
        slot_check_v<DMAX, false, V, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
    } else if constexpr (D <= 8) {
        if (dc == D)
            slot_check_v<D, true, V, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
        else
            slot_check_dispatch<next_degree(D), DMAX, V, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
    } else {
        if (dc <= D)
            slot_check_v<D, false, V, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
        else
            slot_check_dispatch<next_degree(D), DMAX, V, MsgT>(dc, ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
    }
}

template <int V>
constexpr int slot_threads_max() { return V == 2 ? 512 : 640; }

}  // namespace ldpc
