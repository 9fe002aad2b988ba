// Flooding sum-product decoding on sm_103a (Sec. II: two-phase message passing in the
// loop order of Algorithm 1 - check-node phase, variable-node phase, hard decision).
//
// State of a decode lives in HBM, interleaved by codeword (Sec. III-B): every buffer is
// [tile][node][TILE] with the TILE = 128 codewords of one node contiguous.  One warp
// owns one node of one tile; each lane owns V consecutive codewords (V = 4, 2 or 1 with
// the code's largest check degree), so each access of a node is one coalesced 128-bit
// (V = 4) load or store per lane and no cross-lane reduction is needed: the check-node
// reductions run down the check's edges inside each lane's registers.  The cyclic shift
// of a QC block is index arithmetic: edge (b, r) of block b = (l, j, s) joins check
// l*Z + r and variable j*Z + (r + s) mod Z; its message sits at edge index b*Z + r.
//
// Early exit: the check-node kernel of iteration t + 1 also forms the parity of the hard
// decisions of iteration t over each check (the syndrome) and stamps unsat[cw] = t + 1
// when a check fails; the variable-node kernel of iteration t + 1 then freezes every
// codeword no check stamped, recording done_at = t.  Warps whose codewords are all
// frozen return at once, so later launches cost little once a tile has converged.
#include <math.h>

#include "ldpc_internal.h"

namespace ldpc {

// ------------------------------------------------------------------ phi

// phi(x) = -ln tanh(x/2) = ln((1 + t)/(1 - t)) with t = e^-x, on the hardware
// approximations ex2 / lg2 (PTX *.approx.ftz.f32).  The check rule needs phi twice
// per edge with different accuracy demands, so there are two evaluations:
//
//   psi_in(x)  = phi(x) / ln 2 for the incoming |Q| (base-2 units).  Small values (large x)
//                are summed and the sum is fed back through phi, so they need RELATIVE
//                accuracy: for x > 3 the series 2 atanh(t) = 2t + 2t^3/3 + O(t^5) (t < 0.05)
//                is used; below, the closed form.  As x -> 0 the closed form overflows to
//                +inf, which the caller clamps to X / ln 2 = psi(phi(X)), the value the
//                |Q| >= phi(X) clamp of the definition gives.
//   phi_out(s) = phi(s ln 2) for the exclusive sum s (base-2 units).  The result is added to
//                the posterior, so ABSOLUTE accuracy suffices for small results; for a small
//                argument (S = s ln 2 < 1/16) 1 - e^-S loses precision, so it is taken from
//                its series S (1 - S/2 + S^2/6).  S -> 0 gives +inf, clamped to X by the caller;
//                large S underflows t to 0 and gives 0.
// Working in base-2 units removes the ln 2 / log2 e scalings between the two evaluations.
// Both are checked against the library expm1f/log1pf form and the FP64 oracle by the tests.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// ln((1 + t)/(1 - t)) = lg2(1 + t) - lg2(1 - t): two independent logarithms of opposite
// sign (no cancellation), a shorter dependency chain than a reciprocal and one logarithm.
__device__ __forceinline__ float psi_in(float x)
{
    const float t = ex2_approx(-x * kLog2e);
    const float big = t * fmaf(t * t, (2.0f / 3.0f) * kLog2e, 2.0f * kLog2e);
    const float mid = lg2_approx(1.0f + t) - lg2_approx(1.0f - t);
    return x > 3.0f ? big : mid;
}

__device__ __forceinline__ float phi_out(float s2)
{
    const float t = ex2_approx(-s2);
    const float S = s2 * kLn2;
    const float den = S < 0.0625f ? S * fmaf(S, fmaf(S, 1.0f / 6.0f, -0.5f), 1.0f) : 1.0f - t;
    return (lg2_approx(1.0f + t) - lg2_approx(den)) * kLn2;
}

// The plain comparator's phi: the definition log1p(2 / expm1(x)) with the library's
// accurate expm1f/log1pf and an IEEE division.
__device__ __forceinline__ float phi_plain(float x) { return log1pf(__fdiv_rn(2.0f, expm1f(x))); }

// ------------------------------------------------------------------ vector access

template <int V>
__device__ __forceinline__ void ld_f(const float *p, float (&x)[V])
{
    if constexpr (V == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else if constexpr (V == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        x[0] = t.x; x[1] = t.y;
    } else {
        x[0] = __ldg(p);
    }
}

template <typename T, int V>
struct Msg;

template <int V>
struct Msg<float, V> {
    static __device__ __forceinline__ void load(const float *p, float (&x)[V])
    {
        if constexpr (V == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p);
            x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
        } else if constexpr (V == 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p);
            x[0] = t.x; x[1] = t.y;
        } else {
            x[0] = *p;
        }
    }
    static __device__ __forceinline__ void store(float *p, const float (&x)[V])
    {
        if constexpr (V == 4) {
            *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
        } else if constexpr (V == 2) {
            *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
        } else {
            *p = x[0];
        }
    }
};

template <int V>
struct Msg<__half, V> {
    static __device__ __forceinline__ void load(const __half *p, float (&x)[V])
    {
        if constexpr (V == 4) {
            const uint2 u = *reinterpret_cast<const uint2 *>(p);
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
            x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
        } else if constexpr (V == 2) {
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(p));
            x[0] = a.x; x[1] = a.y;
        } else {
            x[0] = __half2float(*p);
        }
    }
    static __device__ __forceinline__ void store(__half *p, const float (&x)[V])
    {
        if constexpr (V == 4) {
            __half2 a = __halves2half2(__float2half_rn(x[0]), __float2half_rn(x[1]));
            __half2 b = __halves2half2(__float2half_rn(x[2]), __float2half_rn(x[3]));
            uint2 u;
            u.x = *reinterpret_cast<uint32_t *>(&a);
            u.y = *reinterpret_cast<uint32_t *>(&b);
            *reinterpret_cast<uint2 *>(p) = u;
        } else if constexpr (V == 2) {
            *reinterpret_cast<__half2 *>(p) = __halves2half2(__float2half_rn(x[0]), __float2half_rn(x[1]));
        } else {
            *p = __float2half_rn(x[0]);
        }
    }
};

template <int V>
__device__ __forceinline__ void ld_i(const int32_t *p, int (&x)[V])
{
    if constexpr (V == 4) {
        const int4 t = *reinterpret_cast<const int4 *>(p);
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else if constexpr (V == 2) {
        const int2 t = *reinterpret_cast<const int2 *>(p);
        x[0] = t.x; x[1] = t.y;
    } else {
        x[0] = *p;
    }
}

// ------------------------------------------------------------------ interleave (kernel 1)

// llr [n_cw][N] -> L [ntiles][N][TILE]; padding codewords get L = 0 and done_at = -1.
// Block: 32 nodes x TILE codewords through shared memory, both sides coalesced.
__global__ void __launch_bounds__(256) k_interleave(const float *__restrict__ llr, int64_t n_cw, int N,
                                                    float *__restrict__ L, int32_t *__restrict__ done_at,
                                                    int32_t *__restrict__ unsat, unsigned int *status)
{
    __shared__ float sm[TILE][33];
    const int tile = blockIdx.y, n0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = w; c < TILE; c += 8) {
        const int64_t cw = (int64_t)tile * TILE + c;
        const int n = n0 + lane;
        const float v = (cw < n_cw && n < N) ? __ldg(llr + cw * N + n) : 0.0f;
        if (!isfinite(v)) atomicOr(status, IN_NONFINITE);
        sm[c][lane] = v + 0.0f;  // -0 -> +0
    }
    __syncthreads();
    for (int nn = w; nn < 32; nn += 8) {
        const int n = n0 + nn;
        if (n >= N) break;
        float *dst = L + ((int64_t)tile * N + n) * TILE;
#pragma unroll
        for (int i = 0; i < TILE / 32; i++) dst[lane + 32 * i] = sm[lane + 32 * i][nn];
    }
    if (blockIdx.x == 0) {
        for (int c = threadIdx.x; c < TILE; c += blockDim.x) {
            const int64_t cw = (int64_t)tile * TILE + c;
            done_at[cw] = cw < n_cw ? 0 : -1;
            unsat[cw] = 0;
        }
    }
}

// ------------------------------------------------------------------ deinterleave (kernel 3)

// app [ntiles][N][TILE] -> bits [n_cw][N] (APP < 0), optional app_out [n_cw][N], and
// iters[cw] = done_at if the codeword converged, else max_iter.
__global__ void __launch_bounds__(256) k_deinterleave(const float *__restrict__ app,
                                                      const int32_t *__restrict__ done_at, int64_t n_cw, int N,
                                                      int max_iter, uint8_t *__restrict__ bits,
                                                      int32_t *__restrict__ iters, float *__restrict__ app_out)
{
    __shared__ float sm[TILE][33];
    const int tile = blockIdx.y, n0 = blockIdx.x * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int nn = w; nn < 32; nn += 8) {
        const int n = n0 + nn;
        if (n >= N) break;
        const float *src = app + ((int64_t)tile * N + n) * TILE;
#pragma unroll
        for (int i = 0; i < TILE / 32; i++) sm[lane + 32 * i][nn] = __ldg(src + lane + 32 * i);
    }
    __syncthreads();
    for (int c = w; c < TILE; c += 8) {
        const int64_t cw = (int64_t)tile * TILE + c;
        const int n = n0 + lane;
        if (cw >= n_cw || n >= N) continue;
        const float v = sm[c][lane];
        bits[cw * N + n] = v < 0.0f ? 1 : 0;
        if (app_out) app_out[cw * N + n] = v;
    }
    if (blockIdx.x == 0) {
        for (int c = threadIdx.x; c < TILE; c += blockDim.x) {
            const int64_t cw = (int64_t)tile * TILE + c;
            if (cw < n_cw) {
                const int d = done_at[cw];
                iters[cw] = d > 0 ? d : max_iter;
            }
        }
    }
}

// ------------------------------------------------------------------ check-node phase

// One warp per (tile, check m, lane group).  For every edge k of check m:
//   Q_k = APP_n - R_k (R = 0 in the first iteration, FIRST), a_k = phi(clamp |Q_k|),
//   R'_k = sgn_k * min(X, phi(sum_{k' != k} a_k')),  sgn_k = product of the other signs.
// a_k carries the sign of Q_k in its sign bit.  The exclusive sums are S - a_k, except
// for an edge holding more than half of S, where the subtraction would cancel: its sum
// is formed directly.  When check_syn, the parity of the previous hard decisions over the
// check (the XOR of the APP sign bits; APP never holds -0) marks unsatisfied codewords.
#ifndef LDPC_CN_MINB
#define LDPC_CN_MINB 4  // resident 256-thread blocks per SM the check-node kernel is compiled for
#endif
#ifndef LDPC_CN_V8
#define LDPC_CN_V8 4    // codewords per lane for codes with check degree <= 8
#endif

template <int DMAX, int V, typename MsgT, bool FIRST>
__global__ void __launch_bounds__(256, LDPC_CN_MINB) k_flood_cn(const CodeDev *__restrict__ cd, const float *__restrict__ app,
                                                     MsgT *__restrict__ R, const int32_t *__restrict__ done_at,
                                                     int32_t *__restrict__ unsat, int t, int check_syn,
                                                     int64_t total_warps, float X)
{
    constexpr int WPN = TILE / (32 * V);
    constexpr uint32_t kSign = 0x80000000u;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= total_warps) return;
    const int lane = threadIdx.x & 31;
    const int M = cd->M, Z = cd->Z;
    const int64_t per_tile = (int64_t)M * WPN;
    const int tile = (int)(gw / per_tile);
    const int rem = (int)(gw - (int64_t)tile * per_tile);
    const int m = rem / WPN, sub = rem - (rem / WPN) * WPN;
    const int l = m / Z, r = m - l * Z;
    const int slot = sub * 32 * V + lane * V;
    const int64_t cw = (int64_t)tile * TILE + slot;

    int dn[V];
    ld_i<V>(done_at + cw, dn);
    bool any = false;
#pragma unroll
    for (int v = 0; v < V; v++) any |= dn[v] == 0;
    if (!__any_sync(0xffffffffu, any)) return;

    const int b0 = cd->rowptr[l];
    const int dc = cd->rowptr[l + 1] - b0;
    const float *ap = app + (int64_t)tile * cd->N * TILE + slot;
    MsgT *rp = R + (int64_t)tile * cd->E * TILE + slot;
    const float Xb = X * kLog2e;  // psi(phi(X)) = X / ln 2

    float a[DMAX][V];
    uint32_t par[V], sg[V];
    float S[V], amax[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
        par[v] = sg[v] = 0u;
        S[v] = 0.0f;
        amax[v] = 0.0f;
    }

#pragma unroll
    for (int k = 0; k < DMAX; k++) {
        if (k < dc) {
            const int ent = cd->ent[b0 + k];
            int x = r + (ent & 0xffff);
            x -= (x >= Z) ? Z : 0;
            const int n = (ent >> 16) * Z + x;
            float av[V];
            ld_f<V>(ap + (int64_t)n * TILE, av);
            float q[V];
            if constexpr (FIRST) {
#pragma unroll
                for (int v = 0; v < V; v++) q[v] = av[v];
            } else {
                float rv[V];
                Msg<MsgT, V>::load(rp + (int64_t)((b0 + k) * Z + r) * TILE, rv);
#pragma unroll
                for (int v = 0; v < V; v++) q[v] = av[v] - rv[v];
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
                par[v] ^= __float_as_uint(av[v]);
                const float mag = fminf(psi_in(fminf(fabsf(q[v]), X)), Xb);
                S[v] += mag;
                amax[v] = fmaxf(amax[v], mag);
                const uint32_t qs = __float_as_uint(q[v]) & kSign;
                sg[v] ^= qs;
                a[k][v] = __uint_as_float(__float_as_uint(mag) | qs);
            }
        }
    }

#pragma unroll
    for (int v = 0; v < V; v++) {
        // direct sum of the others for a dominant edge (a > S/2 can hold for one edge only)
        float Sx = 0.0f;
#pragma unroll
        for (int k = 0; k < DMAX; k++)
            if (k < dc) Sx += (fabsf(a[k][v]) == amax[v]) ? 0.0f : fabsf(a[k][v]);
        const float sx = (amax[v] > 0.5f * S[v]) ? Sx : S[v] - amax[v];
#pragma unroll
        for (int k = 0; k < DMAX; k++) {
            if (k < dc) {
                const float ak = fabsf(a[k][v]);
                const float ex = (ak == amax[v]) ? sx : S[v] - ak;
                const float mag = fminf(phi_out(ex), X);
                a[k][v] = __uint_as_float(__float_as_uint(mag) | ((__float_as_uint(a[k][v]) ^ sg[v]) & kSign));
            }
        }
    }

#pragma unroll
    for (int k = 0; k < DMAX; k++) {
        if (k < dc) {
            float o[V];
#pragma unroll
            for (int v = 0; v < V; v++) o[v] = a[k][v];
            Msg<MsgT, V>::store(rp + (int64_t)((b0 + k) * Z + r) * TILE, o);
        }
    }
    if (check_syn) {
#pragma unroll
        for (int v = 0; v < V; v++)
            if ((par[v] & kSign) && dn[v] == 0) unsat[cw + v] = t;
    }
}

// ------------------------------------------------------------------ variable-node phase

// Messages of D column entries (colent: (b << 16) | s) of variable position c, added onto s
// in the order of the column lists; all D loads are issued before the first add.
template <int D, int V, typename MsgT>
__device__ __forceinline__ void svn_sum(const int32_t *__restrict__ colent, const MsgT *rt, int c, int Z,
                                        float (&s)[V])
{
    float rv[D][V];
#pragma unroll
    for (int k = 0; k < D; k++) {
        const int ce = colent[k];
        int rr = c - (ce & 0xffff);
        rr += (rr < 0) ? Z : 0;
        Msg<MsgT, V>::load(rt + (int64_t)((ce >> 16) * Z + rr) * TILE, rv[k]);
    }
#pragma unroll
    for (int k = 0; k < D; k++)
#pragma unroll
        for (int v = 0; v < V; v++) s[v] += rv[k][v];
}

// One warp per (tile, variable n, lane group): APP_n = L_n + sum over the column's blocks
// of R at edge (b, (c - s) mod Z), c = n mod Z.  Codewords already frozen keep their APP;
// a codeword whose iteration-t check phase stamped no failing check is frozen here with
// done_at = t - 1.
template <int V, typename MsgT>
__global__ void __launch_bounds__(256) k_flood_vn(const CodeDev *__restrict__ cd, const float *__restrict__ L,
                                                  const MsgT *__restrict__ R, float *__restrict__ app,
                                                  int32_t *__restrict__ done_at, const int32_t *__restrict__ unsat,
                                                  int t, int early_exit, int64_t total_warps)
{
    constexpr int WPN = TILE / (32 * V);
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= total_warps) return;
    const int lane = threadIdx.x & 31;
    const int N = cd->N, Z = cd->Z;
    const int64_t per_tile = (int64_t)N * WPN;
    const int tile = (int)(gw / per_tile);
    const int rem = (int)(gw - (int64_t)tile * per_tile);
    const int n = rem / WPN, sub = rem - (rem / WPN) * WPN;
    const int j = n / Z, c = n - j * Z;
    const int slot = sub * 32 * V + lane * V;
    const int64_t cw = (int64_t)tile * TILE + slot;

    int dn[V];
    ld_i<V>(done_at + cw, dn);
    bool act[V];
    bool any = false, all = true;
#pragma unroll
    for (int v = 0; v < V; v++) {
        act[v] = dn[v] == 0;
        if (act[v] && early_exit && t >= 2 && unsat[cw + v] != t) {
            act[v] = false;
            done_at[cw + v] = t - 1;
        }
        any |= act[v];
        all &= act[v];
    }
    if (!__any_sync(0xffffffffu, any)) return;

    float s[V];
    ld_f<V>(L + ((int64_t)tile * N + n) * TILE + slot, s);
    const MsgT *rt = R + (int64_t)tile * cd->E * TILE + slot;
    const int i0 = cd->colptr[j], dv = cd->colptr[j + 1] - i0;
    if (dv == 3)
        svn_sum<3, V, MsgT>(cd->colent + i0, rt, c, Z, s);
    else if (dv == 2)
        svn_sum<2, V, MsgT>(cd->colent + i0, rt, c, Z, s);
    else if (dv == 4)
        svn_sum<4, V, MsgT>(cd->colent + i0, rt, c, Z, s);
    else
        for (int i = 0; i < dv; i++) svn_sum<1, V, MsgT>(cd->colent + i0 + i, rt, c, Z, s);
#pragma unroll
    for (int v = 0; v < V; v++) s[v] += 0.0f;  // -0 -> +0: the APP sign bit is the hard decision
    float *dst = app + ((int64_t)tile * N + n) * TILE + slot;
    if (all) {
        Msg<float, V>::store(dst, s);
    } else {
#pragma unroll
        for (int v = 0; v < V; v++)
            if (act[v]) dst[v] = s[v];
    }
}

// ------------------------------------------------------------------ plain comparator

// The plain FP32 flooding decoder: one thread per (codeword, node), the library phi,
// exclusive sums formed directly over the other edges, no first-iteration or converged-
// warp shortcuts.  Same layouts and early-exit protocol as the optimised kernels.
template <int DMAX>
__global__ void __launch_bounds__(256) k_plain_cn(const CodeDev *__restrict__ cd, const float *__restrict__ app,
                                                  float *__restrict__ R, const int32_t *__restrict__ done_at,
                                                  int32_t *__restrict__ unsat, int t, int check_syn, int ntiles,
                                                  float X, float phiX)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int M = cd->M, Z = cd->Z;
    const int64_t total = (int64_t)ntiles * M * TILE;
    if (gid >= total) return;
    const int64_t tm = gid / TILE;
    const int slot = (int)(gid - tm * TILE);
    const int tile = (int)(tm / M), m = (int)(tm - (int64_t)tile * M);
    const int64_t cw = (int64_t)tile * TILE + slot;
    if (done_at[cw] != 0) return;
    const int l = m / Z, r = m - l * Z;
    const int b0 = cd->rowptr[l], dc = cd->rowptr[l + 1] - b0;
    const float *ap = app + (int64_t)tile * cd->N * TILE + slot;
    float *rp = R + (int64_t)tile * cd->E * TILE + slot;
    float q[DMAX], a[DMAX];
    uint32_t par = 0;
#pragma unroll
    for (int k = 0; k < DMAX; k++) {
        if (k < dc) {
            const int ent = cd->ent[b0 + k];
            const int n = (ent >> 16) * Z + (r + (ent & 0xffff)) % Z;
            const float av = ap[(int64_t)n * TILE];
            par ^= av < 0.0f ? 1u : 0u;
            q[k] = av - rp[(int64_t)((b0 + k) * Z + r) * TILE];
            a[k] = phi_plain(fminf(fmaxf(fabsf(q[k]), phiX), X));
        }
    }
#pragma unroll
    for (int k = 0; k < DMAX; k++) {
        if (k < dc) {
            float sum = 0.0f;
            bool negp = false;
#pragma unroll
            for (int k2 = 0; k2 < DMAX; k2++) {
                if (k2 < dc && k2 != k) {
                    sum += a[k2];
                    negp ^= q[k2] < 0.0f;
                }
            }
            const float mag = fminf(phi_plain(sum), X);
            rp[(int64_t)((b0 + k) * Z + r) * TILE] = negp ? -mag : mag;
        }
    }
    if (check_syn && par) unsat[cw] = t;
}

__global__ void __launch_bounds__(256) k_plain_vn(const CodeDev *__restrict__ cd, const float *__restrict__ L,
                                                  const float *__restrict__ R, float *__restrict__ app,
                                                  int32_t *__restrict__ done_at, const int32_t *__restrict__ unsat,
                                                  int t, int early_exit, int ntiles)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = cd->N, Z = cd->Z;
    const int64_t total = (int64_t)ntiles * N * TILE;
    if (gid >= total) return;
    const int64_t tn = gid / TILE;
    const int slot = (int)(gid - tn * TILE);
    const int tile = (int)(tn / N), n = (int)(tn - (int64_t)tile * N);
    const int64_t cw = (int64_t)tile * TILE + slot;
    if (done_at[cw] != 0) return;
    if (early_exit && t >= 2 && unsat[cw] != t) {
        done_at[cw] = t - 1;
        return;
    }
    const int j = n / Z, c = n - j * Z;
    float s = L[((int64_t)tile * N + n) * TILE + slot];
    const float *rt = R + (int64_t)tile * cd->E * TILE + slot;
    for (int i = cd->colptr[j]; i < cd->colptr[j + 1]; i++) {
        const int ce = cd->colent[i];
        const int rr = (c - (ce & 0xffff) + Z) % Z;
        s += rt[(int64_t)((ce >> 16) * Z + rr) * TILE];
    }
    app[((int64_t)tile * N + n) * TILE + slot] = s;
}

// ------------------------------------------------------------------ host side

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t flood_ws_layout(const CodeDev &c, int64_t n_cw, int msg, FloodWs *ws, char *base)
{
    const int64_t ntiles = (n_cw + TILE - 1) / TILE;
    const size_t node = (size_t)ntiles * TILE;
    const size_t szL = align256(node * c.N * sizeof(float));
    const size_t szR = align256(node * c.E * (msg == LDPC_MSG_F16 ? sizeof(__half) : sizeof(float)));
    const size_t szF = align256(node * sizeof(int32_t));
    size_t off = 0;
    if (ws) {
        ws->L = reinterpret_cast<float *>(base + off);
        ws->app = reinterpret_cast<float *>(base + off + szL);
        ws->R = base + off + 2 * szL;
        ws->done_at = reinterpret_cast<int32_t *>(base + off + 2 * szL + szR);
        ws->unsat = reinterpret_cast<int32_t *>(base + off + 2 * szL + szR + szF);
    }
    off = 2 * szL + szR + 2 * szF;
    return off;
}

template <int DMAX, int V, typename MsgT>
static cudaError_t flood_iterations(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p,
                                    const FloodWs &ws, int64_t ntiles, cudaStream_t s)
{
    constexpr int WPN = TILE / (32 * V);
    const float X = p.phi_clamp;
    const int64_t cn_warps = ntiles * h.M * WPN, vn_warps = ntiles * h.N * WPN;
    const unsigned cn_blocks = (unsigned)((cn_warps + 7) / 8), vn_blocks = (unsigned)((vn_warps + 7) / 8);
    MsgT *R = reinterpret_cast<MsgT *>(ws.R);
    for (int t = 1; t <= p.max_iter; t++) {
        {
            LaunchScope ls(F_CN, s);
            if (t == 1)
                k_flood_cn<DMAX, V, MsgT, true><<<cn_blocks, 256, 0, s>>>(d, ws.L, R, ws.done_at, ws.unsat, t, 0,
                                                                         cn_warps, X);
            else
                k_flood_cn<DMAX, V, MsgT, false><<<cn_blocks, 256, 0, s>>>(d, ws.app, R, ws.done_at, ws.unsat, t,
                                                                          p.early_exit, cn_warps, X);
        }
        {
            LaunchScope ls(F_VN, s);
            k_flood_vn<V, MsgT><<<vn_blocks, 256, 0, s>>>(d, ws.L, R, ws.app, ws.done_at, ws.unsat, t, p.early_exit,
                                                          vn_warps);
        }
    }
    return cudaGetLastError();
}

template <int DMAX>
static cudaError_t plain_iterations(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p,
                                    const FloodWs &ws, int64_t ntiles, cudaStream_t s)
{
    const float X = p.phi_clamp;
    const float phiX = (float)log1p(2.0 / expm1((double)X));
    const int64_t cn_thr = ntiles * h.M * TILE, vn_thr = ntiles * h.N * TILE;
    cudaError_t e = cudaMemsetAsync(ws.R, 0, (size_t)ntiles * TILE * h.E * sizeof(float), s);
    if (e != cudaSuccess) return e;
    for (int t = 1; t <= p.max_iter; t++) {
        {
            LaunchScope ls(F_PLAIN_CN, s);
            k_plain_cn<DMAX><<<(unsigned)((cn_thr + 255) / 256), 256, 0, s>>>(
                d, t == 1 ? ws.L : ws.app, reinterpret_cast<float *>(ws.R), ws.done_at, ws.unsat, t,
                t >= 2 && p.early_exit, (int)ntiles, X, phiX);
        }
        {
            LaunchScope ls(F_PLAIN_VN, s);
            k_plain_vn<<<(unsigned)((vn_thr + 255) / 256), 256, 0, s>>>(
                d, ws.L, reinterpret_cast<float *>(ws.R), ws.app, ws.done_at, ws.unsat, t, p.early_exit, (int)ntiles);
        }
    }
    return cudaGetLastError();
}

cudaError_t flood_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const float *llr,
                         int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, const FloodWs &ws,
                         cudaStream_t s)
{
    const int64_t ntiles = (n_cw + TILE - 1) / TILE;
    const dim3 tgrid((unsigned)((h.N + 31) / 32), (unsigned)ntiles);
    {
        LaunchScope ls(F_INTERLEAVE, s);
        k_interleave<<<tgrid, 256, 0, s>>>(llr, n_cw, h.N, ws.L, ws.done_at, ws.unsat, h.status);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool f16 = p.msg == LDPC_MSG_F16;
    if (p.impl == LDPC_IMPL_PLAIN) {
        if (h.dc_max <= 8) e = plain_iterations<8>(h, d, p, ws, ntiles, s);
        else if (h.dc_max <= 16) e = plain_iterations<16>(h, d, p, ws, ntiles, s);
        else e = plain_iterations<32>(h, d, p, ws, ntiles, s);
    } else if (h.dc_max <= 8) {
        e = f16 ? flood_iterations<8, LDPC_CN_V8, __half>(h, d, p, ws, ntiles, s)
                : flood_iterations<8, LDPC_CN_V8, float>(h, d, p, ws, ntiles, s);
    } else if (h.dc_max <= 16) {
        e = f16 ? flood_iterations<16, 2, __half>(h, d, p, ws, ntiles, s)
                : flood_iterations<16, 2, float>(h, d, p, ws, ntiles, s);
    } else {
        e = f16 ? flood_iterations<32, 1, __half>(h, d, p, ws, ntiles, s)
                : flood_iterations<32, 1, float>(h, d, p, ws, ntiles, s);
    }
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls(F_DEINTERLEAVE, s);
        k_deinterleave<<<tgrid, 256, 0, s>>>(ws.app, ws.done_at, n_cw, h.N, p.max_iter, bits, iters, app_out);
    }
    return cudaGetLastError();
}

}  // namespace ldpc
