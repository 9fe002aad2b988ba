// Horizontal layered sum-product decoding with the decoder state on chip (Sec. II
// "Algorithm 2" schedule with the sum-product check rule of Sec. I).
//
// A persistent grid of one CTA per SM.  Each CTA holds C codeword slots; a slot keeps its
// posterior APP [N] (fp32) and its check-to-variable messages R [E] (fp32 or fp16) in
// shared memory for the whole decode of one codeword.  The slots form barrier groups of K:
// a group's threads cover its K*Z check rows packed into whole warps, and thread u of a
// group owns check row u mod Z of slot u / Z, for every block row (layer).  The Z checks of
// a QC layer touch disjoint variables (each block is one circulant), so the row threads
// update a layer at once and the group's own barrier (a named barrier, or the warp itself
// when the group is one warp) separates consecutive layers: the slots of a group run in
// lock-step, the groups independently, with no CTA-wide barrier.  K trades the idle lanes
// of a warp-aligned slot (Z not a multiple of 32) against waiting for a group's slowest slot.
// Messages are stored in check-row order, edge (b, r) at b*Z + r: the layered schedule has
// no variable-node pass, so the row threads of a warp read and write them contiguously.
// Per check (the arithmetic of the flooding slot decoder, only the schedule differs):
//   Q_k   = APP_n - R_k                                   over the check's edges
//   R'_k  = prod_{other} sgn Q * min(X, phi( sum_{other} phi(clampX |Q|) ))
//           in the product (tanh) domain (slot_common.cuh), stored as fp16 when the
//           messages are half precision
//   APP_n = Q_k + R'_k   with R'_k the stored value, so that the next Q = APP - R removes
//                        exactly what was added
// After every full iteration each slot's hard decisions are checked against all of its
// checks; a slot that converged (early exit) or reached max_iter writes its outputs and
// takes the next codeword from the global work counter at its group's next iteration.
//
// APP is never -0: the refill adds +0 to the (scaled) channel value and Q + R' is -0 only when both
// are -0, which cannot happen while APP is not -0 (then Q = APP - R is not -0).  The sign
// bit therefore is the hard decision [APP < 0] and sgn(0) = +1, as the oracle reads it.
#include "slot_common.cuh"

namespace ldpc {

#ifndef LDPC_LSPA_REFILL_CHUNK
#define LDPC_LSPA_REFILL_CHUNK 1  // channel values a thread requests at once when a slot takes a codeword
#endif
#ifndef LDPC_LSPA_KMAX
#define LDPC_LSPA_KMAX 64  // most slots in one barrier group
#endif

// The FP32-message form keeps APP, Q and R in base-2 units (LLR x log2 e, set at the refill
// and undone at the output), which spares the check rule its scaling multiplies; the
// FP16-message form stays in natural units, so that its stored binary16 message is the
// natural-unit value rounded, as the oracle's binary16 mode rounds it.
// (Measured on the 8192-codeword N = 1944 rate-1/2 sweep: base-2 units 9.22 info Gbit/s,
// natural units 8.98; the flooding slot decoder measured the other way round.)
#ifndef LDPC_LSPA_B2
#define LDPC_LSPA_B2 1
#endif
template <typename MsgT>
constexpr bool kBase2 = LDPC_LSPA_B2 && sizeof(MsgT) == 4;

struct LayeredSpaArgs {
    const float *llr;
    int64_t n_cw;
    int C, strideA, strideR;  // slots per CTA; per-slot APP and R strides (elements)
    int K, TPG;               // slots per barrier group; threads per group (whole warps)
    int max_iter, early_exit;
    float X;
    uint8_t *bits;
    int32_t *iters;
    float *app_out;
    unsigned long long *next;
};

template <typename MsgT>
struct MsgIO;
template <>
struct MsgIO<float> {
    // store the message; return the value as stored
    static __device__ __forceinline__ float st(float *p, float x)
    {
        *p = x;
        return x;
    }
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
};
template <>
struct MsgIO<__half> {
    static __device__ __forceinline__ float st(__half *p, float x)
    {
        const __half h = __float2half_rn(x);
        *p = h;
        return __half2float(h);
    }
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
};

// Edge descriptor of block b = (row l, column j, shift s) for the layered slots: .x = byte
// offset of the posterior j*Z + s, .y = byte offset of the message row b*Z, .z = Z - s.
// Check row r reaches variable position (r + s) mod Z: .x from the thread's posterior base
// (position r), less one block (ZA bytes) when r >= .z; its message is .y from its message
// base (row r), with no wrap.
__device__ __forceinline__ int lspa_app_off(const int4 d, int r, int ZA) { return d.x - (r >= d.z ? ZA : 0); }

// One check of row r (degree <= 8) in the product (tanh) domain: with d_k = e^-a_k,
// a_k = |Q_k| clamped to [phi(X), X], the pair (alpha, beta) of the other edges' maps
// (alpha, beta) <- (alpha + d beta, beta + d alpha) from (1, 0) gives
// R'_k = ln(alpha / beta) = phi(sum_{other} phi(a)) (slot_common.cuh); one ex2 and two lg2
// per edge.  The FP32 form holds Q per edge; the FP16 form (1024 threads, 64 registers)
// forms it again from APP and R, neither of which is written before its own edge is.
template <int D, bool EXACT, typename MsgT>
__device__ __forceinline__ void layer_check_tanh(int dc, const int4 *__restrict__ ed, char *Ar, char *Rr, int r, int ZA,
                                                 float Xb, float Pb)
{
    constexpr uint32_t kSign = 0x80000000u;
    constexpr bool B2 = kBase2<MsgT>, kHoldQ = sizeof(MsgT) == 4;
    MsgT *Rl = at<MsgT>(Rr, ed[0].y);
    const int Zm = ZA / (int)sizeof(float);
    float d[D];
    int ao[D];
    float q[kHoldQ ? D : 1];
    uint32_t sg = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        d[k] = 0.0f;  // a missing edge (k >= dc) is the identity map
        ao[k] = 0;
        if (EXACT || k < dc) {
            ao[k] = lspa_app_off(ed[k], r, ZA);
            const float qk = *at<float>(Ar, ao[k]) - MsgIO<MsgT>::ld(Rl + k * Zm);
            if constexpr (kHoldQ) q[k] = qk;
            sg ^= __float_as_uint(qk);
            d[k] = tanh_d<B2>(qk, Xb, Pb);
        }
    }
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
            const float mag = tanh_mag<B2>(al, be);
            float qk;
            if constexpr (kHoldQ)
                qk = q[k];
            else
                qk = *at<float>(Ar, ao[k]) - MsgIO<MsgT>::ld(Rl + k * Zm);
            const float out = __uint_as_float(__float_as_uint(mag) | ((__float_as_uint(qk) ^ sg) & kSign));
            *at<float>(Ar, ao[k]) = qk + MsgIO<MsgT>::st(Rl + k * Zm, out);
        }
        if (k == 0) {
            pb = d[0];
        } else if (k < D - 1) {
            const float t = fmaf(d[k], pb, pa);
            pb = fmaf(d[k], pa, pb);
            pa = t;
        }
    }
}

// One check of row r in the layer whose blocks start at descriptor `ed`, computed from and
// written back to the slot's APP (thread base Ar) and R (thread base Rr): rows up to degree 8
// hold their state per edge, wider rows take the grouped form (see slot_common.cuh), with Q
// formed from APP and R in both passes (neither is written before its own edge is) and
// APP = Q + R' at the store.
template <int D, bool EXACT, typename MsgT>
__device__ __forceinline__ void layer_check(int dc, const int4 *__restrict__ ed, char *Ar, char *Rr, int r, int ZA,
                                            float Xb, float Pb)
{
    if constexpr (D <= 8) {
        layer_check_tanh<D, EXACT, MsgT>(dc, ed, Ar, Rr, r, ZA, Xb, Pb);
    } else {
        MsgT *Rl = at<MsgT>(Rr, ed[0].y);
        const int Zm = ZA / (int)sizeof(float);
        auto qof = [&](int k, bool) -> float {
            return *at<float>(Ar, lspa_app_off(ed[k], r, ZA)) - MsgIO<MsgT>::ld(Rl + k * Zm);
        };
        auto put = [&](int k, float m, float q) {
            *at<float>(Ar, lspa_app_off(ed[k], r, ZA)) = q + MsgIO<MsgT>::st(Rl + k * Zm, m);
        };
        tanh_check_wide<D, kBase2<MsgT>>(dc, Xb, Pb, qof, put);
    }
}

template <int D, int DMAX, typename MsgT>
__device__ __forceinline__ void layer_check_dispatch(int dc, const int4 *__restrict__ ed, char *Ar, char *Rr, int r,
                                                     int ZA, float Xb, float Pb)
{
    if constexpr (D >= DMAX) {
        layer_check<DMAX, false, MsgT>(dc, ed, Ar, Rr, r, ZA, Xb, Pb);
    } else if constexpr (D <= 8) {
        if (dc == D)
            layer_check<D, true, MsgT>(dc, ed, Ar, Rr, r, ZA, Xb, Pb);
        else
            layer_check_dispatch<next_degree(D), DMAX, MsgT>(dc, ed, Ar, Rr, r, ZA, Xb, Pb);
    } else {
        if (dc <= D)
            layer_check<D, false, MsgT>(dc, ed, Ar, Rr, r, ZA, Xb, Pb);
        else
            layer_check_dispatch<next_degree(D), DMAX, MsgT>(dc, ed, Ar, Rr, r, ZA, Xb, Pb);
    }
}

// XOR of the posterior sign bits of check row r of one block row (degree dc): straight-line
// bodies for the common degrees (every lane of a warp takes the same branch).
template <int D>
__device__ __forceinline__ uint32_t lspa_parity(const int4 *__restrict__ ed, const char *Ar, int r, int ZA)
{
    uint32_t par = 0;
#pragma unroll
    for (int k = 0; k < D; k++) par ^= __float_as_uint(*at<float>(Ar, lspa_app_off(ed[k], r, ZA)));
    return par;
}
__device__ __forceinline__ uint32_t lspa_row_parity(int dc, const int4 *__restrict__ ed, const char *Ar, int r,
                                                    int ZA)
{
    switch (dc) {
    case 4: return lspa_parity<4>(ed, Ar, r, ZA);
    case 5: return lspa_parity<5>(ed, Ar, r, ZA);
    case 6: return lspa_parity<6>(ed, Ar, r, ZA);
    case 7: return lspa_parity<7>(ed, Ar, r, ZA);
    case 8: return lspa_parity<8>(ed, Ar, r, ZA);
    default: {
        uint32_t par = 0;
        for (int k = 0; k < dc; k++) par ^= __float_as_uint(*at<float>(Ar, lspa_app_off(ed[k], r, ZA)));
        return par;
    }
    }
}

// Table space (ints) ahead of the slots: four per block for its edge descriptor, then the
// block-row pointers.
__host__ __device__ inline int lspa_tables_ints(int nnz, int mb) { return 4 * nnz + mb + 1; }

// Threads per CTA for an instance: high-degree checks keep more values live per thread.
// fp32 slots are limited to a few per CTA by shared memory, so their threads get more
// registers (672 = 7 slots of three warps at 96 registers); fp16 slots are twice as many
// and run the register-lean check form.
template <int DMAX, typename MsgT>
constexpr int lspa_threads_max()
{
    return sizeof(MsgT) == 4 ? (DMAX <= 16 ? 672 : 512) : (DMAX <= 8 ? 1024 : (DMAX <= 16 ? 768 : 512));
}

// The barrier of one slot group: its warps only (named barrier group + 1; barrier 0 is the
// CTA's), or nothing beyond the warp itself when the group is one warp.
__device__ __forceinline__ void group_sync(int grp, int tpg)
{
    if (tpg == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(tpg) : "memory");
}

template <int DMAX, typename MsgT>
__global__ void __launch_bounds__(lspa_threads_max<DMAX, MsgT>(), 1) k_layered_spa(const CodeDev *__restrict__ cd,
                                                                                    const LayeredSpaArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = cd->N, Z = cd->Z, mb = cd->mb, nb = cd->nb, nnz = cd->nnz;
    const int C = a.C, K = a.K, TPG = a.TPG;
    int32_t *bad = reinterpret_cast<int32_t *>(smem);                 // [SLOTS_MAX] unsatisfied check seen
    int32_t *gany = bad + SLOTS_MAX;                                   // [SLOTS_MAX / 2][2] group vote
    int64_t *fresh = reinterpret_cast<int64_t *>(gany + SLOTS_MAX);    // [SLOTS_MAX] the slot's codeword
    int4 *t_ed = reinterpret_cast<int4 *>(fresh + SLOTS_MAX);         // edge descriptor per block
    int32_t *t_rowptr = reinterpret_cast<int32_t *>(t_ed + nnz);
    float *APPs = reinterpret_cast<float *>(smem + slots_smem_head(lspa_tables_ints(nnz, mb)));
    MsgT *Rs = reinterpret_cast<MsgT *>(APPs + (size_t)C * a.strideA);

    const int tid = threadIdx.x, nth = blockDim.x;
    const float Xb = a.X * kSLog2e, Pb = s_phi_b2(a.X);  // the clamp [phi(X), X] in base-2 units
    for (int i = tid; i < nnz; i += nth) {
        const int e = cd->ent[i], sh = e & 0xffff;
        t_ed[i] = make_int4((int)sizeof(float) * ((e >> 16) * Z + sh), (int)sizeof(MsgT) * i * Z, Z - sh, 0);
    }
    const int ZA = (int)sizeof(float) * Z;
    for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
    const int g = tid / TPG, u = tid - (tid / TPG) * TPG;
    const int c = g * K + u / Z, r = u - (u / Z) * Z;
    const bool mine = u < K * Z && c < C;  // a row of a slot (else an idle lane of the group)
    if (tid == 0)
        for (int i = 0; i < SLOTS_MAX; i++) gany[i] = 0;
    if (mine && r == 0) {
        const unsigned long long k = atomicAdd(a.next, 1ull);
        fresh[c] = k < (unsigned long long)a.n_cw ? (int64_t)k : -1;
        bad[c] = 0;
    }
    __syncthreads();
    if (g * K >= C) return;  // whole warps beyond the last group
    float *A = APPs + (size_t)(mine ? c : 0) * a.strideA;
    MsgT *Rc = Rs + (size_t)(mine ? c : 0) * a.strideR;
    char *Ar = reinterpret_cast<char *>(A + r), *Rr = reinterpret_cast<char *>(Rc + r);
    int ph = 0;
    // OR of a predicate over the group (every thread of the group calls it at the same
    // point; the vote alternates between two words so that clearing the next one races with
    // nothing)
    auto group_any = [&](bool pred) {
        if (pred) gany[2 * g + ph] = 1;
        group_sync(g, TPG);
        const bool any = gany[2 * g + ph] != 0;
        if (u == 0) gany[2 * g + (ph ^ 1)] = 0;
        ph ^= 1;
        return any;
    };

    // a slot given codeword k loads APP = L (+0: no -0 in APP) and clears its messages; the
    // channel values of a chunk are all requested before any is used
    auto refill = [&](int64_t k) {
        const float *L = a.llr + k * N;
        constexpr int CH = LDPC_LSPA_REFILL_CHUNK;
        for (int j0 = 0; j0 < nb; j0 += CH) {
            float v[CH];
#pragma unroll
            for (int w = 0; w < CH; w++)
                if (j0 + w < nb) v[w] = __ldg(L + (j0 + w) * Z + r);
#pragma unroll
            for (int w = 0; w < CH; w++)
                if (j0 + w < nb) {
                    if (!isfinite(v[w])) atomicOr(cd->status, IN_NONFINITE);
                    A[(j0 + w) * Z + r] = kBase2<MsgT> ? fmaf(v[w], kSLog2e, 0.0f) : v[w] + 0.0f;
                }
        }
        for (int b = 0; b < nnz; b++) Rc[b * Z + r] = MsgT(0.0f);
    };

    int64_t cw = mine ? fresh[c] : -1;
    int t = 0;
    if (cw >= 0) refill(cw);
    if (!group_any(cw >= 0)) return;

    for (;;) {
        const bool busy = cw >= 0;
        for (int l = 0; l < mb; l++) {
            if (busy) {
                const int b0 = t_rowptr[l];
                layer_check_dispatch<2, DMAX, MsgT>(t_rowptr[l + 1] - b0, t_ed + b0, Ar, Rr, r, ZA, Xb, Pb);
            }
            group_sync(g, TPG);
        }
        if (busy) t++;
        // syndrome of the hard decisions (APP sign bits): row r of every layer
        if (busy && a.early_exit) {
            uint32_t par_any = 0;
            for (int l = 0; l < mb; l++) {
                const int b0 = t_rowptr[l];
                par_any |= lspa_row_parity(t_rowptr[l + 1] - b0, t_ed + b0, Ar, r, ZA);
            }
            if (par_any & 0x80000000u) bad[c] = 1;
        }
        group_sync(g, TPG);
        bool done = false;
        if (busy) {
            done = (a.early_exit && bad[c] == 0) || t >= a.max_iter;
            if (done) {
                uint8_t *Bo = a.bits + cw * N;
                float *Ao = a.app_out ? a.app_out + cw * N : nullptr;
                for (int j = 0; j < nb; j++) {
                    const float v = A[j * Z + r];
                    Bo[j * Z + r] = v < 0.0f ? 1 : 0;
                    if (Ao) Ao[j * Z + r] = kBase2<MsgT> ? v * kSLn2 : v;
                }
                if (r == 0) {
                    a.iters[cw] = t;
                    const unsigned long long k = atomicAdd(a.next, 1ull);
                    fresh[c] = k < (unsigned long long)a.n_cw ? (int64_t)k : -1;
                }
            }
        }
        group_sync(g, TPG);
        if (busy) {
            if (r == 0) bad[c] = 0;
            if (done) {
                cw = fresh[c];
                t = 0;
                if (cw >= 0) refill(cw);
            }
        }
        if (!group_any(cw >= 0)) break;
    }
}

static size_t lspa_slot_bytes(const CodeDev &h, int msg)
{
    return (size_t)((h.N + 3) & ~3) * sizeof(float) +
           (size_t)((h.E + 7) & ~7) * (msg == LDPC_MSG_F16 ? sizeof(__half) : sizeof(float));
}

static int lspa_threads_for(int dc_max, int msg)
{
    const int d = dc_max <= 8 ? 8 : dc_max <= 16 ? 16 : dc_max <= 24 ? 24 : 32;
    if (msg == LDPC_MSG_F16)
        return d == 8 ? lspa_threads_max<8, __half>() : d == 16 ? lspa_threads_max<16, __half>()
                                                               : lspa_threads_max<32, __half>();
    return d <= 16 ? lspa_threads_max<16, float>() : lspa_threads_max<32, float>();
}

static size_t lspa_smem(const CodeDev &h, int msg, int C)
{
    return slots_smem_head(lspa_tables_ints(h.nnz, h.mb)) + (size_t)C * lspa_slot_bytes(h, msg);
}

// Slots per CTA and their grouping: the most slots that fit the instance's threads, 15 named
// barriers and shared memory, with the fewest slots per group among the arrangements that
// reach that count.
struct LspaShape {
    int C, K, TPG;
};
static LspaShape lspa_shape(const CodeDev &h, int msg, int64_t cap = SLOTS_MAX)
{
    LspaShape best = {0, 1, 32};
    if (h.dc_max > 32 || h.N >= 65536) return best;
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t limit = lim > 0 ? (size_t)lim : 227 * 1024;
    int cmax = SLOTS_MAX;
    while (cmax > 0 && lspa_smem(h, msg, cmax) > limit) cmax--;
    if (cap >= 1 && cap < cmax) cmax = (int)cap;  // a small batch spreads over the SMs
    const int tmax = lspa_threads_for(h.dc_max, msg);
    for (int K = 1; K <= cmax && K <= LDPC_LSPA_KMAX; K++) {
        const int tpg = ((K * h.Z + 31) / 32) * 32;
        int G = tmax / tpg;
        if (tpg > 32 && G > 15) G = 15;
        int C = G * K;
        if (C > cmax) C = cmax;
        if (C > best.C) best = {C, K, tpg};
    }
    return best;
}

int layered_spa_slots_per_cta(const CodeDev &h, int msg) { return lspa_shape(h, msg).C; }

template <int DMAX, typename MsgT>
static cudaError_t launch_lspa(const CodeDev &h, const CodeDev *d, const LayeredSpaArgs &a, int msg, cudaStream_t s)
{
    const size_t sm = lspa_smem(h, msg, a.C);
    cudaError_t e = ensure_smem<k_layered_spa<DMAX, MsgT>>(sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t ctas = nsm;
    const int64_t need = (a.n_cw + a.C - 1) / a.C;
    if (need < ctas) ctas = need;
    LaunchScope ls(F_LAYERED_SPA, s);
    const int groups = (a.C + a.K - 1) / a.K;
    k_layered_spa<DMAX, MsgT><<<(unsigned)ctas, groups * a.TPG, sm, s>>>(d, a);
    return cudaGetLastError();
}

template <typename MsgT>
static cudaError_t launch_lspa_d(const CodeDev &h, const CodeDev *d, const LayeredSpaArgs &a, int msg, cudaStream_t s)
{
    if (h.dc_max <= 8) return launch_lspa<8, MsgT>(h, d, a, msg, s);
    if (h.dc_max <= 16) return launch_lspa<16, MsgT>(h, d, a, msg, s);
    if (h.dc_max <= 24) return launch_lspa<24, MsgT>(h, d, a, msg, s);
    return launch_lspa<32, MsgT>(h, d, a, msg, s);
}

cudaError_t layered_spa_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const float *llr,
                               int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, void *counter,
                               cudaStream_t s)
{
    LayeredSpaArgs a;
    a.llr = llr;
    a.n_cw = n_cw;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const LspaShape sh = lspa_shape(h, p.msg, (n_cw + nsm - 1) / nsm);
    a.C = sh.C;
    if (a.C < 1) return cudaErrorInvalidValue;
    a.K = sh.K;
    a.TPG = sh.TPG;
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
    return p.msg == LDPC_MSG_F16 ? launch_lspa_d<__half>(h, d, a, p.msg, s) : launch_lspa_d<float>(h, d, a, p.msg, s);
}

}  // namespace ldpc
