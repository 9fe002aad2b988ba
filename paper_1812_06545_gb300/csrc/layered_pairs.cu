// Horizontal layered normalised min-sum with two codewords per thread (Sec. II "Algorithm 2":
// the checks of a layer are computed from the current variable values, which are updated at
// once; Sec. III-A frame-level parallelism), bit-exact with the integer definition.
//
// Every quantity of the integer min-sum is an integer of magnitude below 2048, which binary16
// represents exactly, and the packed half-precision instructions (add, min/max, compare,
// fused multiply-add) act on two such values at once and round only when the exact result
// is not representable.  So a thread carries the same check row of two codewords in the two
// halves of each 32-bit register and runs every step of the check once for both:
//   Q_k   = sat(APP_n - R_k, msg_sat)                      add, add, min, max
//   min1, min2 over |Q_k| (duplicates counted)             and, 3 x min/max per edge
//   S     = XOR of the sign bits of Q_k                    xor of the whole words
//   mag_k = alpha * (|Q_k| == min1 ? min2 : min1)          compare mask, select
//   R_k   = mag_k with sign S xor sign(Q_k)                xor of the sign bits
//   APP_n = sat(Q_k + R_k, app_sat)                        add (+ min, max if it can bind)
// The edge whose |Q| equals min1 takes min2; when two edges share min1, min2 = min1 and the
// choice is immaterial, so no argmin is tracked.  alpha * m = floor(alpha_num * m /
// 2^alpha_shift) is formed per check as round(alpha m - delta) with delta = 1/2 -
// 2^-(alpha_shift + 1): the fractions of alpha m are multiples of 2^-alpha_shift, so alpha m -
// delta lies strictly within 1/2 of floor(alpha m), and adding 1536 (binary16 spacing 1 in
// [1024, 2048)) rounds it there; the host admits only parameters for which alpha m - delta is
// itself exact (layered_pairs_exact).  Zero is never negative: APP starts at +0 (the
// quantiser's -0 becomes +0), and a sum of two opposite values that cancel is +0, so the sign
// bit of APP is the hard decision and that of Q is [Q < 0].
//
// Storage (shared memory, one CTA per SM, persistent, the slot and barrier-group arrangement
// of k_layered_slots with a thread slot holding two codewords): APP as half2 [slot][N], and R
// as two bytes per edge, each R + 128; R is widened to binary16 by placing the byte under the
// exponent of 1024 (1024 + R + 128, one byte permute) and narrowed again by adding 1152 and
// taking the low byte of each half.  Messages are in check-row order, edge (b, r) at b*Z + r.
// Each lane of a thread slot holds its own codeword: it converges, writes its outputs and is
// refilled from the work counter independently of the other lane.
#include <cuda_fp16.h>
#include <string.h>

#include "ldpc_internal.h"
#include "layered_pairs.h"

namespace ldpc {

#ifndef LDPC_PAIRS_KMAX
#define LDPC_PAIRS_KMAX 1  // most thread slots in one barrier group (one: every slot runs on its own)
#endif
#ifndef LDPC_PAIRS_REFILL_NOINLINE
#define LDPC_PAIRS_REFILL_NOINLINE 0  // 1: refill / output as out-of-line functions
#endif
#if LDPC_PAIRS_REFILL_NOINLINE
#define LDPC_PAIRS_COLD __device__ __noinline__
#else
#define LDPC_PAIRS_COLD __device__ __forceinline__
#endif
#ifndef LDPC_PAIRS_REFILL_CHUNK
#define LDPC_PAIRS_REFILL_CHUNK 4  // channel values a thread requests at once when a lane takes a codeword
#endif

// One launch decodes every codeword of up to MULTI_MAX_REQS requests of one code: the
// codewords are the items of one work sequence (request i's codewords are items item0 ..
// item0 + n_cw - 1), taken from a global work counter.
struct LayeredPairArgs {
    int llr_type;
    float scale;
    int n_req;
    int64_t n_items;
    int C2, K, TPG;        // thread slots (two codewords each), thread slots per group, threads per group
    int strideA, strideR;  // APP stride (half2 elements) and R stride (byte pairs) per thread slot
    int max_iter, early_exit, msg_sat, app_sat;
    // binary16 pairs: +-msg_sat, +-app_sat, alpha = alpha_num / 2^alpha_shift and -delta =
    // 2^-(alpha_shift + 1) - 1/2, in both halves
    uint32_t sat, nsat, appmax, appmin, alpha, ndelta;
    unsigned long long *next;
    ReqDev reqs[MULTI_MAX_REQS];
};

__device__ __forceinline__ uint32_t h2u(__half2 x) { return *reinterpret_cast<uint32_t *>(&x); }
__device__ __forceinline__ __half2 u2h(uint32_t x) { return *reinterpret_cast<__half2 *>(&x); }

constexpr uint32_t kH1152 = 0x64806480u;    // binary16 1152 in both halves
constexpr uint32_t kH1536 = 0x66006600u;    // 1536
constexpr uint32_t kHm1536 = 0xE600E600u;   // -1536
constexpr uint32_t kHInf = 0x7C007C00u;     // +infinity
constexpr uint32_t kSign2 = 0x80008000u;
constexpr uint32_t kMag2 = 0x7FFF7FFFu;

// R of both codewords of an edge: two biased bytes -> 1024 + (R + 128) in each half
__device__ __forceinline__ __half2 widen_r(uint32_t two_bytes) { return u2h(__byte_perm(two_bytes, 0x64646464u, 0x5140)); }
// R (binary16 pair) -> the two biased bytes (low byte of R + 1152 in each half)
__device__ __forceinline__ uint32_t narrow_r(__half2 r) { return __byte_perm(h2u(__hadd2(r, u2h(kH1152))), 0u, 0x0020); }

// The APP byte offset of edge k of a layer for row r of a thread slot, in one of two forms:
// from the offset table (one 16-bit load: the table holds the offset of every (block, row)), or
// from the layer's edge descriptors (an 8-byte load shared by all rows: .x = offset of block
// column position s, .y = Z - s; row r reaches position r + s, less Z when r >= Z - s).
template <bool TABLE>
struct EdgeAddr;
template <>
struct EdgeAddr<true> {
    const uint16_t *orow;  // row r's entry of the layer's first block; edge k is Z entries further
    int Z;
    __device__ __forceinline__ int operator()(int k) const { return orow[k * Z]; }
};
template <>
struct EdgeAddr<false> {
    const int2 *ed;  // the layer's first block's descriptor
    int rA, r, ZA;   // byte offset of position r, the row, and 4 Z
    __device__ __forceinline__ int operator()(int k) const
    {
        const int2 d = ed[k];
        return rA + d.x - (r >= d.y ? ZA : 0);
    }
};

#ifndef LDPC_PAIRS_FENCE
#define LDPC_PAIRS_FENCE 0  // edges between compiler fences in the unrolled edge loops (0: none)
#endif
// A compiler-only fence every LDPC_PAIRS_FENCE edges: loads are not hoisted across it, which
// bounds how many edges' values the unrolled loops keep live at once.
__device__ __forceinline__ void edge_fence(int k)
{
    if constexpr (LDPC_PAIRS_FENCE > 0)
        if (k % LDPC_PAIRS_FENCE == LDPC_PAIRS_FENCE - 1) asm volatile("" ::: "memory");
}

#ifndef LDPC_PAIRS_BREAK
#define LDPC_PAIRS_BREAK 1  // leave the unrolled edge loops every this many edges once past dc (0: never)
#endif
// Whether an unrolled edge loop is past the row's degree at edge k: every LDPC_PAIRS_BREAK
// edges a warp-uniform test (every row of a layer has the same degree) leaves the loop, so
// the edges of a wide body past dc cost no predicated instructions.  Measured on 65536
// codewords of the N = 1944 rate-5/6 code (rows of degree 18-21 in the degree-24 body): a
// test at every edge 2.15 -> 1.87 ms per decode, every 4 edges 1.92, every 8 edges 2.09,
// bit-identical; it also frees the registers of the skipped edges (80 -> 71, no spill).
__device__ __forceinline__ bool edges_done(int k, int dc)
{
    if constexpr (LDPC_PAIRS_BREAK > 0) return k > 0 && k % LDPC_PAIRS_BREAK == 0 && k >= dc;
    return false;
}

// One check row of a layer for the two codewords of a thread slot (edges past dc skipped under
// a uniform guard).  ea: the edges' APP offsets, Ab: APP base of the slot, Rrow: the byte pairs
// of the layer's first edge of row r (edge k is Z pairs further).  The second pass forms each
// APP offset again rather than holding it.
template <int D, bool SATAPP, bool TABLE>
__device__ __forceinline__ void pair_check(int dc, const EdgeAddr<TABLE> &ea, char *Ab, uint16_t *Rrow, int Z,
                                           const LayeredPairArgs &k_)
{
    uint32_t q[D];
    __half2 mn1 = u2h(kHInf), mn2 = u2h(kHInf);
    uint32_t S = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        if (edges_done(k, dc)) break;
        if (k < dc) {
            const __half2 app = *reinterpret_cast<const __half2 *>(Ab + ea(k));
            const __half2 rb = widen_r(Rrow[k * Z]);
            __half2 qq = __hadd2(__hsub2(app, rb), u2h(kH1152));
            qq = __hmax2(__hmin2(qq, u2h(k_.sat)), u2h(k_.nsat));
            const uint32_t qb = h2u(qq);
            const __half2 mag = u2h(qb & kMag2);
            mn2 = __hmin2(mn2, __hmax2(mn1, mag));
            mn1 = __hmin2(mn1, mag);
            S ^= qb;
            q[k] = qb;
        }
        edge_fence(k);
    }
    // alpha * min as floor(alpha m): round(alpha m - delta) at binary16 spacing 1 (+-1536)
    const __half2 m1 = __hadd2(__hadd2(__hfma2(mn1, u2h(k_.alpha), u2h(k_.ndelta)), u2h(kH1536)), u2h(kHm1536));
    const __half2 m2 = __hadd2(__hadd2(__hfma2(mn2, u2h(k_.alpha), u2h(k_.ndelta)), u2h(kH1536)), u2h(kHm1536));
    const uint32_t Sm = S & kSign2;
    const uint32_t A1 = h2u(m1) ^ Sm, A2 = h2u(m2) ^ Sm;  // magnitudes carrying the sign of the whole check
#pragma unroll
    for (int k = 0; k < D; k++) {
        if (edges_done(k, dc)) break;
        if (k < dc) {
            const uint32_t qb = q[k];
            const uint32_t eq = __heq2_mask(u2h(qb & kMag2), mn1);
            const uint32_t rn = ((eq & A2) | (~eq & A1)) ^ (qb & kSign2);
            __half2 an = __hadd2(u2h(qb), u2h(rn));
            if constexpr (SATAPP) an = __hmax2(__hmin2(an, u2h(k_.appmax)), u2h(k_.appmin));
            Rrow[k * Z] = (uint16_t)narrow_r(u2h(rn));
            *reinterpret_cast<__half2 *>(Ab + ea(k)) = an;
        }
        edge_fence(k);
    }
}

// Parity word (XOR of the APP words: sign bits 15 and 31 are the two codewords') of check row r
// of one block row, edges past dc skipped under a uniform guard.
template <int D, bool TABLE>
__device__ __forceinline__ uint32_t pair_parity(int dc, const EdgeAddr<TABLE> &ea, const char *Ab)
{
    uint32_t par = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        if (edges_done(k, dc)) break;
        if (k < dc) par ^= *reinterpret_cast<const uint32_t *>(Ab + ea(k));
        edge_fence(k);
    }
    return par;
}

__device__ __forceinline__ int sat_q(int x, int s) { return max(-s, min(s, x)); }

// Load codeword k of request rq into lane v of a thread slot, this thread's row r: APP =
// quantised LLRs (+0 for zero) at positions j*Z + r, R = 0 (biased byte 128) for every block;
// the channel values of a chunk are all requested before any is used.
LDPC_PAIRS_COLD void lpair_refill(const LayeredPairArgs &a, const CodeDev *__restrict__ cd, __half *Ah,
                                          uint16_t *Rc, int v, int rq, int k, int r, int N, int Z, int nb, int nnz)
{
    const void *llr = a.reqs[rq].llr;
    constexpr int CH = LDPC_PAIRS_REFILL_CHUNK;
    for (int j0 = 0; j0 < nb; j0 += CH) {
        int q[CH];
        if (a.llr_type == LDPC_LLR_I8) {
            int raw[CH];
#pragma unroll
            for (int w = 0; w < CH; w++)
                if (j0 + w < nb) raw[w] = static_cast<const int8_t *>(llr)[(int64_t)k * N + (j0 + w) * Z + r];
#pragma unroll
            for (int w = 0; w < CH; w++)
                if (j0 + w < nb) {
                    if (raw[w] < -a.msg_sat || raw[w] > a.msg_sat) atomicOr(cd->status, IN_I8_RANGE);
                    q[w] = sat_q(raw[w], a.msg_sat);
                }
        } else {
            float in[CH];
#pragma unroll
            for (int w = 0; w < CH; w++)
                if (j0 + w < nb) in[w] = __ldg(static_cast<const float *>(llr) + (int64_t)k * N + (j0 + w) * Z + r);
#pragma unroll
            for (int w = 0; w < CH; w++)
                if (j0 + w < nb) {
                    if (!isfinite(in[w])) atomicOr(cd->status, IN_NONFINITE);
                    const float rr = rintf(__fmul_rn(a.scale, in[w]));
                    q[w] = rr > (float)a.msg_sat ? a.msg_sat : (rr < -(float)a.msg_sat ? -a.msg_sat : (int)rr);
                }
        }
#pragma unroll
        for (int w = 0; w < CH; w++)
            if (j0 + w < nb) Ah[2 * ((j0 + w) * Z + r) + v] = __int2half_rn(q[w]);
    }
    for (int b = 0; b < nnz; b++) reinterpret_cast<uint8_t *>(Rc + b * Z + r)[v] = 128;
}

// Write lane v's outputs for codeword k of request rq (row r's positions): hard decisions, the
// posterior (if asked for), and, from row 0, the iteration count.
LDPC_PAIRS_COLD void lpair_output(const LayeredPairArgs &a, const __half *Ah, int v, int rq, int k, int t, int r,
                                          int N, int Z, int nb)
{
    const ReqDev &q = a.reqs[rq];
    uint8_t *Bo = q.bits + (int64_t)k * N;
    float *Ao = q.app ? q.app + (int64_t)k * N : nullptr;
    for (int j = 0; j < nb; j++) {
        const __half x = Ah[2 * (j * Z + r) + v];
        Bo[j * Z + r] = (__half_as_ushort(x) & 0x8000u) ? 1 : 0;
        if (Ao) Ao[j * Z + r] = __half2float(x);
    }
    if (r == 0) q.iters[k] = t;
}

// the barrier of one group (named barrier group + 1), or the warp when the group is one warp
__device__ __forceinline__ void pgroup_sync(int grp, int tpg)
{
    if (tpg == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(tpg) : "memory");
}

// Table space (ints) ahead of the slots: the lanes' next and current requests, the block-row pointers, the
// edge descriptors (two ints per block), and with TABLE the APP offset table: entry b*Z + r (16 bits) is the byte offset
// 4 (j Z + (r + s) mod Z) of the position that row r of block b = (row l, column j, shift s)
// reaches, for every thread slot of the CTA.
__host__ __device__ inline int lpairs_tables_ints(int nnz, int mb, int Z, bool table)
{
    return 2 * SLOTS_MAX + mb + 1 + 2 * nnz + (table ? (nnz * Z + 1) / 2 : 0);  // + the lanes' requests
}

// Threads per CTA: up to 1024 for rows of degree <= 16; 768 above, where the register file
// must hold the Q words of up to 32 edges per thread (64 vs 80 registers per thread).
__host__ __device__ constexpr int lpairs_threads(int dmax) { return dmax <= 16 ? 1024 : 768; }

template <int DMAX, bool SATAPP, bool TABLE>
__global__ void __launch_bounds__(lpairs_threads(DMAX), 1) k_layered_pairs(const CodeDev *__restrict__ cd, const __grid_constant__ LayeredPairArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = cd->N, Z = cd->Z, mb = cd->mb, nb = cd->nb, nnz = cd->nnz;
    const int C2 = a.C2, K = a.K, TPG = a.TPG;
    int32_t *bad = reinterpret_cast<int32_t *>(smem);               // [2 * C2] unsatisfied check seen, per codeword
    int32_t *gany = bad + SLOTS_MAX;                                 // [groups][2] group vote
    int64_t *fresh = reinterpret_cast<int64_t *>(gany + SLOTS_MAX);  // [2 * C2] next codeword per lane (request-local)
    int32_t *sreq = reinterpret_cast<int32_t *>(fresh + SLOTS_MAX);   // [2 * C2] its request
    int32_t *creq = sreq + SLOTS_MAX;  // [2 * C2] request of the codeword each lane decodes
    int2 *t_ed = reinterpret_cast<int2 *>(creq + SLOTS_MAX);
    int32_t *t_rowptr = reinterpret_cast<int32_t *>(t_ed + nnz);
    uint16_t *t_off = reinterpret_cast<uint16_t *>(t_rowptr + mb + 1);
    __half2 *APPs = reinterpret_cast<__half2 *>(smem + slots_smem_head(lpairs_tables_ints(nnz, mb, Z, TABLE)));
    uint16_t *Rs = reinterpret_cast<uint16_t *>(APPs + (size_t)C2 * a.strideA);

    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < nnz; i += nth) {
        const int e = cd->ent[i], sh = e & 0xffff;
        t_ed[i] = make_int2(4 * ((e >> 16) * Z + sh), Z - sh);
    }
    if constexpr (TABLE)
        for (int i = tid; i < nnz * Z; i += nth) {
            const int b = i / Z, rr = i - b * Z;
            const int e = cd->ent[b], sh = e & 0xffff;
            const int x = rr + sh;
            t_off[i] = (uint16_t)(4 * ((e >> 16) * Z + (x >= Z ? x - Z : x)));
        }
    for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
    const int g = tid / TPG, u = tid - (tid / TPG) * TPG;
    const int c = g * K + u / Z, r = u - (u / Z) * Z;
    const bool mine = u < K * Z && c < C2;  // a row of a thread slot (else an idle lane of the group)
    if (tid == 0)
        for (int i = 0; i < SLOTS_MAX; i++) gany[i] = 0;
    // a lane's leader takes the next item of the work sequence and finds its request
    auto grab = [&](int lane) {
        const unsigned long long k = atomicAdd(a.next, 1ull);
        int64_t loc = -1;
        int rq = -1;
        if (k < (unsigned long long)a.n_items) {
            for (rq = 0; rq < a.n_req - 1; rq++)
                if ((int64_t)k < a.reqs[rq].item0 + a.reqs[rq].n_cw) break;
            loc = (int64_t)k - a.reqs[rq].item0;
        }
        fresh[lane] = loc;
        sreq[lane] = rq;
    };
    if (mine && r == 0) {
#pragma unroll
        for (int v = 0; v < 2; v++) {
            grab(2 * c + v);
            bad[2 * c + v] = 0;
        }
    }
    __syncthreads();
    if (g * K >= C2) return;  // whole warps beyond the last group
    char *Ab = reinterpret_cast<char *>(APPs + (size_t)(mine ? c : 0) * a.strideA);
    __half *Ah = reinterpret_cast<__half *>(Ab);
    uint16_t *Rc = Rs + (size_t)(mine ? c : 0) * a.strideR;
    // the edges' APP offsets of layer l for this thread's row
    auto edges = [&](int b0) {
        if constexpr (TABLE)
            return EdgeAddr<true>{t_off + b0 * Z + r, Z};
        else
            return EdgeAddr<false>{t_ed + b0, 4 * r, r, 4 * Z};
    };

    int ph = 0;
    auto group_any = [&](bool pred) {
        if (pred) gany[2 * g + ph] = 1;
        pgroup_sync(g, TPG);
        const bool any = gany[2 * g + ph] != 0;
        if (u == 0) gany[2 * g + (ph ^ 1)] = 0;
        ph ^= 1;
        return any;
    };

    // a lane taking codeword fresh / sreq: its request is kept in shared memory (creq, read again
    // at the output), not in registers
    auto take = [&](int v) {
        const int rqv = sreq[2 * c + v];
        if (r == 0) creq[2 * c + v] = rqv;
        lpair_refill(a, cd, Ah, Rc, v, rqv, (int)fresh[2 * c + v], r, N, Z, nb, nnz);
    };
    int cw[2];  // request-local codeword in each lane (-1: empty; requests hold at most 2^31)
    int t[2] = {0, 0};
#pragma unroll
    for (int v = 0; v < 2; v++) {
        cw[v] = mine ? (int)fresh[2 * c + v] : -1;
        if (cw[v] >= 0) take(v);
    }
    if (!group_any(cw[0] >= 0 || cw[1] >= 0)) return;

    for (;;) {
        const bool busy0 = cw[0] >= 0, busy1 = cw[1] >= 0, busy = busy0 || busy1;
        for (int l = 0; l < mb; l++) {
            if (busy) {
                const int b0 = t_rowptr[l], dc = t_rowptr[l + 1] - b0;
                pair_check<DMAX, SATAPP, TABLE>(dc, edges(b0), Ab, Rc + b0 * Z + r, Z, a);
            }
            pgroup_sync(g, TPG);
        }
        t[0] += busy0;
        t[1] += busy1;
        // syndrome of both lanes' hard decisions: row r of every layer
        if (busy && a.early_exit) {
            uint32_t par_any = 0;
            for (int l = 0; l < mb; l++) {
                const int b0 = t_rowptr[l];
                par_any |= pair_parity<DMAX, TABLE>(t_rowptr[l + 1] - b0, edges(b0), Ab);
            }
            if (busy0 && (par_any & 0x8000u)) bad[2 * c] = 1;
            if (busy1 && (par_any & 0x80000000u)) bad[2 * c + 1] = 1;
        }
        pgroup_sync(g, TPG);
        bool done[2];
#pragma unroll
        for (int v = 0; v < 2; v++) {
            done[v] = cw[v] >= 0 && ((a.early_exit && bad[2 * c + v] == 0) || t[v] >= a.max_iter);
            if (done[v]) {
                lpair_output(a, Ah, v, creq[2 * c + v], cw[v], t[v], r, N, Z, nb);
                if (r == 0) grab(2 * c + v);
            }
        }
        pgroup_sync(g, TPG);
#pragma unroll
        for (int v = 0; v < 2; v++) {
            if (cw[v] >= 0 && r == 0) bad[2 * c + v] = 0;
            if (done[v]) {
                cw[v] = (int)fresh[2 * c + v];
                t[v] = 0;
                if (cw[v] >= 0) take(v);
            }
        }
        if (!group_any(cw[0] >= 0 || cw[1] >= 0)) break;
    }
}

// ------------------------------------------------------------------ host side

// Whether the half-precision form computes the integer min-sum exactly for these parameters:
// every message magnitude floor(alpha_num * m / 2^alpha_shift) <= 127 (one biased byte), and
// alpha m - delta exact in binary16 for every m <= msg_sat (its numerator 2 alpha_num m -
// 2^alpha_shift + 1 over 2^(alpha_shift + 1) below 2^11).
bool layered_pairs_exact(const ldpc_decode_params &p)
{
    if (p.msg_sat < 1 || p.msg_sat > 127 || p.app_sat < p.msg_sat || p.app_sat > 127) return false;
    if (p.nms_alpha_shift < 0 || p.nms_alpha_shift > 10 || p.nms_alpha_num < 0) return false;
    const long long top = ((long long)p.nms_alpha_num * p.msg_sat) >> p.nms_alpha_shift;
    if (top > 127) return false;
    return 2LL * p.nms_alpha_num * p.msg_sat + (1LL << p.nms_alpha_shift) <= 2047;
}

// Strides congruent to Z modulo the banks' width in elements (32 words of APP, 64 byte pairs
// of R), so that a warp whose rows run from one thread slot into the next sees one contiguous
// bank sequence.
static int pair_stride(int n, int Z, int m) { return n + (((Z % m) - (n % m)) % m + m) % m; }

#ifndef LDPC_PAIRS_TABLE_MAXD
#define LDPC_PAIRS_TABLE_MAXD 8  // the offset table for codes of row degree up to this, descriptors above
#endif
static bool lpairs_table(const CodeDev &h) { return h.dc_max <= LDPC_PAIRS_TABLE_MAXD; }

static size_t lpairs_smem(const CodeDev &h, int C2)
{
    return slots_smem_head(lpairs_tables_ints(h.nnz, h.mb, h.Z, lpairs_table(h))) +
           (size_t)C2 * ((size_t)pair_stride(h.N, h.Z, 32) * 4 + (size_t)pair_stride(h.E, h.Z, 64) * 2) + 16;
}

struct LpairShape {
    int C2, K, TPG;
};
// Thread slots per CTA and their grouping: the most thread slots that fit 1024 threads, 15
// named barriers and the shared-memory budget, with the fewest per group among the
// arrangements reaching that count.
static LpairShape lpairs_shape(const CodeDev &h, int64_t cap2 = SLOTS_MAX / 2)
{
    LpairShape best = {0, 1, 32};
    if (h.dc_max > 32 || 4 * h.N > 65535) return best;  // APP byte offsets in 16 bits
    const int tmax = lpairs_threads(h.dc_max <= 8 ? 8 : h.dc_max <= 16 ? 16 : h.dc_max <= 24 ? 24 : 32);
    int cmax = SLOTS_MAX / 2;
    while (cmax > 0 && lpairs_smem(h, cmax) > 227 * 1024) cmax--;
    if (cap2 >= 1 && cap2 < cmax) cmax = (int)cap2;
    for (int K = 1; K <= cmax && K <= LDPC_PAIRS_KMAX; K++) {
        const int tpg = ((K * h.Z + 31) / 32) * 32;
        int G = tmax / tpg;
        if (tpg > 32 && G > 15) G = 15;
        int C = G * K;
        if (C > cmax) C = cmax;
        if (C > best.C2) best = {C, K, tpg};
    }
    return best;
}

int layered_pairs_per_cta(const CodeDev &h) { return 2 * lpairs_shape(h).C2; }

template <int DMAX, bool SATAPP, bool TABLE>
static cudaError_t launch_lpairs(const CodeDev &h, const CodeDev *d, const LayeredPairArgs &a, int ctas, cudaStream_t s)
{
    const size_t sm = lpairs_smem(h, a.C2);
    cudaError_t e = ensure_smem<k_layered_pairs<DMAX, SATAPP, TABLE>>(sm);
    if (e != cudaSuccess) return e;
    LaunchScope ls(F_LAYERED, s);
    const int groups = (a.C2 + a.K - 1) / a.K;
    k_layered_pairs<DMAX, SATAPP, TABLE><<<(unsigned)ctas, groups * a.TPG, sm, s>>>(d, a);
    return cudaGetLastError();
}

template <int DMAX, bool SATAPP>
static cudaError_t launch_lpairs_t(const CodeDev &h, const CodeDev *d, const LayeredPairArgs &a, int ctas,
                                   cudaStream_t s)
{
    return lpairs_table(h) ? launch_lpairs<DMAX, SATAPP, true>(h, d, a, ctas, s)
                           : launch_lpairs<DMAX, SATAPP, false>(h, d, a, ctas, s);
}

template <bool SATAPP>
static cudaError_t launch_lpairs_d(const CodeDev &h, const CodeDev *d, const LayeredPairArgs &a, int ctas,
                                   cudaStream_t s)
{
    if (h.dc_max <= 8) return launch_lpairs_t<8, SATAPP>(h, d, a, ctas, s);
    if (h.dc_max <= 16) return launch_lpairs_t<16, SATAPP>(h, d, a, ctas, s);
    if (h.dc_max <= 24) return launch_lpairs_t<24, SATAPP>(h, d, a, ctas, s);
    return launch_lpairs_t<32, SATAPP>(h, d, a, ctas, s);
}

// Decode the codewords of n requests of one code (reqs[i].code all the same) in one launch.
cudaError_t layered_pairs_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p,
                                 const HostReq *reqs, int n, int llr_type, void *counter, cudaStream_t s)
{
    if (!layered_pairs_exact(p) || n < 1 || n > MULTI_MAX_REQS) return cudaErrorInvalidValue;
    LayeredPairArgs a;
    memset(&a, 0, sizeof a);
    int64_t items = 0;
    for (int i = 0; i < n; i++) {
        if (reqs[i].n_cw <= 0) continue;
        ReqDev &q = a.reqs[a.n_req++];
        q.llr = reqs[i].llr;
        q.bits = reqs[i].bits;
        q.iters = reqs[i].iters;
        q.app = reqs[i].app;
        q.n_cw = reqs[i].n_cw;
        q.item0 = items;
        items += reqs[i].n_cw;
    }
    if (items == 0) return cudaSuccess;
    a.n_items = items;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // a small batch spreads over the SMs rather than filling a few CTAs' slots
    const int64_t per_cta = (items + nsm - 1) / nsm;
    const LpairShape sh = lpairs_shape(h, (per_cta + 1) / 2);
    if (sh.C2 < 1) return cudaErrorInvalidValue;
    a.llr_type = llr_type;
    a.scale = p.llr_scale;
    a.C2 = sh.C2;
    a.K = sh.K;
    a.TPG = sh.TPG;
    a.strideA = pair_stride(h.N, h.Z, 32);
    a.strideR = pair_stride(h.E, h.Z, 64);
    a.max_iter = p.max_iter;
    a.early_exit = p.early_exit;
    a.msg_sat = p.msg_sat;
    a.app_sat = p.app_sat;
    auto pair = [](float x) {
        const unsigned short hb = __half_as_ushort(__float2half_rn(x));  // exact for these values
        return (uint32_t)hb | ((uint32_t)hb << 16);
    };
    a.sat = pair((float)p.msg_sat);
    a.nsat = pair(-(float)p.msg_sat);
    a.appmax = pair((float)p.app_sat);
    a.appmin = pair(-(float)p.app_sat);
    a.alpha = pair((float)p.nms_alpha_num / (float)(1 << p.nms_alpha_shift));
    a.ndelta = pair(1.0f / (float)(2 << p.nms_alpha_shift) - 0.5f);
    a.next = static_cast<unsigned long long *>(counter);
    int64_t ctas = nsm;
    const int64_t need = (items + 2 * a.C2 - 1) / (2 * a.C2);
    if (need < ctas) ctas = need;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const long long top = ((long long)p.nms_alpha_num * p.msg_sat) >> p.nms_alpha_shift;
    return p.msg_sat + top > p.app_sat ? launch_lpairs_d<true>(h, d, a, (int)ctas, s)
                                       : launch_lpairs_d<false>(h, d, a, (int)ctas, s);
}

}  // namespace ldpc
