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
//   check-node phase   every busy slot: Q = APP - R, R' from the check rule in the product
//                      (tanh) domain (slot_common.cuh), written in place; the parity of the hard decisions
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
//   barrier (with the "any slot busy" vote)
// Codewords therefore leave as soon as they converge and free slots are refilled at once:
// early exit saves whole rounds of work instead of idling lanes of a tile.
//
// Single slots (one codeword per thread) run the rounds in lock-step over the whole CTA.
// Paired slots (two codewords per thread) run them in barrier groups: a group's thread slots
// have their rows packed into whole warps and synchronise on their own named barrier, so
// the groups of a CTA run their rounds independently; the host forms groups only where
// they need no more warps than one lock-step group.
//
// One launch serves several requests (mixed codes): requests of the same code form a
// group with its own work counter; each CTA starts on a group chosen in proportion to the
// groups' work, and when its group runs dry and its slots have drained it reloads the code
// tables and layout of the group with the most codewords left.  A single batch is the
// one-group case.
#include <string.h>

#include "slot_common.cuh"

namespace ldpc {

// Channel values a thread loads at once when a slot takes a codeword: 8, and 12 for single
// slots of codes of row degree <= 8, which have the registers for it (measured 1.2 % faster on
// the N = 1944 rate-1/2 sweep; 12 costs paired slots 2 % there, and wider instances spill).
#ifndef LDPC_REFILL_CHUNK
#define LDPC_REFILL_CHUNK 8
#endif
#ifndef LDPC_REFILL_CHUNK_NARROW
#define LDPC_REFILL_CHUNK_NARROW 12
#endif

// Per-slot strides of APP and R (elements): at least the length, and congruent to Z modulo
// the 32 shared-memory banks, so that a warp whose rows run from the end of one slot group
// into the start of the next sees the two groups' rows as one contiguous bank sequence.
__host__ __device__ inline int slot_stride(int n, int Z) { return n + ((Z % 32) - (n % 32) + 32) % 32; }

struct FloodMultiArgs {
    MultiDesc d;
    unsigned long long *next;  // [n_groups] work counters, zero at launch
    int tbl_ints;              // table space reserved (max over groups), in int32
    int max_iter, early_exit;
    float X;
};

// The check-node phase of one thread for codes of row degree <= 8: row r of every W-th block
// row from w0 (in degree order), one loop per degree over the rows of that degree (exact
// bodies, no per-row dispatch; the branch above degree 8 serves wider instances).  Flooding
// checks are independent, so the order of the rows changes no result.
template <int D, int DMAX, int V, typename MsgT>
__device__ __forceinline__ void cn_rows(const int32_t *t_rord, const int32_t *t_dbeg, const int32_t *t_rowptr,
                                        const int4 *__restrict__ t_ed, const char *Ar, char *Rr, int r, int ZA,
                                        int ZR, float Xb, float Pb, uint32_t (&pbad)[V], int w0, int W)
{
    if constexpr (D <= 8) {
        if constexpr (D <= DMAX) {
            const int i1 = t_dbeg[D - 1];
            for (int i = t_dbeg[D - 2] + w0; i < i1; i += W)
                slot_check_v<D, true, V, MsgT>(D, t_ed + t_rowptr[t_rord[i]], Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
        }
        cn_rows<D + 1, DMAX, V, MsgT>(t_rord, t_dbeg, t_rowptr, t_ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad, w0, W);
    } else if constexpr (DMAX > 8) {
        const int i1 = t_dbeg[8];
        for (int i = t_dbeg[7] + w0; i < i1; i += W) {
            const int l = t_rord[i], b0 = t_rowptr[l];
            slot_check_dispatch<12, DMAX, V, MsgT>(t_rowptr[l + 1] - b0, t_ed + b0, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
        }
    }
}

// Sum of the messages of one variable (column degree dv, message offsets ce) into sacc, in
// the order of the column lists.  The common degrees get straight-line bodies; every lane
// of a warp takes the same branch (a warp covers one block column).
// (messages in base-2 units when kSlotB2: each is added as R ln 2)
template <typename MsgT>
__device__ __forceinline__ float vn_add(float s, float rv)
{
    return kSlotB2<MsgT> ? fmaf(rv, kSLn2, s) : s + rv;
}
template <int D, int V, typename MsgT>
__device__ __forceinline__ void vn_sum(const int32_t *__restrict__ ce, const char *Rr, float (&sacc)[V])
{
#pragma unroll
    for (int k = 0; k < D; k++) {
        float rv[V];
        SMsg<MsgT, V>::ld(at<MsgT>(Rr, ce[k]), rv);
#pragma unroll
        for (int v = 0; v < V; v++) sacc[v] = vn_add<MsgT>(sacc[v], rv[v]);
    }
}
template <int V, typename MsgT>
__device__ __forceinline__ void vn_column(int dv, const int32_t *__restrict__ ce, const char *Rr, float (&sacc)[V])
{
    if (dv == 3)
        vn_sum<3, V, MsgT>(ce, Rr, sacc);
    else if (dv == 2)
        vn_sum<2, V, MsgT>(ce, Rr, sacc);
    else if (dv == 4)
        vn_sum<4, V, MsgT>(ce, Rr, sacc);
    else
        for (int i = 0; i < dv; i++) {
            float rv[V];
            SMsg<MsgT, V>::ld(at<MsgT>(Rr, ce[i]), rv);
#pragma unroll
            for (int v = 0; v < V; v++) sacc[v] = vn_add<MsgT>(sacc[v], rv[v]);
        }
}

// Barrier groups of a CTA: named barriers 1..15 (barrier 0 is the CTA's).
constexpr int FLOOD_GROUPS_MAX = 15;

template <int DMAX, int V, typename MsgT, bool SPREAD>
__global__ void __launch_bounds__(slot_threads_max<V>(), 1) k_flood_slots(const __grid_constant__ FloodMultiArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *bad = reinterpret_cast<int32_t *>(smem);            // [SLOTS_MAX] unsatisfied check seen this round
    int32_t *sreq = bad + SLOTS_MAX;                             // [SLOTS_MAX] request of the next codeword
    int64_t *fresh = reinterpret_cast<int64_t *>(sreq + SLOTS_MAX);  // [SLOTS_MAX] next codeword (request-local)
    int32_t *misc = reinterpret_cast<int32_t *>(fresh + SLOTS_MAX);  // [4] code-group hand-over
    int4 *t_ed = reinterpret_cast<int4 *>(misc + 4);  // 16-byte aligned: the head is a multiple of 16 bytes
    float *APPs = reinterpret_cast<float *>(smem + slots_smem_head(a.tbl_ints));

    const int tid = threadIdx.x, nth = blockDim.x;
    const float Xb = a.X * kSLog2e, Pb = s_phi_b2(a.X);  // the clamp [phi(X), X] in base-2 units
    constexpr uint32_t kSign = 0x80000000u;
    int grp = 0;
    {
        const float u = (blockIdx.x + 0.5f) / gridDim.x;
        while (grp < a.d.n_groups - 1 && a.d.groups[grp].cumw < u) grp++;
    }

    for (;;) {
        const GroupDev &gd = a.d.groups[grp];
        const CodeDev *cd = gd.code;
        const int N = gd.N, Z = gd.Z, mb = gd.mb, nb = gd.nb, nnz = gd.nnz;
        const int C = gd.C, G = gd.C / V;
        const int strideA = slot_stride(N, Z), strideR = slot_stride(gd.E, Z);
        MsgT *Rs = reinterpret_cast<MsgT *>(APPs + (((size_t)C * strideA + 3) & ~(size_t)3));
        int32_t *t_colent = reinterpret_cast<int32_t *>(t_ed + nnz);
        int32_t *t_rowptr = t_colent + nnz;
        int32_t *t_colptr = t_rowptr + mb + 1;
        // tables, pre-scaled to byte offsets from a thread's own bases (position r of slot
        // group g): t_ed[b] is the edge descriptor of block b (see EdgeRef); t_colent[i] is
        // the message offset of block row-major index b*Z for the i-th block of the column
        // lists.  Messages are stored at the variable's position inside its block: edge
        // (b, r) of check row r lives at b*Z + (r + s) mod Z, so the check-node phase
        // computes the wrap once for both addresses and the variable-node phase, summing
        // column position r of block column j, reads b*Z + r.
        constexpr int SA = (int)sizeof(float) * V, SR = (int)sizeof(MsgT) * V;
        for (int i = tid; i < nnz; i += nth) {
            const int e = cd->ent[i], j = e >> 16, sh = e & 0xffff;
            t_ed[i] = make_int4(SA * (j * Z + sh), SR * (i * Z + sh), Z - sh, 0);
            t_colent[i] = SR * (cd->colent[i] >> 16) * Z;
        }
        for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
        for (int i = tid; i <= nb; i += nth) t_colptr[i] = cd->colptr[i];
        // block rows ordered by degree (the check-node phase runs one loop per degree up to 8,
        // so that a row needs no degree dispatch): t_rord[t_dbeg[d - 2] .. t_dbeg[d - 1]) are
        // the rows of degree d, t_rord[t_dbeg[7] .. mb) those above degree 8
        int32_t *t_rord = t_colptr + nb + 1, *t_dbeg = t_rord + mb;
        for (int i = tid; i < mb; i += nth) t_rord[i] = cd->rord[i];
        for (int i = tid; i < 9; i += nth) t_dbeg[i] = cd->dbeg[i];
        // barrier group bg of this thread (paired slots, V = 2): K thread slots whose K*Z rows
        // are packed into TPG threads (whole warps); thread u of the group owns row u mod Z of
        // thread slot bg*K + u / Z.  Single slots (V = 1) run as one lock-step group of the
        // whole CTA: thread tid owns row tid mod Z of thread slot tid / Z.
        const int K = V == 2 ? gd.K : G, TPG = V == 2 ? gd.TPG : nth;
        const int bg = V == 2 ? tid / TPG : 0, u = V == 2 ? tid - bg * TPG : tid;
        // single slots spread over W groups of Z threads: thread u is group w0 = (u / Z) mod W
        // of slot (u / Z) / W and works on block rows and columns w0, w0 + W, ... at position r
        const int W = SPREAD ? gd.W : 1;  // a compile-time 1 unless spread (no loop strides to pay)
        const int g = bg * K + (SPREAD ? u / (Z * W) : u / Z), r = u - (u / Z) * Z;
        const int w0 = SPREAD ? (u / Z) % W : 0;
        const bool mine = g < G && (V == 1 || u < K * Z);
        const bool member = bg * K < G;  // the group has slots (else whole idle warps)
        const bool lead = r == 0 && w0 == 0;  // the thread that takes codewords for the slot

        // a slot's leader takes the group's next codeword and finds its request
        auto grab = [&](int s) {
            const unsigned long long k = atomicAdd(a.next + grp, 1ull);
            int64_t loc = -1;
            int rq = -1;
            if (k < (unsigned long long)gd.n_items) {
                for (rq = gd.req_begin; rq < gd.req_end - 1; rq++)
                    if ((int64_t)k < a.d.reqs[rq].item0 + a.d.reqs[rq].n_cw) break;
                loc = (int64_t)k - a.d.reqs[rq].item0;
            }
            fresh[s] = loc;
            sreq[s] = rq;
        };
        if (mine && lead) {
#pragma unroll
            for (int v = 0; v < V; v++) {
                grab(g * V + v);
                bad[g * V + v] = 0;
            }
        }
        __syncthreads();

        float *A = APPs + (size_t)(mine ? g : 0) * strideA * V;
        MsgT *Rc = Rs + (size_t)(mine ? g : 0) * strideR * V;
        const char *Ar = reinterpret_cast<const char *>(A + r * V);
        char *Rr = reinterpret_cast<char *>(Rc + r * V);
        const int ZA = SA * Z, ZR = SR * Z;
        int64_t cw[V];  // request-local codeword in each of this thread's slots (-1: empty)
        int rq[V];      // its request
        int t[V];       // iterations completed on it
#pragma unroll
        for (int v = 0; v < V; v++) {
            cw[v] = mine ? fresh[g * V + v] : -1;
            rq[v] = mine ? sreq[g * V + v] : -1;
            t[v] = 0;
        }

        // load a new codeword into slot v, this thread's columns: APP = L (+0 for -0), R = 0
        auto refill = [&](int v) {
            const float *Lr = static_cast<const float *>(a.d.reqs[rq[v]].llr) + cw[v] * N;
            constexpr int CH = (V == 1 && DMAX <= 8) ? LDPC_REFILL_CHUNK_NARROW : LDPC_REFILL_CHUNK;
            for (int j0 = w0; j0 < nb; j0 += CH * W) {
                float x[CH];
#pragma unroll
                for (int u = 0; u < CH; u++)
                    if (j0 + u * W < nb) x[u] = __ldg(Lr + (j0 + u * W) * Z + r);
#pragma unroll
                for (int u = 0; u < CH; u++)
                    if (j0 + u * W < nb) {
                        if (!isfinite(x[u])) atomicOr(cd->status, IN_NONFINITE);
                        A[((j0 + u * W) * Z + r) * V + v] = x[u] + 0.0f;
                    }
            }
            for (int b = w0; b < nnz; b += W) {
                if constexpr (sizeof(MsgT) == 2)
                    Rc[(b * Z + r) * V + v] = __float2half_rn(0.0f);
                else
                    Rc[(b * Z + r) * V + v] = 0.0f;
            }
        };

        // the barrier of this thread's group, and the barrier that also returns the OR of a
        // predicate over the group (bar.red: a reduction on a named barrier)
        auto gsync = [&]() {
            if constexpr (V == 1)
                __syncthreads();
            else if (TPG == 32)
                __syncwarp();
            else
                asm volatile("bar.sync %0, %1;" ::"r"(bg + 1), "r"(TPG) : "memory");
        };
        auto group_any = [&](bool pred) -> bool {
            if constexpr (V == 1) return __syncthreads_or(pred) != 0;
            if (TPG == 32) {
                __syncwarp();
                return __any_sync(0xffffffffu, pred);
            }
            int any_set;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
                "selp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(any_set)
                : "r"((unsigned)pred), "r"(bg + 1), "r"(TPG)
                : "memory");
            return any_set != 0;
        };

        bool any = false;
#pragma unroll
        for (int v = 0; v < V; v++) {
            if (cw[v] >= 0) refill(v);
            any |= cw[v] >= 0;
        }
        any = V == 1 ? __syncthreads_or(any) != 0 : member && group_any(any);

        while (any) {
            // ---------------- check-node phase: row r of every block row, all V slots at once
            if (mine && (cw[0] >= 0 || (V > 1 && cw[V - 1] >= 0))) {
                uint32_t pbad[V];
#pragma unroll
                for (int v = 0; v < V; v++) pbad[v] = 0;
                if constexpr (DMAX == 8) {
                    cn_rows<2, DMAX, V, MsgT>(t_rord, t_dbeg, t_rowptr, t_ed, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad, w0, W);
                } else {
                    // codes with rows above degree 8: per-row dispatch in row order (measured
                    // faster here than the per-degree loops on the mixed-code launch)
                    for (int l = w0; l < mb; l += W) {
                        const int b0 = t_rowptr[l], dc = t_rowptr[l + 1] - b0;
                        slot_check_dispatch<2, DMAX, V, MsgT>(dc, t_ed + b0, Ar, Rr, r, ZA, ZR, Xb, Pb, pbad);
                    }
                }
#pragma unroll
                for (int v = 0; v < V; v++)
                    if (cw[v] >= 0 && (pbad[v] & kSign)) bad[g * V + v] = 1;
            }
            gsync();

            // ---------------- decision, variable-node phase, output
            bool done[V];
            bool act[V];
            bool anyact = false;
#pragma unroll
            for (int v = 0; v < V; v++) {
                const bool conv = mine && cw[v] >= 0 && t[v] >= 1 && a.early_exit && bad[g * V + v] == 0;
                act[v] = mine && cw[v] >= 0 && !conv;
                done[v] = conv;
                anyact |= act[v];
            }
            if (anyact) {
                for (int j0 = w0; j0 < nb; j0 += 4 * W) {
                    float lv[4][V];
#pragma unroll
                    for (int u = 0; u < 4; u++)
#pragma unroll
                        for (int v = 0; v < V; v++)
                            if (j0 + u * W < nb && act[v])
                                lv[u][v] = __ldg(static_cast<const float *>(a.d.reqs[rq[v]].llr) + cw[v] * N +
                                                 (j0 + u * W) * Z + r);
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int j = j0 + u * W;
                        if (j < nb) {
                            float sacc[V];
#pragma unroll
                            for (int v = 0; v < V; v++) sacc[v] = lv[u][v];
                            const int i0 = t_colptr[j];
                            vn_column<V, MsgT>(t_colptr[j + 1] - i0, t_colent + i0, Rr, sacc);
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
                    const ReqDev &q = a.d.reqs[rq[v]];
                    uint8_t *Bo = q.bits + cw[v] * N;
                    float *Ao = q.app ? q.app + cw[v] * N : nullptr;
                    for (int j = w0; j < nb; j += W) {
                        const float x = A[(j * Z + r) * V + v];
                        Bo[j * Z + r] = x < 0.0f ? 1 : 0;
                        if (Ao) Ao[j * Z + r] = x;
                    }
                    if (lead) {
                        q.iters[cw[v]] = t[v];
                        grab(g * V + v);
                    }
                }
            }
            gsync();

            // ---------------- refill finished slots
            any = false;
            if (mine) {
#pragma unroll
                for (int v = 0; v < V; v++) {
                    if (lead) bad[g * V + v] = 0;
                    if (done[v]) {
                        cw[v] = fresh[g * V + v];
                        rq[v] = sreq[g * V + v];
                        t[v] = 0;
                        if (cw[v] >= 0) refill(v);
                    }
                    any |= cw[v] >= 0;
                }
            }
            any = group_any(any);
        }

        // this group is dry here and every slot has drained: move to the group with the
        // most codewords left, or stop
        if (tid == 0) {
            int best = -1;
            long long most = 0;
            for (int q = 0; q < a.d.n_groups; q++) {
                const long long left = a.d.groups[q].n_items - (long long)atomicAdd(a.next + q, 0ull);
                if (left > most) {
                    most = left;
                    best = q;
                }
            }
            misc[0] = best;
        }
        __syncthreads();
        grp = misc[0];
        __syncthreads();
        if (grp < 0) return;
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

static size_t max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? (size_t)v : 227 * 1024;
}

static int tables_ints(const CodeDev &h) { return 5 * h.nnz + h.mb + 1 + h.nb + 1 + h.mb + 9; }

// Shared memory of C slots of a code: the APP region (16-byte aligned end) and the messages.
static size_t slots_bytes(const CodeDev &h, int msg, int C)
{
    const size_t sa = ((size_t)C * slot_stride(h.N, h.Z) * sizeof(float) + 15) & ~(size_t)15;
    return sa + (size_t)C * slot_stride(h.E, h.Z) * (msg == LDPC_MSG_F16 ? sizeof(__half) : sizeof(float));
}

// Slots of one code per CTA with V codewords per thread, given the table space reserved.
static int slots_for(const CodeDev &h, int msg, int V, int tbl_ints, size_t limit)
{
    if (h.dc_max > 32 || h.N >= 65536) return 0;
    int C = (int)((V == 2 ? slot_threads_max<2>() : slot_threads_max<1>()) / h.Z) * V;
    if (C > SLOTS_MAX) C = SLOTS_MAX;
    while (C > 0 && slots_smem_head(tbl_ints) + slots_bytes(h, msg, C) > limit) C--;
    C -= C % V;
    return C;
}

int slots_supported(const CodeDev &h, int msg) { return slots_for(h, msg, 1, tables_ints(h), 227 * 1024) > 0; }

int slots_pairable(const CodeDev &h, int msg) { return slots_for(h, msg, 2, tables_ints(h), max_smem_optin()) >= 2; }

// Codewords per thread: two when pairing the slots of the first code costs no slot and no
// check has degree above 16 (high-degree checks keep too many values live per edge to pair).
#ifndef LDPC_SLOTS_V
#define LDPC_SLOTS_V 2
#endif
static int choose_v(const CodeDev &h, int msg, int tbl_ints, size_t limit)
{
    if (LDPC_SLOTS_V < 2 || h.dc_max > 16) return 1;
    const int c1 = slots_for(h, msg, 1, tbl_ints, limit), c2 = slots_for(h, msg, 2, tbl_ints, limit);
    return (c2 >= 2 && c2 >= c1) ? 2 : 1;
}

template <int DMAX, int V, typename MsgT, bool SPREAD = false>
static cudaError_t launch_multi(const FloodMultiArgs &a, size_t smem, int threads, int ctas, cudaStream_t s)
{
    cudaError_t e = ensure_smem<k_flood_slots<DMAX, V, MsgT, SPREAD>>(smem);
    if (e != cudaSuccess) return e;
    LaunchScope ls(F_SLOTS, s);
    k_flood_slots<DMAX, V, MsgT, SPREAD><<<(unsigned)ctas, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// spread: single slots of a small batch whose block rows and columns are spread over W > 1
// thread groups (V = 1 only)
template <typename MsgT>
static cudaError_t launch_multi_d(int dmax, int V, bool spread, const FloodMultiArgs &a, size_t smem, int threads,
                                  int ctas, cudaStream_t s)
{
    if (spread) {
        if (dmax <= 8) return launch_multi<8, 1, MsgT, true>(a, smem, threads, ctas, s);
        if (dmax <= 16) return launch_multi<16, 1, MsgT, true>(a, smem, threads, ctas, s);
        if (dmax <= 24) return launch_multi<24, 1, MsgT, true>(a, smem, threads, ctas, s);
        return launch_multi<32, 1, MsgT, true>(a, smem, threads, ctas, s);
    }
    if (dmax <= 8)
        return V == 2 ? launch_multi<8, 2, MsgT>(a, smem, threads, ctas, s)
                      : launch_multi<8, 1, MsgT>(a, smem, threads, ctas, s);
    if (dmax <= 16)
        return V == 2 ? launch_multi<16, 2, MsgT>(a, smem, threads, ctas, s)
                      : launch_multi<16, 1, MsgT>(a, smem, threads, ctas, s);
    if (dmax <= 24)
        return V == 2 ? launch_multi<24, 2, MsgT>(a, smem, threads, ctas, s)
                      : launch_multi<24, 1, MsgT>(a, smem, threads, ctas, s);
    return V == 2 ? launch_multi<32, 2, MsgT>(a, smem, threads, ctas, s)
                  : launch_multi<32, 1, MsgT>(a, smem, threads, ctas, s);
}

// Group the requests by code object, size every group's slots for a common shared-memory
// layout and launch one persistent grid over all of them.
cudaError_t flood_multi_decode(const HostReq *reqs, int n, const ldpc_decode_params &p, void *counters, cudaStream_t s)
{
    FloodMultiArgs a;  // ~7 KB, passed by value as the kernel parameter
    memset(&a, 0, sizeof a);
    const size_t limit = max_smem_optin();
    int ng = 0, nr = 0;
    const ldpc_code *codes[MULTI_MAX_GROUPS];
    for (int i = 0; i < n; i++) {
        if (reqs[i].n_cw <= 0) continue;
        int g = 0;
        while (g < ng && codes[g] != reqs[i].code) g++;
        if (g == ng) {
            if (ng == MULTI_MAX_GROUPS) return cudaErrorInvalidValue;
            codes[ng++] = reqs[i].code;
        }
    }
    if (ng == 0) return cudaSuccess;
    int tbl = 0, dmax = 0;
    for (int g = 0; g < ng; g++) {
        tbl = tables_ints(codes[g]->host) > tbl ? tables_ints(codes[g]->host) : tbl;
        dmax = codes[g]->host.dc_max > dmax ? codes[g]->host.dc_max : dmax;
    }
    const int tuned = codes[0]->tuned_flood[p.msg == LDPC_MSG_F16 ? 1 : 0];
    int V = tuned == SCHED_SLOTS_V2 ? 2 : tuned == SCHED_SLOTS_V1 ? 1 : choose_v(codes[0]->host, p.msg, tbl, limit);
    if (!tuned && dmax > 16) V = 1;
    // a small batch (every group's codewords per SM leave room to spread a single slot over at
    // least two thread groups) decodes in single slots spread over the threads: lower latency
    bool small = !tuned;
    for (int g = 0; g < ng && small; g++) {
        int64_t items = 0;
        for (int i = 0; i < n; i++)
            if (reqs[i].n_cw > 0 && reqs[i].code == codes[g]) items += reqs[i].n_cw;
        const int64_t per_sm = (items + sm_count() - 1) / sm_count();
        small = per_sm * 2 * codes[g]->host.Z <= slot_threads_max<1>() && codes[g]->host.mb >= 2;
    }
    if (small) V = 1;
    for (int g = 0; g < ng && V == 2; g++)
        if (slots_for(codes[g]->host, p.msg, 2, tbl, limit) < 2) V = 1;
    size_t smem = 0;
    int threads = 32;
    double wsum = 0.0;
    int64_t min_ctas = 0;
    for (int g = 0; g < ng; g++) {
        const CodeDev &h = codes[g]->host;
        GroupDev &gd = a.d.groups[g];
        gd.code = codes[g]->dev;
        gd.C = slots_for(h, p.msg, V, tbl, limit);
        if (gd.C < V) return cudaErrorInvalidValue;
        {
            // a small batch spreads over the SMs rather than filling a few CTAs' slots
            int64_t items = 0;
            for (int i = 0; i < n; i++)
                if (reqs[i].n_cw > 0 && reqs[i].code == codes[g]) items += reqs[i].n_cw;
            int64_t cap = (items + sm_count() - 1) / sm_count();
            cap = ((cap + V - 1) / V) * V;
            if (cap < gd.C) gd.C = (int)cap;
        }
        gd.N = h.N;
        gd.E = h.E;
        gd.Z = h.Z;
        gd.mb = h.mb;
        gd.nb = h.nb;
        gd.nnz = h.nnz;
        gd.dc_max = h.dc_max;
        gd.req_begin = nr;
        int64_t items = 0;
        for (int i = 0; i < n; i++) {
            if (reqs[i].n_cw <= 0 || reqs[i].code != codes[g]) continue;
            ReqDev &q = a.d.reqs[nr++];
            q.llr = reqs[i].llr;
            q.bits = reqs[i].bits;
            q.iters = reqs[i].iters;
            q.app = reqs[i].app;
            q.n_cw = reqs[i].n_cw;
            q.item0 = items;
            items += reqs[i].n_cw;
        }
        gd.req_end = nr;
        gd.n_items = items;
        const size_t sm = slots_smem_head(tbl) + slots_bytes(h, p.msg, gd.C);
        smem = sm > smem ? sm : smem;
        // barrier groups (paired slots): the smallest group of thread slots whose whole-warp
        // groups need no more threads than one lock-step group of all of them (the idle lanes
        // of a group are only those of its last warp); one group when none does, and always
        // for single slots
        const int G = gd.C / V;
        // single slots of a small batch (slots capped below what the threads allow) spread each
        // slot's block rows and columns over W groups of Z threads, up to the thread budget; other
        // launches keep W = 1 and the kernel instance without the spread
        gd.W = 1;
        if (small) {
            const int wmax = slot_threads_max<1>() / (G * h.Z);
            gd.W = wmax < 1 ? 1 : (wmax > h.mb ? h.mb : wmax);
        }
        const int t0 = ((G * gd.W * h.Z + 31) / 32) * 32;
        gd.K = G;
        gd.TPG = t0;
        for (int k = 1; V == 2 && k < G; k++) {
            const int tp = ((k * h.Z + 31) / 32) * 32, ng = (G + k - 1) / k;
            if (ng <= FLOOD_GROUPS_MAX && ng * tp <= t0) {
                gd.K = k;
                gd.TPG = tp;
                break;
            }
        }
        const int th = ((G + gd.K - 1) / gd.K) * gd.TPG;
        threads = th > threads ? th : threads;
        wsum += (double)items * h.E;
        min_ctas += (items + gd.C - 1) / gd.C;
    }
    double acc = 0.0;
    for (int g = 0; g < ng; g++) {
        acc += (double)a.d.groups[g].n_items * a.d.groups[g].E;
        a.d.groups[g].cumw = (float)(acc / wsum);
    }
    a.d.groups[ng - 1].cumw = 1.0f;
    a.d.n_groups = ng;
    a.next = static_cast<unsigned long long *>(counters);
    a.tbl_ints = tbl;
    a.max_iter = p.max_iter;
    a.early_exit = p.early_exit;
    a.X = p.phi_clamp;
    int ctas = sm_count();
    if (min_ctas < ctas) ctas = (int)min_ctas;
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * ng, s);
    if (e != cudaSuccess) return e;
    bool spread = false;
    for (int g = 0; g < ng; g++) spread |= a.d.groups[g].W > 1;
    return p.msg == LDPC_MSG_F16 ? launch_multi_d<__half>(dmax, V, spread, a, smem, threads, ctas, s)
                                 : launch_multi_d<float>(dmax, V, spread, a, smem, threads, ctas, s);
}

}  // namespace ldpc
