// Flooding sum-product decoding of codes too large for one SM: the cluster slot decoder.
//
// A thread-block cluster of CL CTAs (CL SMs) holds one codeword for the whole decode, split
// between its CTAs: CTA q owns a contiguous range of block rows (their checks and the
// messages R of their edges) and a contiguous range of block columns (their posteriors
// APP).  The two ranges are balanced by block count.  A check of CTA q reads the posteriors
// of its variables wherever they live (distributed shared memory of the cluster); a variable
// of CTA q reads the messages of its edges wherever they live.  One round (Sec. II two-phase
// message passing, Algorithm 1 loop order), each phase closed by a cluster barrier:
//   check-node phase   every owned check: Q = APP - R, R' from the check rule in the product
//                      (tanh) domain of the slot decoders, written in place; the parity of the APP sign
//                      bits over the check flags an unsatisfied check of the previous
//                      iteration's decisions
//   decision           no CTA of the cluster flagged a check and >= 1 iteration done: the
//                      codeword has converged (its APP from that iteration is final)
//   variable-node phase otherwise every owned variable: APP = L + sum of the new R
// A finished codeword is written out and the cluster's leader takes the next codeword from
// the global work counter.  Messages sit in check-row order, edge (b, r) of the owned block b
// at (b - first owned block) * Z + r; posteriors at (j - first owned column) * Z + c.
#include <string.h>

#include <cooperative_groups.h>

#include "slot_common.cuh"

namespace cg = cooperative_groups;

namespace ldpc {

constexpr int CLUSTER_CTAS = 2;

// One launch decodes every codeword of up to MULTI_MAX_REQS requests of one code: the codewords
// are the items of one work sequence (request i's are items item0 .. item0 + n_cw - 1).
struct ClusterArgs {
    int n_req;
    int64_t n_items;
    unsigned long long *next;
    int row_split[CLUSTER_CTAS + 1];  // block rows [row_split[q], row_split[q+1]) belong to CTA q
    int ncols[CLUSTER_CTAS];          // block columns CTA q holds the posteriors of
    int col_owner[NB_MAX];            // owner of block column j
    int col_slot[NB_MAX];             // its place among the owner's columns
    int col_list[CLUSTER_CTAS][NB_MAX];  // CTA q's columns in place order
    int max_iter, early_exit;
    float X;
    ReqDev reqs[MULTI_MAX_REQS];
};

// 32-bit shared::cluster addresses: the address of shared variable p in CTA `rank` of the
// cluster, and loads through such an address (the CTA's own memory or the other's).  Posteriors
// and messages are read this way, so an operand's address is one 32-bit add from a per-owner
// base, whichever CTA holds it.
__device__ __forceinline__ uint32_t cl_map(const void *p, unsigned rank)
{
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(out)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return out;
}
__device__ __forceinline__ float cl_ld(const float *, uint32_t addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ float cl_ld(const __half *, uint32_t addr)
{
    unsigned short v;
    asm volatile("ld.shared::cluster.u16 %0, [%1];" : "=h"(v) : "r"(addr));
    return __half2float(__ushort_as_half(v));
}

__host__ __device__ inline int cl_owner(const int *split, int x)
{
    int q = 0;
    while (q < CLUSTER_CTAS - 1 && x >= split[q + 1]) q++;
    return q;
}

// An owned row of degree <= 8 in the product (tanh) domain (see slot_common.cuh): d_k = e^-a_k
// with a_k = |Q_k| clamped to [phi(X), X], the other edges' maps combined from prefix and
// suffix pairs, R_k = ln(alpha / beta); one ex2 and two lg2 per edge.
template <int D, bool EXACT, typename MsgT>
__device__ __forceinline__ uint32_t cl_check_tanh(int dc, const int4 *__restrict__ ed, MsgT *Rr, uint32_t app_0,
                                                  uint32_t app_1, int r, int Z, float Xb, float Pb)
{
    constexpr uint32_t kSign = 0x80000000u;
    float d[D];
    uint32_t qs[D];
    uint32_t sg = 0, par = 0;
    const uint32_t rb = 4u * (uint32_t)r, ZA = 4u * (uint32_t)Z;
#pragma unroll
    for (int k = 0; k < D; k++) {
        d[k] = 0.0f;  // a missing edge (k >= dc) is the identity map
        qs[k] = 0;
        if (EXACT || k < dc) {
            const int4 e = ed[k];
            const float ap = cl_ld((const float *)nullptr, (e.z ? app_1 : app_0) + e.x + rb - (r >= e.y ? ZA : 0u));
            const float qv = ap - (float)Rr[k * Z];
            par ^= __float_as_uint(ap);
            qs[k] = __float_as_uint(qv) & kSign;
            sg ^= qs[k];
            d[k] = tanh_d<false>(qv, Xb, Pb);
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
            Rr[k * Z] = MsgT(__uint_as_float(__float_as_uint(tanh_mag<false>(al, be)) | (qs[k] ^ sg)));
        }
        if (k == 0) {
            pb = d[0];
        } else if (k < D - 1) {
            const float t = fmaf(d[k], pb, pa);
            pb = fmaf(d[k], pa, pb);
            pa = t;
        }
    }
    return par;
}

// One check of an owned row: Q = APP - R over its edges (posteriors wherever they live), the
// check rule in the product (tanh) domain (slot_common.cuh), messages written in place;
// returns the parity of the posteriors' sign bits.  Rows above degree 8 take the grouped
// form, with Q formed from APP and R in both passes.
template <int D, bool EXACT, typename MsgT>
__device__ __forceinline__ uint32_t cl_check(int dc, const int4 *__restrict__ ed, MsgT *Rr, uint32_t app_0,
                                             uint32_t app_1, int r, int Z, float Xb, float Pb)
{
    if constexpr (D <= 8) {
        return cl_check_tanh<D, EXACT, MsgT>(dc, ed, Rr, app_0, app_1, r, Z, Xb, Pb);
    } else {
        uint32_t par = 0;
        const uint32_t rb = 4u * (uint32_t)r, ZA = 4u * (uint32_t)Z;
        auto qof = [&](int k, bool first) -> float {
            const int4 e = ed[k];
            const float ap = cl_ld((const float *)nullptr, (e.z ? app_1 : app_0) + e.x + rb - (r >= e.y ? ZA : 0u));
            if (first) par ^= __float_as_uint(ap);
            return ap - (float)Rr[k * Z];
        };
        auto put = [&](int k, float m, float) { Rr[k * Z] = MsgT(m); };
        if constexpr (D <= 12)  // hold the factors (no second remote load) where that does not spill
            tanh_check_wide_held<D, false>(dc, Xb, Pb, [&](int k) { return qof(k, true); },
                                           [&](int k, float m) { put(k, m, 0.0f); });
        else
            tanh_check_wide<D, false>(dc, Xb, Pb, qof, put);
        return par;
    }
}

template <int D, int DMAX, typename MsgT>
__device__ __forceinline__ uint32_t cl_check_dispatch(int dc, const int4 *__restrict__ ent, MsgT *Rr,
                                                      uint32_t app_0, uint32_t app_1, int r, int Z, float Xb,
                                                      float Pb)
{
    if constexpr (D >= DMAX) {
        return cl_check<DMAX, false, MsgT>(dc, ent, Rr, app_0, app_1, r, Z, Xb, Pb);
    } else if constexpr (D <= 8) {
        if (dc == D) return cl_check<D, true, MsgT>(dc, ent, Rr, app_0, app_1, r, Z, Xb, Pb);
        return cl_check_dispatch<next_degree(D), DMAX, MsgT>(dc, ent, Rr, app_0, app_1, r, Z, Xb, Pb);
    } else {
        if (dc <= D) return cl_check<D, false, MsgT>(dc, ent, Rr, app_0, app_1, r, Z, Xb, Pb);
        return cl_check_dispatch<next_degree(D), DMAX, MsgT>(dc, ent, Rr, app_0, app_1, r, Z, Xb, Pb);
    }
}

// Sum of the messages of variable position c of one block column (column degree dv; entry
// descriptors cd, see the kernel) onto sum, in the order of the column lists: straight-line
// bodies for the common degrees (every lane of a warp takes the same branch).
template <int D, typename MsgT>
__device__ __forceinline__ float cl_vn_sum(const int4 *__restrict__ cd, uint32_t r_0, uint32_t r_1, int c, int Z,
                                           float sum)
{
    constexpr uint32_t SZ = sizeof(MsgT);
#pragma unroll
    for (int k = 0; k < D; k++) {
        const int4 d = cd[k];
        sum += cl_ld((const MsgT *)nullptr, (d.z ? r_1 : r_0) + d.x + SZ * (uint32_t)c + (c < d.y ? SZ * Z : 0u));
    }
    return sum;
}
template <typename MsgT>
__device__ __forceinline__ float cl_vn_column(int dv, const int4 *__restrict__ cd, uint32_t r_0, uint32_t r_1, int c,
                                              int Z, float sum)
{
    constexpr uint32_t SZ = sizeof(MsgT);
    switch (dv) {
    case 2: return cl_vn_sum<2, MsgT>(cd, r_0, r_1, c, Z, sum);
    case 3: return cl_vn_sum<3, MsgT>(cd, r_0, r_1, c, Z, sum);
    case 4: return cl_vn_sum<4, MsgT>(cd, r_0, r_1, c, Z, sum);
    default:
        for (int k = 0; k < dv; k++) {
            const int4 d = cd[k];
            sum += cl_ld((const MsgT *)nullptr, (d.z ? r_1 : r_0) + d.x + SZ * (uint32_t)c + (c < d.y ? SZ * Z : 0u));
        }
        return sum;
    }
}

// Shared memory ahead of the posterior array: flags and codeword (16 bytes), the block-row
// and block-column pointers, then two descriptors (int4) per block.
__host__ __device__ inline size_t cl_tables_bytes(int nnz)
{
    return (((size_t)16 + 4 * (MB_MAX + 1 + NB_MAX + 1) + 15) & ~(size_t)15) + (size_t)32 * nnz;
}

// threads per CTA: higher check degrees keep more values live per thread
template <int DMAX>
constexpr int cl_threads() { return DMAX <= 8 ? 1024 : (DMAX <= 16 ? 768 : 512); }

template <int DMAX, typename MsgT>
__global__ void __cluster_dims__(CLUSTER_CTAS, 1, 1) __launch_bounds__(cl_threads<DMAX>(), 1)
    k_flood_cluster(const CodeDev *__restrict__ cd, const __grid_constant__ ClusterArgs a)
{
    constexpr uint32_t kSign = 0x80000000u;
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int tid = threadIdx.x, nth = blockDim.x;
    const int Z = cd->Z, mb = cd->mb, nb = cd->nb, nnz = cd->nnz;
    const float Xb = a.X * kSLog2e, Pb = s_phi_b2(a.X);  // the clamp [phi(X), X] in base-2 units

    // bookkeeping: [0] bad flags (2, alternating by round), [2] the codeword being decoded
    // (int64 at 8: request << 32 | request-local index, -1 when the work is done)
    int32_t *flags = reinterpret_cast<int32_t *>(smem);
    int64_t *cwp = reinterpret_cast<int64_t *>(smem + 8);
    int32_t *t_rowptr = reinterpret_cast<int32_t *>(smem + 16);  // [mb + 1]
    int32_t *t_colptr = t_rowptr + MB_MAX + 1;                    // [nb + 1]
    // check-node descriptor of block b = (row l, column j, shift s): .x = the posterior
    // index of position s of column j in its owner, .y = Z - s, .z = the owner; check row r
    // reads .x + r, less Z when r >= .y.  Variable-node descriptor of the i-th entry of the
    // column lists (block b, shift s): .x = the index of b's message row in its owner, less
    // s, .y = s, .z = the owner; variable position c reads .x + c, plus Z when c < .y
    // (message row (c - s) mod Z, which holds the edge of variable c).
    int4 *t_ed = reinterpret_cast<int4 *>(smem + (((size_t)16 + 4 * (MB_MAX + 1 + NB_MAX + 1) + 15) & ~(size_t)15));
    int4 *t_cd = t_ed + nnz;
    const int row0 = a.row_split[q], row1 = a.row_split[q + 1];
    // block b's owner of posteriors and its base there; column entry's owner of messages
    for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
    for (int i = tid; i <= nb; i += nth) t_colptr[i] = cd->colptr[i];
    __syncthreads();
    const int blk0 = t_rowptr[row0], blk1 = t_rowptr[row1];
    for (int b = tid; b < nnz; b += nth) {
        const int e = cd->ent[b];
        const int j = e >> 16, s = e & 0xffff;
        t_ed[b] = make_int4(4 * (a.col_slot[j] * Z + s), Z - s, a.col_owner[j], 0);
    }
    for (int i = tid; i < nnz; i += nth) {
        const int ce = cd->colent[i];
        const int b = ce >> 16, s = ce & 0xffff;
        int l = 0;
        while (l < mb - 1 && b >= cd->rowptr[l + 1]) l++;
        const int qo = cl_owner(a.row_split, l);
        t_cd[i] = make_int4((int)sizeof(MsgT) * ((b - cd->rowptr[a.row_split[qo]]) * Z - s), s, qo, 0);
    }
    const size_t off_app = cl_tables_bytes(nnz);
    float *app = reinterpret_cast<float *>(smem + off_app);
    // R starts at the same offset in every CTA (after the largest posterior share), so that
    // mapping an address into another CTA of the cluster finds that CTA's messages
    int napp_max = 0;
#pragma unroll
    for (int k = 0; k < CLUSTER_CTAS; k++) napp_max = a.ncols[k] * Z > napp_max ? a.ncols[k] * Z : napp_max;
    MsgT *R = reinterpret_cast<MsgT *>(smem + off_app + (((size_t)napp_max * 4 + 15) & ~(size_t)15));
    // the cluster's posterior and message arrays, by owning CTA (generic pointers; the own
    // CTA's are plain shared memory)
    static_assert(CLUSTER_CTAS == 2, "the owner selects below assume two CTAs");
    const uint32_t app_0 = cl_map(app, 0), app_1 = cl_map(app, 1);
    const uint32_t r_0 = cl_map(R, 0), r_1 = cl_map(R, 1);
    const int n_var = a.ncols[q] * Z;
    // The check and variable loops without a division per item: thread tid works on position
    // tid mod Z of block rows / columns tid / Z, tid / Z + RS, ... (RS = nth / Z rows per pass;
    // threads beyond RS * Z idle there).  When Z exceeds the thread count (RS = 0), thread tid
    // works on positions tid, tid + nth, ... of every block row / column instead.
    const int RS = nth / Z;
    const int p0 = RS > 0 ? tid % Z : tid, ps = RS > 0 ? Z : nth;     // positions
    const int l0 = RS > 0 ? tid / Z : 0, ls = RS > 0 ? RS : 1;        // block rows / columns
    const bool works = RS == 0 || tid / Z < RS;
    const int *my_cols = a.col_list[q];
    int64_t *cw0 = cluster.map_shared_rank(cwp, 0);
    cluster.sync();  // tables built in every CTA before any remote access

    for (;;) {
        // the leader (CTA 0, thread 0) takes the next codeword; every CTA reads it
        if (q == 0 && tid == 0) {
            const unsigned long long k = atomicAdd(a.next, 1ull);
            int64_t v = -1;
            if (k < (unsigned long long)a.n_items) {
                int rq = 0;
                while (rq < a.n_req - 1 && (int64_t)k >= a.reqs[rq].item0 + a.reqs[rq].n_cw) rq++;
                v = ((int64_t)rq << 32) | ((int64_t)k - a.reqs[rq].item0);
            }
            cwp[0] = v;
        }
        cluster.sync();  // also: no CTA still reads another's flags of the previous codeword
        const int64_t item = *cw0;
        if (item < 0) break;
        const ReqDev &req = a.reqs[(int)(item >> 32)];
        const int64_t cw = item & 0xffffffffll;
        if (tid == 0) flags[0] = flags[1] = 0;
        // load: APP = L (+0: no -0) for owned variables, R = 0 for owned edges
        const float *L = static_cast<const float *>(req.llr) + cw * cd->N;
        for (int i = tid; i < n_var; i += nth) {
            const int jl = i / Z, c = i - jl * Z;
            const float v = __ldg(L + my_cols[jl] * Z + c);
            if (!isfinite(v)) atomicOr(cd->status, IN_NONFINITE);
            app[i] = v + 0.0f;
        }
        for (int i = tid; i < (blk1 - blk0) * Z; i += nth) R[i] = MsgT(0.0f);
        cluster.sync();
        int t = 0;
        bool done = false;
        while (!done) {
            const int tr = t;  // this round's flag is flags[tr & 1]
            // ---------------- check-node phase over the owned checks
            bool pbad = false;
            auto check_row = [&](int lr, int r) {
                const int l = row0 + lr;
                const int b0 = t_rowptr[l];
                const uint32_t par = cl_check_dispatch<2, DMAX, MsgT>(t_rowptr[l + 1] - b0, t_ed + b0,
                                                                      R + (b0 - blk0) * Z + r, app_0, app_1, r, Z,
                                                                      Xb, Pb);
                pbad |= (par & kSign) != 0;
            };
            for (int r = p0; works && r < Z; r += ps)
                for (int lr = l0; lr < row1 - row0; lr += ls) check_row(lr, r);
            if (pbad) flags[tr & 1] = 1;
            cluster.sync();
            // ---------------- decision (the same in every CTA: all flags are read after the barrier)
            bool any_bad = false;
#pragma unroll
            for (int k = 0; k < CLUSTER_CTAS; k++) any_bad |= cluster.map_shared_rank(flags, k)[tr & 1] != 0;
            const bool conv = tr >= 1 && a.early_exit && !any_bad;
            if (!conv) {
                // ---------------- variable-node phase over the owned variables
                auto var_col = [&](int jl, int c) {
                    const int j = my_cols[jl];
                    const int e0 = t_colptr[j];
                    const float sum = cl_vn_column<MsgT>(t_colptr[j + 1] - e0, t_cd + e0, r_0, r_1, c, Z,
                                                         __ldg(L + j * Z + c));
                    app[jl * Z + c] = sum + 0.0f;  // -0 -> +0: the sign bit is the decision
                };
                for (int c = p0; works && c < Z; c += ps)
                    for (int jl = l0; jl < a.ncols[q]; jl += ls) var_col(jl, c);
                t++;
            }
            done = conv || t >= a.max_iter;
            // the other flag was read by every CTA in the previous round (before this round's
            // first barrier): clear it for the next round, which writes it after the barrier below
            if (tid == 0) flags[(tr + 1) & 1] = 0;
            cluster.sync();
        }
        // output: each CTA writes its variables
        uint8_t *Bo = req.bits + cw * cd->N;
        float *Ao = req.app ? req.app + cw * cd->N : nullptr;
        for (int i = tid; i < n_var; i += nth) {
            const int jl = i / Z, c = i - jl * Z;
            const int n = my_cols[jl] * Z + c;
            const float v = app[i];
            Bo[n] = v < 0.0f ? 1 : 0;
            if (Ao) Ao[n] = v;
        }
        if (q == 0 && tid == 0) req.iters[cw] = t;
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}


// ------------------------------------------------------------------ host side

// bytes of the table area ahead of APP (the kernel's layout)

// Split the block rows between the cluster's CTAs in contiguous ranges of about equal block
// counts, then give each block column to the CTA that owns most of its blocks' rows (its
// posteriors are then read locally by most of its checks), moving the least attached columns
// while a CTA would need more shared memory than the largest allowed.  Returns the per-CTA
// shared memory (the same layout in every CTA), or 0 if no assignment fits.
static size_t cl_plan(const CodeDev &h, int msg, ClusterArgs &a, size_t limit)
{
    a.row_split[0] = 0;
    for (int q = 1; q < CLUSTER_CTAS; q++) {
        const int want = (int)((int64_t)h.nnz * q / CLUSTER_CTAS);
        int l = a.row_split[q - 1] + 1;
        while (l < h.mb && h.rowptr[l] < want) l++;
        a.row_split[q] = l < h.mb ? l : h.mb - 1;
    }
    a.row_split[CLUSTER_CTAS] = h.mb;
    const size_t msz = msg == LDPC_MSG_F16 ? sizeof(__half) : sizeof(float);
    size_t nr = 0;
    for (int q = 0; q < CLUSTER_CTAS; q++) {
        const size_t nm = (size_t)(h.rowptr[a.row_split[q + 1]] - h.rowptr[a.row_split[q]]) * h.Z;
        nr = nm > nr ? nm : nr;
    }
    // affinity of column j to CTA q: its blocks in q's rows
    int aff[NB_MAX][CLUSTER_CTAS] = {};
    for (int j = 0; j < h.nb; j++)
        for (int i = h.colptr[j]; i < h.colptr[j + 1]; i++) {
            const int b = h.colent[i] >> 16;
            int l = 0;
            while (l < h.mb - 1 && b >= h.rowptr[l + 1]) l++;
            aff[j][cl_owner(a.row_split, l)]++;
        }
    int cnt[CLUSTER_CTAS] = {};
    for (int j = 0; j < h.nb; j++) {
        int best = 0;
        for (int q = 1; q < CLUSTER_CTAS; q++)
            if (aff[j][q] > aff[j][best] || (aff[j][q] == aff[j][best] && cnt[q] < cnt[best])) best = q;
        a.col_owner[j] = best;
        cnt[best]++;
    }
    // the posterior share of a CTA may not exceed what its shared memory has left
    const size_t fixed = cl_tables_bytes(h.nnz) + nr * msz;
    const int cap = limit > fixed ? (int)((limit - fixed) / (4 * (size_t)h.Z)) : 0;
    for (int q = 0; q < CLUSTER_CTAS; q++) {
        while (cnt[q] > cap) {
            // move q's column with the least attachment to q to the CTA with the most room
            int jm = -1;
            for (int j = 0; j < h.nb; j++)
                if (a.col_owner[j] == q && (jm < 0 || aff[j][q] < aff[jm][q])) jm = j;
            int to = -1;
            for (int k = 0; k < CLUSTER_CTAS; k++)
                if (k != q && cnt[k] < cap && (to < 0 || cnt[k] < cnt[to])) to = k;
            if (jm < 0 || to < 0) return 0;
            a.col_owner[jm] = to;
            cnt[q]--;
            cnt[to]++;
        }
    }
    for (int q = 0; q < CLUSTER_CTAS; q++) a.ncols[q] = 0;
    for (int j = 0; j < h.nb; j++) {
        const int q = a.col_owner[j];
        a.col_slot[j] = a.ncols[q];
        a.col_list[q][a.ncols[q]++] = j;
    }
    int nmax = 0;
    for (int q = 0; q < CLUSTER_CTAS; q++) nmax = a.ncols[q] > nmax ? a.ncols[q] : nmax;
    return cl_tables_bytes(h.nnz) + (((size_t)nmax * h.Z * 4 + 15) & ~(size_t)15) + nr * msz;
}

static size_t cl_limit()
{
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return lim > 0 ? (size_t)lim : 227 * 1024;
}

int cluster_supported(const CodeDev &h, int msg)
{
    if (h.dc_max > 32 || h.mb < CLUSTER_CTAS || h.nb < CLUSTER_CTAS) return 0;
    if ((int64_t)h.N >= (1 << 19) || (int64_t)h.E >= (1 << 20))
        return 0;  // the packed table fields (posterior and message bases)
    ClusterArgs a;
    memset(&a, 0, sizeof a);
    const size_t need = cl_plan(h, msg, a, cl_limit());
    return need > 0 && need <= cl_limit();
}

template <int DMAX, typename MsgT>
static cudaError_t launch_cluster(const ClusterArgs &a, size_t smem, int64_t n_cw, const CodeDev *d, cudaStream_t s)
{
    cudaError_t e = ensure_smem<k_flood_cluster<DMAX, MsgT>>(smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLUSTER_CTAS, 1, 1);
    cfg.blockDim = dim3(cl_threads<DMAX>(), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    // clusters that fit the device at once, queried once per device and shared-memory size
    static int cached[64];
    static size_t cached_smem[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int clusters = __atomic_load_n(&cached[dev], __ATOMIC_RELAXED);
    if (clusters < 1 || __atomic_load_n(&cached_smem[dev], __ATOMIC_RELAXED) != smem) {
        e = cudaOccupancyMaxActiveClusters(&clusters, k_flood_cluster<DMAX, MsgT>, &cfg);
        if (e != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            int nsm = 2;
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            clusters = nsm / CLUSTER_CTAS;
        }
        __atomic_store_n(&cached_smem[dev], smem, __ATOMIC_RELAXED);
        __atomic_store_n(&cached[dev], clusters, __ATOMIC_RELAXED);
    }
    if ((int64_t)clusters > n_cw) clusters = (int)n_cw;
    LaunchScope ls(F_SLOTS, s);
    k_flood_cluster<DMAX, MsgT><<<(unsigned)(clusters * CLUSTER_CTAS), cl_threads<DMAX>(), smem, s>>>(d, a);
    return cudaGetLastError();
}

cudaError_t flood_cluster_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const HostReq *reqs,
                                 int n, void *counter, cudaStream_t s)
{
    if (n < 1 || n > MULTI_MAX_REQS) return cudaErrorInvalidValue;
    ClusterArgs a;
    memset(&a, 0, sizeof a);
    const size_t smem = cl_plan(h, p.msg, a, cl_limit());
    if (smem == 0) return cudaErrorInvalidValue;
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
    a.next = static_cast<unsigned long long *>(counter);
    a.max_iter = p.max_iter;
    a.early_exit = p.early_exit;
    a.X = p.phi_clamp;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool f16 = p.msg == LDPC_MSG_F16;
    if (h.dc_max <= 8)
        return f16 ? launch_cluster<8, __half>(a, smem, items, d, s) : launch_cluster<8, float>(a, smem, items, d, s);
    if (h.dc_max <= 16)
        return f16 ? launch_cluster<16, __half>(a, smem, items, d, s) : launch_cluster<16, float>(a, smem, items, d, s);
    return f16 ? launch_cluster<32, __half>(a, smem, items, d, s) : launch_cluster<32, float>(a, smem, items, d, s);
}

}  // namespace ldpc
