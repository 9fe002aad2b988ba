// Horizontal layered normalised min-sum in saturated 8-bit arithmetic on sm_103a
// (Sec. II "Algorithm 2": the checks of a layer are computed from the current variable
// values and those values are updated at once; Sec. III-A frame-level parallelism).
//
// One CTA decodes C codewords from start to finish with all decoder state on chip:
// posterior APP int8 [C][N] and check-to-variable messages R int8 [C][E] in shared
// memory; HBM sees only the channel LLRs in and the hard decisions / iteration counts
// out.  Thread (c, r) owns row r of every block row (layer) of codeword c.  In a QC
// layer the Z checks touch disjoint variables (each block is one circulant), so the Z
// row threads of a codeword update a layer concurrently; a CTA barrier separates layers.
//
// Arithmetic per check, every step in int32 then saturated exactly as specified:
//   Q_k   = sat(APP_n - R_k, msg_sat)
//   min1  = smallest |Q|, min2 = second smallest (duplicates counted), arg = first edge
//           attaining min1 (if two edges tie then min2 = min1 and the choice is immaterial)
//   S     = XOR of the signs [Q_k < 0]
//   R_k   = +-((alpha_num * (k == arg ? min2 : min1)) >> alpha_shift), negative iff
//           S xor [Q_k < 0]
//   APP_n = sat(Q_k + R_k, app_sat)
// After every iteration the hard decisions [APP < 0] are checked against all checks; a
// codeword with zero syndrome stops and reports that iteration (early exit).
#include <string.h>

#include "ldpc_internal.h"

namespace ldpc {

__device__ __forceinline__ int sat_i(int x, int s) { return max(-s, min(s, x)); }

struct LayeredArgs {
    const void *llr;
    int llr_type;
    float scale;
    int64_t n_cw;
    int C;
    int max_iter, early_exit, alpha_num, alpha_shift, msg_sat, app_sat;
    uint8_t *bits;
    int32_t *iters;
    float *app_out;
};

template <int DMAX>
__global__ void __launch_bounds__(512) k_layered_nms(const CodeDev *__restrict__ cd, LayeredArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = cd->N, E = cd->E, Z = cd->Z, mb = cd->mb;
    const int C = a.C;
    const int strideA = (N + 15) & ~15, strideR = (E + 15) & ~15;
    int8_t *APP = reinterpret_cast<int8_t *>(smem);
    int8_t *Rm = APP + (size_t)C * strideA;
    int *flag = reinterpret_cast<int *>(Rm + (size_t)C * strideR);  // [C] syndrome failure flags
    int *active = flag + C;                                          // [C] 1 while decoding
    int *its = active + C;                                           // [C] iterations run
    const int64_t cw0 = (int64_t)blockIdx.x * C;
    const int tid = threadIdx.x, nth = blockDim.x;

    // load + quantise the channel LLRs, clear the messages
    for (int i = tid; i < C * N; i += nth) {
        const int c = i / N, n = i - c * N;
        const int64_t cw = cw0 + c;
        int q = 0;
        if (cw < a.n_cw) {
            if (a.llr_type == LDPC_LLR_I8) {
                const int raw = static_cast<const int8_t *>(a.llr)[cw * N + n];
                if (raw < -a.msg_sat || raw > a.msg_sat) atomicOr(cd->status, IN_I8_RANGE);
                q = sat_i(raw, a.msg_sat);
            } else {
                const float in = static_cast<const float *>(a.llr)[cw * N + n];
                if (!isfinite(in)) atomicOr(cd->status, IN_NONFINITE);
                const float p = __fmul_rn(a.scale, in);
                const float rr = rintf(p);
                q = rr > (float)a.msg_sat ? a.msg_sat : (rr < -(float)a.msg_sat ? -a.msg_sat : (int)rr);
            }
        }
        APP[c * strideA + n] = (int8_t)q;
    }
    for (int i = tid; i < C * strideR / 4; i += nth) reinterpret_cast<int *>(Rm)[i] = 0;
    for (int c = tid; c < C; c += nth) {
        flag[c] = 0;
        active[c] = (cw0 + c) < a.n_cw ? 1 : 0;
        its[c] = a.max_iter;
    }
    __syncthreads();

    const int c = tid / Z, r = tid - (tid / Z) * Z;
    const bool mine = c < C;
    int8_t *A = APP + (mine ? c : 0) * strideA;
    int8_t *Rc = Rm + (mine ? c : 0) * strideR;

    for (int t = 1; t <= a.max_iter; t++) {
        for (int l = 0; l < mb; l++) {
            const int b0 = cd->rowptr[l], dc = cd->rowptr[l + 1] - b0;
            if (mine && active[c]) {
                int q[DMAX];
                int min1 = 0x7fffffff, min2 = 0x7fffffff, arg = -1;
                unsigned S = 0;
#pragma unroll
                for (int k = 0; k < DMAX; k++) {
                    if (k < dc) {
                        const int ent = cd->ent[b0 + k];
                        int x = r + (ent & 0xffff);
                        x -= (x >= Z) ? Z : 0;
                        const int n = (ent >> 16) * Z + x;
                        const int qq = sat_i((int)A[n] - (int)Rc[(b0 + k) * Z + r], a.msg_sat);
                        const int mag = qq < 0 ? -qq : qq;
                        if (mag < min1) {
                            min2 = min1;
                            min1 = mag;
                            arg = k;
                        } else if (mag < min2) {
                            min2 = mag;
                        }
                        S ^= qq < 0 ? 1u : 0u;
                        q[k] = qq;
                    }
                }
#pragma unroll
                for (int k = 0; k < DMAX; k++) {
                    if (k < dc) {
                        const int ent = cd->ent[b0 + k];
                        int x = r + (ent & 0xffff);
                        x -= (x >= Z) ? Z : 0;
                        const int n = (ent >> 16) * Z + x;
                        const int mag = (k == arg) ? min2 : min1;
                        const int magp = (a.alpha_num * mag) >> a.alpha_shift;
                        const int rn = (S ^ (q[k] < 0 ? 1u : 0u)) ? -magp : magp;
                        Rc[(b0 + k) * Z + r] = (int8_t)rn;
                        A[n] = (int8_t)sat_i(q[k] + rn, a.app_sat);
                    }
                }
            }
            __syncthreads();
        }
        if (!a.early_exit) continue;
        // syndrome of the hard decisions: thread (c, r) checks row r of every layer
        if (mine && active[c]) {
            unsigned bad = 0;
            for (int l = 0; l < mb && !bad; l++) {
                const int b0 = cd->rowptr[l], b1 = cd->rowptr[l + 1];
                unsigned par = 0;
                for (int b = b0; b < b1; b++) {
                    const int ent = cd->ent[b];
                    int x = r + (ent & 0xffff);
                    x -= (x >= Z) ? Z : 0;
                    par ^= A[(ent >> 16) * Z + x] < 0 ? 1u : 0u;
                }
                bad |= par;
            }
            if (bad) flag[c] = 1;
        }
        __syncthreads();
        int still = 0;
        for (int cc = 0; cc < C; cc++) still |= active[cc] && flag[cc];
        __syncthreads();
        if (tid < C) {
            if (active[tid] && !flag[tid]) {
                its[tid] = t;
                active[tid] = 0;
            }
            flag[tid] = 0;
        }
        __syncthreads();
        if (!still) break;
    }

    // hard decisions, posterior and iteration counts out (row-contiguous in HBM)
    for (int i = tid; i < C * N; i += nth) {
        const int cc = i / N, n = i - cc * N;
        const int64_t cw = cw0 + cc;
        if (cw >= a.n_cw) continue;
        const int v = APP[cc * strideA + n];
        a.bits[cw * N + n] = v < 0 ? 1 : 0;
        if (a.app_out) a.app_out[cw * N + n] = (float)v;
    }
    for (int cc = tid; cc < C; cc += nth)
        if (cw0 + cc < a.n_cw) a.iters[cw0 + cc] = its[cc];
}

// ------------------------------------------------------------------ slot decoder

// Persistent form: one CTA per SM holds C codeword slots (APP and R of each in shared
// memory), arranged in barrier groups of K slots.  A group's threads cover its K*Z check rows
// packed into whole warps; thread u of a group owns row u mod Z of slot u / Z, for every
// layer.  A group's own barrier (a named barrier, or the warp itself when the group is one
// warp) separates its layers, so the slots of a group run in lock-step while the groups run
// independently: K trades the idle lanes of a warp-aligned slot (Z not a multiple of 32)
// against waiting for the slowest slot of a group.  Messages are stored in check-row order,
// edge (b, r) at b*Z + r (contiguous for the row threads; the layered schedule has no
// variable-node pass).  After every full iteration each slot's hard decisions are checked
// against all of its checks; a slot that converged (or reached max_iter) writes its outputs
// and takes the next codeword from the global work counter at the group's next iteration.
// One launch decodes every codeword of up to MULTI_MAX_REQS requests of one code, the items of
// one work sequence (request i's codewords are items item0 .. item0 + n_cw - 1).
struct LayeredSlotArgs {
    int llr_type;
    float scale;
    int n_req;
    int64_t n_items;
    int C, K, TPG, strideA, strideR;  // slots, slots per group, threads per group, strides
    int max_iter, early_exit, alpha_num, alpha_shift, msg_sat, app_sat;
    unsigned long long *next;
    ReqDev reqs[MULTI_MAX_REQS];
};

// The barrier of one group: its warps only (named barrier group + 1; barrier 0 is the CTA's),
// or nothing beyond the warp itself when the group is one warp.
__device__ __forceinline__ void lgroup_sync(int grp, int tpg)
{
    if (tpg == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "r"(tpg) : "memory");
}

// Parity of the hard decisions (APP < 0) of check row r of one block row (degree dc):
// straight-line bodies for the common degrees (every lane of a warp takes the same branch).
template <int D>
__device__ __forceinline__ unsigned lslots_parity(const int2 *__restrict__ ed, const int8_t *A, int r, int Z)
{
    unsigned par = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
        const int2 d = ed[k];
        par ^= A[r + d.x - (r >= d.y ? Z : 0)] < 0 ? 1u : 0u;
    }
    return par;
}
__device__ __forceinline__ unsigned lslots_row_parity(int dc, const int2 *__restrict__ ed, const int8_t *A, int r,
                                                      int Z)
{
    switch (dc) {
    case 4: return lslots_parity<4>(ed, A, r, Z);
    case 5: return lslots_parity<5>(ed, A, r, Z);
    case 6: return lslots_parity<6>(ed, A, r, Z);
    case 7: return lslots_parity<7>(ed, A, r, Z);
    case 8: return lslots_parity<8>(ed, A, r, Z);
    default: {
        unsigned par = 0;
        for (int k = 0; k < dc; k++) {
            const int2 d = ed[k];
            par ^= A[r + d.x - (r >= d.y ? Z : 0)] < 0 ? 1u : 0u;
        }
        return par;
    }
    }
}

// Table space (ints) ahead of the slots: the slots' next and current requests, two per block for
// its edge descriptor, then the block-row pointers.
__host__ __device__ inline int lslots_tables_ints(int nnz, int mb) { return 2 * SLOTS_MAX + 2 * nnz + mb + 1; }

template <int DMAX>
__global__ void __launch_bounds__(1024, 1) k_layered_slots(const CodeDev *__restrict__ cd,
                                                           const __grid_constant__ LayeredSlotArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = cd->N, Z = cd->Z, mb = cd->mb, nb = cd->nb, nnz = cd->nnz;
    const int C = a.C, K = a.K, TPG = a.TPG;
    int32_t *bad = reinterpret_cast<int32_t *>(smem);                 // [SLOTS_MAX] unsatisfied check seen
    int32_t *gany = bad + SLOTS_MAX;                                   // [SLOTS_MAX / 2][2] group vote
    int64_t *fresh = reinterpret_cast<int64_t *>(gany + SLOTS_MAX);    // [SLOTS_MAX] next codeword (request-local)
    int32_t *sreq = reinterpret_cast<int32_t *>(fresh + SLOTS_MAX);    // [SLOTS_MAX] its request
    int32_t *creq = sreq + SLOTS_MAX;                                   // [SLOTS_MAX] request being decoded
    // edge descriptor of block b = (row l, column j, shift s): .x = j*Z + s, .y = Z - s; check
    // row r reaches APP offset r + .x, less Z when r >= .y (position (r + s) mod Z of column j)
    int2 *t_ed = reinterpret_cast<int2 *>(creq + SLOTS_MAX);
    int32_t *t_rowptr = reinterpret_cast<int32_t *>(t_ed + nnz);
    int8_t *APPs = reinterpret_cast<int8_t *>(smem + slots_smem_head(lslots_tables_ints(nnz, mb)));
    int8_t *Rs = APPs + (size_t)C * a.strideA;

    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < nnz; i += nth) {
        const int e = cd->ent[i], sh = e & 0xffff;
        t_ed[i] = make_int2((e >> 16) * Z + sh, Z - sh);
    }
    for (int i = tid; i <= mb; i += nth) t_rowptr[i] = cd->rowptr[i];
    const int g = tid / TPG, u = tid - (tid / TPG) * TPG;
    const int c = g * K + u / Z, r = u - (u / Z) * Z;
    const bool mine = u < K * Z && c < C;  // a row of a slot (else an idle lane of the group)
    if (tid == 0)
        for (int i = 0; i < SLOTS_MAX; i++) gany[i] = 0;
    // a slot's leader takes the next item of the work sequence and finds its request
    auto grab = [&]() {
        const unsigned long long k = atomicAdd(a.next, 1ull);
        int64_t loc = -1;
        int rq = -1;
        if (k < (unsigned long long)a.n_items) {
            for (rq = 0; rq < a.n_req - 1; rq++)
                if ((int64_t)k < a.reqs[rq].item0 + a.reqs[rq].n_cw) break;
            loc = (int64_t)k - a.reqs[rq].item0;
        }
        fresh[c] = loc;
        sreq[c] = rq;
    };
    if (mine && r == 0) {
        grab();
        bad[c] = 0;
    }
    __syncthreads();
    if (g * K >= C) return;  // whole warps beyond the last group
    int8_t *A = APPs + (size_t)(mine ? c : 0) * a.strideA;
    int8_t *Rc = Rs + (size_t)(mine ? c : 0) * a.strideR;
    int ph = 0;
    // OR of a predicate over the group (every thread of the group calls it at the same
    // point; the vote alternates between two words so that clearing the next one races with
    // nothing)
    auto group_any = [&](bool pred) {
        if (pred) gany[2 * g + ph] = 1;
        lgroup_sync(g, TPG);
        const bool any = gany[2 * g + ph] != 0;
        if (u == 0) gany[2 * g + (ph ^ 1)] = 0;
        ph ^= 1;
        return any;
    };

    // load codeword k of request rq (the request is kept in shared memory, creq, for the output)
    auto refill = [&](int64_t k) {
        const int rq = sreq[c];
        if (r == 0) creq[c] = rq;
        const void *llr = a.reqs[rq].llr;
        for (int j = 0; j < nb; j++) {
            const int64_t i = k * N + j * Z + r;
            int q;
            if (a.llr_type == LDPC_LLR_I8) {
                const int raw = static_cast<const int8_t *>(llr)[i];
                if (raw < -a.msg_sat || raw > a.msg_sat) atomicOr(cd->status, IN_I8_RANGE);
                q = sat_i(raw, a.msg_sat);
            } else {
                const float in = __ldg(static_cast<const float *>(llr) + i);
                if (!isfinite(in)) atomicOr(cd->status, IN_NONFINITE);
                const float rr = rintf(__fmul_rn(a.scale, in));
                q = rr > (float)a.msg_sat ? a.msg_sat : (rr < -(float)a.msg_sat ? -a.msg_sat : (int)rr);
            }
            A[j * Z + r] = (int8_t)q;
        }
        for (int b = 0; b < nnz; b++) Rc[b * Z + r] = 0;
    };

    int64_t cw = mine ? fresh[c] : -1;
    int t = 0;
    if (cw >= 0) refill(cw);
    if (!group_any(cw >= 0)) return;

    for (;;) {
        const bool busy = cw >= 0;
        for (int l = 0; l < mb; l++) {
            if (busy) {
                const int b0 = t_rowptr[l], dc = t_rowptr[l + 1] - b0;
                int8_t *Rr = Rc + b0 * Z + r;
                int qx[DMAX];  // (APP offset << 8) | (Q & 0xff): one register per edge (N < 2^16)
                int min1 = 0x7fffffff, min2 = 0x7fffffff, arg = -1;
                unsigned S = 0;
#pragma unroll
                for (int k = 0; k < DMAX; k++) {
                    if (k < dc) {
                        const int2 d = t_ed[b0 + k];
                        const int ao = r + d.x - (r >= d.y ? Z : 0);
                        const int qq = sat_i((int)A[ao] - (int)Rr[k * Z], a.msg_sat);
                        const int mag = qq < 0 ? -qq : qq;
                        if (mag < min1) {
                            min2 = min1;
                            min1 = mag;
                            arg = k;
                        } else if (mag < min2) {
                            min2 = mag;
                        }
                        S ^= qq < 0 ? 1u : 0u;
                        qx[k] = (ao << 8) | (qq & 0xff);
                    }
                }
                const int m1 = (a.alpha_num * min1) >> a.alpha_shift;
                const int m2 = (a.alpha_num * min2) >> a.alpha_shift;
#pragma unroll
                for (int k = 0; k < DMAX; k++) {
                    if (k < dc) {
                        const int qq = (int)(int8_t)(qx[k] & 0xff);
                        const int magp = (k == arg) ? m2 : m1;
                        const int rn = (S ^ (qq < 0 ? 1u : 0u)) ? -magp : magp;
                        Rr[k * Z] = (int8_t)rn;
                        A[qx[k] >> 8] = (int8_t)sat_i(qq + rn, a.app_sat);
                    }
                }
            }
            lgroup_sync(g, TPG);
        }
        if (busy) t++;
        // syndrome of the hard decisions: row r of every layer
        if (busy && a.early_exit) {
            unsigned par_any = 0;
            for (int l = 0; l < mb; l++) {
                const int b0 = t_rowptr[l];
                par_any |= lslots_row_parity(t_rowptr[l + 1] - b0, t_ed + b0, A, r, Z);
            }
            if (par_any) bad[c] = 1;
        }
        lgroup_sync(g, TPG);
        bool done = false;
        if (busy) {
            done = (a.early_exit && bad[c] == 0) || t >= a.max_iter;
            if (done) {
                const ReqDev &q = a.reqs[creq[c]];
                uint8_t *Bo = q.bits + cw * N;
                float *Ao = q.app ? q.app + cw * N : nullptr;
                for (int j = 0; j < nb; j++) {
                    const int v = A[j * Z + r];
                    Bo[j * Z + r] = v < 0 ? 1 : 0;
                    if (Ao) Ao[j * Z + r] = (float)v;
                }
                if (r == 0) {
                    q.iters[cw] = t;
                    grab();
                }
            }
        }
        lgroup_sync(g, TPG);
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

static int pick_C(const CodeDev &h) { return h.Z >= 512 ? 1 : (512 / h.Z); }

static size_t layered_smem(const CodeDev &h, int C)
{
    return (size_t)C * (((h.N + 15) & ~15) + ((h.E + 15) & ~15)) + 3 * sizeof(int) * C;
}

int layered_supported(const CodeDev &h)
{
    return h.Z <= 512 && h.dc_max <= 32 && layered_smem(h, 1) <= 200 * 1024;
}

template <int DMAX>
static cudaError_t launch_layered(const CodeDev &h, const CodeDev *d, const LayeredArgs &a, cudaStream_t s)
{
    const size_t sm = layered_smem(h, a.C);
    cudaError_t e = ensure_smem<k_layered_nms<DMAX>>(sm);
    if (e != cudaSuccess) return e;
    const int threads = ((a.C * h.Z + 31) / 32) * 32;
    const unsigned blocks = (unsigned)((a.n_cw + a.C - 1) / a.C);
    LaunchScope ls(F_LAYERED, s);
    k_layered_nms<DMAX><<<blocks, threads, sm, s>>>(d, a);
    return cudaGetLastError();
}

static size_t lslots_smem(const CodeDev &h, int C)
{
    return slots_smem_head(lslots_tables_ints(h.nnz, h.mb)) + (size_t)C * (((h.N + 15) & ~15) + ((h.E + 15) & ~15));
}

// Slots per CTA and their grouping: the most slots that fit 1024 threads, 15 named barriers
// and the shared-memory budget, with the fewest slots per group among the arrangements that
// reach that count (fewer idle lanes first, then more independence).
struct LslotShape {
    int C, K, TPG;
};
static LslotShape lslots_shape(const CodeDev &h, int64_t cap = SLOTS_MAX)
{
    LslotShape best = {0, 1, 32};
    if (h.dc_max > 32 || h.N >= 65536) return best;
    int cmax = SLOTS_MAX;
    while (cmax > 0 && lslots_smem(h, cmax) > 200 * 1024) cmax--;
    if (cap >= 1 && cap < cmax) cmax = (int)cap;  // a small batch spreads over the SMs
    for (int K = 1; K <= cmax; K++) {
        const int tpg = ((K * h.Z + 31) / 32) * 32;
        int G = 1024 / tpg;
        if (tpg > 32 && G > 15) G = 15;
        int C = G * K;
        if (C > cmax) C = cmax;
        if (C > best.C) best = {C, K, tpg};
    }
    return best;
}

int layered_slots_per_cta(const CodeDev &h) { return lslots_shape(h).C; }

template <int DMAX>
static cudaError_t launch_lslots(const CodeDev &h, const CodeDev *d, const LayeredSlotArgs &a, cudaStream_t s)
{
    const size_t sm = lslots_smem(h, a.C);
    cudaError_t e = ensure_smem<k_layered_slots<DMAX>>(sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t ctas = nsm;
    const int64_t need = (a.n_items + a.C - 1) / a.C;
    if (need < ctas) ctas = need;
    LaunchScope ls(F_LAYERED, s);
    const int groups = (a.C + a.K - 1) / a.K;
    k_layered_slots<DMAX><<<(unsigned)ctas, groups * a.TPG, sm, s>>>(d, a);
    return cudaGetLastError();
}

// Decode the codewords of n requests of one code (reqs[i].code all the same) in one launch.
cudaError_t layered_slots_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const HostReq *reqs,
                                 int n, int llr_type, void *counter, cudaStream_t s)
{
    if (n < 1 || n > MULTI_MAX_REQS) return cudaErrorInvalidValue;
    LayeredSlotArgs a;
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
    a.llr_type = llr_type;
    a.scale = p.llr_scale;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const LslotShape sh = lslots_shape(h, (items + nsm - 1) / nsm);
    a.C = sh.C;
    if (a.C < 1) return cudaErrorInvalidValue;
    a.K = sh.K;
    a.TPG = sh.TPG;
    a.strideA = (h.N + 15) & ~15;
    a.strideR = (h.E + 15) & ~15;
    a.max_iter = p.max_iter;
    a.early_exit = p.early_exit;
    a.alpha_num = p.nms_alpha_num;
    a.alpha_shift = p.nms_alpha_shift;
    a.msg_sat = p.msg_sat;
    a.app_sat = p.app_sat;
    a.next = static_cast<unsigned long long *>(counter);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (h.dc_max <= 8) return launch_lslots<8>(h, d, a, s);
    if (h.dc_max <= 16) return launch_lslots<16>(h, d, a, s);
    if (h.dc_max <= 24) return launch_lslots<24>(h, d, a, s);
    return launch_lslots<32>(h, d, a, s);
}

cudaError_t layered_decode(const CodeDev &h, const CodeDev *d, const ldpc_decode_params &p, const void *llr,
                           int llr_type, int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, cudaStream_t s)
{
    LayeredArgs a;
    a.llr = llr;
    a.llr_type = llr_type;
    a.scale = p.llr_scale;
    a.n_cw = n_cw;
    a.C = pick_C(h);
    while (a.C > 1 && layered_smem(h, a.C) > 100 * 1024) a.C--;
    a.max_iter = p.max_iter;
    a.early_exit = p.early_exit;
    a.alpha_num = p.nms_alpha_num;
    a.alpha_shift = p.nms_alpha_shift;
    a.msg_sat = p.msg_sat;
    a.app_sat = p.app_sat;
    a.bits = bits;
    a.iters = iters;
    a.app_out = app_out;
    if (h.dc_max <= 8) return launch_layered<8>(h, d, a, s);
    if (h.dc_max <= 16) return launch_layered<16>(h, d, a, s);
    if (h.dc_max <= 24) return launch_layered<24>(h, d, a, s);
    return launch_layered<32>(h, d, a, s);
}

}  // namespace ldpc
