// Internal declarations shared by the library's translation units (CUDA path only).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ldpc.h"

namespace ldpc {

constexpr int MB_MAX = 64;
constexpr int NB_MAX = 128;
constexpr int NNZ_MAX = 1024;
constexpr int Z_MAX = 1024;
// Codewords per interleaved tile.  Flooding state lives in HBM as [tile][node][TILE]:
// the TILE codewords of one node are contiguous, so a warp reading one node for its
// lanes' codewords issues one coalesced 128-bit access per lane (Sec. III-B interleaving).
constexpr int TILE = 128;

// Device-side description of a QC code.  Nonzero blocks are numbered b = 0..nnz-1 in
// row-major order; edge (b, r) joins check l*Z + r to variable j*Z + (r + s) mod Z, and
// its message lives at edge index b*Z + r.
struct CodeDev {
    int32_t mb, nb, Z, nnz;
    int32_t N, M, K, E;
    int32_t dc_max, dv_max, pad0, pad1;
    int32_t rowptr[MB_MAX + 1];  // blocks of block row l: [rowptr[l], rowptr[l+1])
    int32_t ent[NNZ_MAX];        // (j << 16) | s for block b
    int32_t colptr[NB_MAX + 1];  // entries of block column j: [colptr[j], colptr[j+1])
    int32_t colent[NNZ_MAX];     // (b << 16) | s for those blocks
    unsigned int *status;        // the device's input status word (library-owned, one per device)
    // block rows by degree: rord[dbeg[d - 2] .. dbeg[d - 1]) are the rows of degree d (2..8),
    // rord[dbeg[7] .. dbeg[8]) those above degree 8 (for the flooding slot decoder)
    int32_t rord[MB_MAX];
    int32_t dbeg[12];
};

// Bits of the input status word: kernels that load channel LLRs set them (atomicOr, only
// when an offending value is seen); ldpc_stream_check reads and clears the word.
enum InputFlag : unsigned int { IN_NONFINITE = 1u, IN_I8_RANGE = 2u };

// Per-kernel-family timing and launch accounting (see ldpc_profile_* in ldpc.h).
enum Family { F_INTERLEAVE = 0, F_CN = 1, F_VN = 2, F_DEINTERLEAVE = 3, F_LAYERED = 4, F_PLAIN_CN = 5,
              F_PLAIN_VN = 6, F_SLOTS = 7, F_LAYERED_SPA = 8, F_COUNT = 9 };
struct LaunchScope {
    LaunchScope(int family, cudaStream_t s);
    ~LaunchScope();
    int family;
    cudaStream_t stream;
    cudaEvent_t ev[2];
    bool on;
};

// Flooding workspace carve-up (all regions 256-byte aligned).
struct FloodWs {
    float *L;          // [ntiles][N][TILE] channel LLRs, interleaved
    float *app;        // [ntiles][N][TILE] posterior LLRs
    void *R;           // [ntiles][E][TILE] check-to-variable messages (fp32 or fp16)
    int32_t *done_at;  // [ntiles*TILE] 0 = decoding, t = converged after iteration t, -1 = padding
    int32_t *unsat;    // [ntiles*TILE] last iteration at which a check was found unsatisfied
};
size_t flood_ws_layout(const CodeDev &c, int64_t n_cw, int msg, FloodWs *ws, char *base);

cudaError_t flood_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p, const float *llr,
                         int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, const FloodWs &ws,
                         cudaStream_t s);
cudaError_t layered_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p, const void *llr,
                           int llr_type, int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out,
                           cudaStream_t s);
int layered_supported(const CodeDev &host);
// Persistent slot form of the layered min-sum (0 slots: code too large for it); every codeword
// of n requests of one code in one launch.
int layered_slots_per_cta(const CodeDev &host);
cudaError_t layered_slots_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p,
                                 const struct HostReq *reqs, int n, int llr_type, void *counter, cudaStream_t s);

// ---------------------------------------------------------------- slot decoders
// Persistent decoders with per-codeword work queues (flood_slots.cu, layered_kernels.cu).
// One launch serves up to MULTI_MAX_REQS requests over up to MULTI_MAX_GROUPS distinct
// codes; the descriptors travel as a kernel parameter.  The work counters (8 bytes per
// group) live in the caller's workspace and are zeroed on the stream before the launch.
constexpr int SLOTS_MAX = 64;  // codeword slots per CTA
constexpr int MULTI_MAX_GROUPS = 16;
constexpr int MULTI_MAX_REQS = 128;
constexpr size_t SLOTS_WS_BYTES = 256;  // >= 8 * MULTI_MAX_GROUPS

struct ReqDev {
    const void *llr;
    uint8_t *bits;
    int32_t *iters;
    float *app;
    int64_t n_cw;
    int64_t item0;  // index of its first codeword in its group's work sequence
};
struct GroupDev {
    const CodeDev *code;
    int C;       // slots per CTA for this code
    int K, TPG;  // thread slots per barrier group; threads per group (whole warps)
    int req_begin, req_end;
    int N, E, Z, mb, nb, nnz, dc_max;
    int64_t n_items;
    float cumw;  // cumulative share of the launch's work (initial CTA placement)
    // single slots: thread groups of Z threads a slot's block rows and columns are spread over
    // (1 unless a small batch leaves threads to spare).  Kept last: the field ahead of the
    // others changed the slot decoder's parameter loads and cost it 2-3 % (measured).
    int W;
};
struct MultiDesc {
    int n_groups;
    GroupDev groups[MULTI_MAX_GROUPS];
    ReqDev reqs[MULTI_MAX_REQS];
};
struct HostReq {
    const ldpc_code *code;
    const void *llr;
    int64_t n_cw;
    uint8_t *bits;
    int32_t *iters;
    float *app;
};

// Shared memory ahead of the slot arrays: per-slot bookkeeping and the code tables.
__host__ __device__ inline size_t slots_smem_head(int tbl_ints)
{
    return ((size_t)SLOTS_MAX * 16 + 16 + (size_t)tbl_ints * 4 + 15) & ~(size_t)15;
}

// Layered sum-product slot decoder (layered_spa.cu): slots per CTA (0: code too large).
int layered_spa_slots_per_cta(const CodeDev &host, int msg);
cudaError_t layered_spa_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p, const float *llr,
                               int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, void *counter,
                               cudaStream_t s);

// Flooding SPA cluster decoder (flood_cluster.cu): one codeword per two-SM cluster, for codes
// whose codeword does not fit one CTA; every codeword of n requests of one code in one launch.
int cluster_supported(const CodeDev &host, int msg);
cudaError_t flood_cluster_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p,
                                 const HostReq *reqs, int n, void *counter, cudaStream_t s);

// Flooding SPA slot decoder: supported when one codeword of the code fits a CTA.
int slots_supported(const CodeDev &host, int msg);
int slots_pairable(const CodeDev &host, int msg);
cudaError_t flood_multi_decode(const HostReq *reqs, int n, const ldpc_decode_params &p, void *counters,
                               cudaStream_t s);

// Record a message for ldpc_last_error() on the calling thread.
void set_error(const char *msg);

// The device's input status word (allocated on first use; see InputFlag).
cudaError_t device_status_word(int dev, unsigned int **out);

}  // namespace ldpc

// Schedule choices stored by ldpc_autotune (0: not tuned, the built-in heuristic decides).
enum Schedule { SCHED_UNTUNED = 0, SCHED_SLOTS_V1 = 1, SCHED_SLOTS_V2 = 2, SCHED_STREAMING = 3 };

struct ldpc_code {
    ldpc::CodeDev host;
    ldpc::CodeDev *dev;
    int device;
    int tuned_flood[2];  // per message type (F32, F16)
    int tuned_layered;
};

namespace ldpc {
// Raise a kernel's dynamic shared-memory limit once per device and size.  The attribute is
// host-side state; setting it only when it grows keeps repeated launches (and launches
// inside a stream capture, after the first eager one) free of the call.
template <auto Kernel>
inline cudaError_t ensure_smem(size_t bytes)
{
    static int set_bytes[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if ((size_t)__atomic_load_n(&set_bytes[dev], __ATOMIC_RELAXED) >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) __atomic_store_n(&set_bytes[dev], (int)bytes, __ATOMIC_RELAXED);
    return e;
}
}  // namespace ldpc
