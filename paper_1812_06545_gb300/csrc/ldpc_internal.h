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
};

// Per-kernel-family timing and launch accounting (see ldpc_profile_* in ldpc.h).
enum Family { F_INTERLEAVE = 0, F_CN = 1, F_VN = 2, F_DEINTERLEAVE = 3, F_LAYERED = 4, F_PLAIN_CN = 5,
              F_PLAIN_VN = 6, F_SLOTS = 7, F_COUNT = 8 };
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
// Persistent slot form of the layered min-sum (0 slots: code too large for it).
int layered_slots_per_cta(const CodeDev &host);
cudaError_t layered_slots_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p, const void *llr,
                                 int llr_type, int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out,
                                 void *counter, cudaStream_t s);

// On-chip slot decoder for the flooding forms (flood_slots.cu).  counter: 8 bytes of
// device memory, zeroed on the stream before the launch.
constexpr size_t SLOTS_WS_BYTES = 256;
int slots_supported(const CodeDev &host, int msg);
cudaError_t slots_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p, const float *llr,
                         int64_t n_cw, uint8_t *bits, int32_t *iters, float *app_out, void *counter, cudaStream_t s);

// Record a message for ldpc_last_error() on the calling thread.
void set_error(const char *msg);

}  // namespace ldpc

struct ldpc_code {
    ldpc::CodeDev host;
    ldpc::CodeDev *dev;
    int device;
};
