// Declarations of the layered min-sum with two codewords per thread in packed half precision
// (layered_pairs.cu), kept apart from ldpc_internal.h so that the other kernels' sources do not
// change with it.
#pragma once

#include "ldpc_internal.h"

namespace ldpc {

// Layered min-sum with two codewords per thread in packed half precision (layered_pairs.cu):
// exact for the parameters layered_pairs_exact admits; codewords per CTA (0: code too large).
bool layered_pairs_exact(const ldpc_decode_params &p);
int layered_pairs_per_cta(const CodeDev &host);
// Every codeword of n requests of one code in one launch (one work sequence).
cudaError_t layered_pairs_decode(const CodeDev &host, const CodeDev *dev, const ldpc_decode_params &p,
                                 const HostReq *reqs, int n, int llr_type, void *counter, cudaStream_t s);

}  // namespace ldpc
