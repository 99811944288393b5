// BF16 tensor-core edge kernels (placeholder until the tcgen05 path lands).
#include "kernels.h"

namespace mp {

int launch_edge_fwd_bf16(const Model&, const EdgeArgs&, cudaStream_t, int) { return MP_ERR_UNSUPPORTED; }
int launch_edge_bwd_bf16(const Model&, const EdgeArgs&, cudaStream_t, int) { return MP_ERR_UNSUPPORTED; }

}  // namespace mp
