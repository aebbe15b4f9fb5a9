// Tensor-core (tcgen05) implicit-GEMM conv path -- placeholder until built.
#include "gw_internal.h"

namespace gw {

int tc_supported() { return 0; }

void tc_pack_layer(LayerDev&, const std::vector<double>&, int, gw_ctx*, size_t*, std::vector<void*>&) {
  throw Error(GW_ENOTIMPL, "tensor-core path not built");
}

void launch_conv_tc(const LayerDev&, const TcAct&, int, const TcOut&, int, int*, cudaStream_t) {
  throw Error(GW_ENOTIMPL, "tensor-core path not built");
}

}  // namespace gw
