// Tensor-core (tcgen05) contraction of a wave: not available in this build yet.
#include "common.cuh"

namespace ext4pcf {

bool tc_supported(const Layout&, int) { return false; }

size_t contract_tc_scratch(const Layout&, int) { return 0; }

cudaError_t contract_wave_tc(const Layout&, const float2*, const float2*, int, double*, int, void*, size_t,
                             int*, long long, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace ext4pcf
