// Stage 2 on tensor cores: placeholder until the split-BF16 tcgen05 kernel lands.
#include "su2_internal.h"

namespace su2 {

bool tc_supported(int) { return false; }

cudaError_t launch_contract_forward_tc(const BandArgs&, const void*, void*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace su2
