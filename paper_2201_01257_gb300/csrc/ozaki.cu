// Split-precision (Ozaki-style) block-sparse contraction: placeholder until the
// tcgen05 kernels land.
#include "tamm_contract.h"

namespace tamm {
void run_contract_ozaki(tamm_ctx*, double, tamm_tensor*, const char*, double, const tamm_tensor*, const char*,
                        const tamm_tensor*, const char*, int) {
  throw Error(TAMM_EUNSUPPORTED, "split-precision path not built");
}
}  // namespace tamm
