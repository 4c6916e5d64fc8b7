// ms_kind_radix.cu -- multisplit launchers for the "radix" bucket identifier.
#include "ms_run.cuh"

namespace ms {

cudaError_t run_multisplit_radix(const Call& c, DeviceCtx& ctx) { return run_ms_kind<kRadix>(c, ctx); }

}  // namespace ms
