// ms_kind_delta.cu -- multisplit launchers for the "delta" bucket identifier.
#include "ms_run.cuh"

namespace ms {

cudaError_t run_multisplit_delta(const Call& c, DeviceCtx& ctx) { return run_ms_kind<kDelta>(c, ctx); }

}  // namespace ms
