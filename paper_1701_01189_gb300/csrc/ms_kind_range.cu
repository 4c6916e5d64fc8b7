// ms_kind_range.cu -- multisplit launchers for the "range" bucket identifier.
#include "ms_run.cuh"

namespace ms {

cudaError_t run_multisplit_range(const Call& c, DeviceCtx& ctx) { return run_ms_kind<kRange>(c, ctx); }

}  // namespace ms
