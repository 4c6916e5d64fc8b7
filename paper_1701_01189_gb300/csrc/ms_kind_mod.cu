// ms_kind_mod.cu -- multisplit launchers for the "mod" bucket identifier.
#include "ms_run.cuh"

namespace ms {

cudaError_t run_multisplit_mod(const Call& c, DeviceCtx& ctx) { return run_ms_kind<kMod>(c, ctx); }

}  // namespace ms
