// P_tilde in FP32 with Rana's sweep and the V-cycles in BF16 storage
// (per-row scaling, FP32 arithmetic): the A5-like split of Sec. 5.
#include "precond.cuh"

namespace aao {
PrecondBase* make_precond_f32_bf16(Handle* h) { return new Precond<float, __nv_bfloat16>(h); }
}  // namespace aao
