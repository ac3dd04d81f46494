// P_tilde in FP32 with Rana's sweep and the V-cycles in FP16 storage
// (per-row scaling, FP32 arithmetic): approach A5 of Sec. 5.
#include "precond.cuh"

namespace aao {
PrecondBase* make_precond_f32_f16(Handle* h) { return new Precond<float, __half>(h); }
}  // namespace aao
