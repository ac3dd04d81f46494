// P_tilde with FP32 storage and arithmetic (approach A2 of Sec. 5).
#include "precond.cuh"

namespace aao {
PrecondBase* make_precond_f32_bf16(Handle* h);
PrecondBase* make_precond_f32_f16(Handle* h);
PrecondBase* make_precond_f32(Handle* h, int prec_Pint) {
    if (prec_Pint == AAO_FP32) return new Precond<float, float>(h);
    if (prec_Pint == AAO_BF16) return make_precond_f32_bf16(h);
    if (prec_Pint == AAO_FP16) return make_precond_f32_f16(h);
    return nullptr;
}
}  // namespace aao
