// P_tilde entirely in 16-bit storage (BF16 or FP16, per-row scaling, FP32
// arithmetic): the A4-like variant of Sec. 5.
#include "precond.cuh"

namespace aao {
PrecondBase* make_precond_lowP(Handle* h, int prec_P) {
    if (prec_P == AAO_BF16) return new Precond<__nv_bfloat16, __nv_bfloat16>(h);
    if (prec_P == AAO_FP16) return new Precond<__half, __half>(h);
    return nullptr;
}
}  // namespace aao
