// P_tilde with FP64 storage and arithmetic (approach A1 of Sec. 5).
#include "precond.cuh"

namespace aao {
PrecondBase* make_precond_f64(Handle* h) { return new Precond<double, double>(h); }
}  // namespace aao
