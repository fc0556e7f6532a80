// Instantiation of the context for dim 3, order 2 (FP32 and FP64).
#include "mdl_ctx_impl.cuh"

namespace mdl {
CtxBase* make_ctx_f32_3_2() { return new Ctx<float, 3, 2>(); }
CtxBase* make_ctx_f64_3_2() { return new Ctx<double, 3, 2>(); }
}  // namespace mdl
