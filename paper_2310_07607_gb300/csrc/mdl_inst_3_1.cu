// Instantiation of the context for dim 3, order 1 (FP32 and FP64).
#include "mdl_ctx_impl.cuh"

namespace mdl {
CtxBase* make_ctx_f32_3_1() { return new Ctx<float, 3, 1>(); }
CtxBase* make_ctx_f64_3_1() { return new Ctx<double, 3, 1>(); }
}  // namespace mdl
