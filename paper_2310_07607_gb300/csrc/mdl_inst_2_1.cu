// Instantiation of the context for dim 2, order 1 (FP32 and FP64).
#include "mdl_ctx_impl.cuh"

namespace mdl {
CtxBase* make_ctx_f32_2_1() { return new Ctx<float, 2, 1>(); }
CtxBase* make_ctx_f64_2_1() { return new Ctx<double, 2, 1>(); }
}  // namespace mdl
