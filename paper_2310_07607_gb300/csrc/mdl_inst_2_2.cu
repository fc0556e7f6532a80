// Instantiation of the context for dim 2, order 2 (FP32 and FP64).
#include "mdl_ctx_impl.cuh"

namespace mdl {
CtxBase* make_ctx_f32_2_2() { return new Ctx<float, 2, 2>(); }
CtxBase* make_ctx_f64_2_2() { return new Ctx<double, 2, 2>(); }
}  // namespace mdl
