// mdl_capi.cu -- the C ABI: argument checks, dispatch to the (precision, dim, order) context.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <string>

#include "../../include/mdl.h"
#include "mdl_ctx.h"
#include "mdl_geometry.h"
#include "mdl_kernels.cuh"

namespace mdl {

__global__ void k_fill_inf(double* p, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = INFINITY;
}

}  // namespace mdl

namespace mdl {

int check_problem(const mdl_problem* p, std::string* why) {
    if (!p) { *why = "problem is NULL"; return MDL_E_ARG; }
    if (p->dim != 2 && p->dim != 3) { *why = "dim must be 2 or 3"; return MDL_E_ARG; }
    if (p->order != 1 && p->order != 2) { *why = "order must be 1 or 2"; return MDL_E_ARG; }
    for (int k = 0; k < p->dim; ++k) {
        if (!(p->extent[k] > 0)) { *why = "extent must be positive"; return MDL_E_ARG; }
        if (p->base[k] < 1 || p->base[k] > 65535) { *why = "base must be in [1, 65535]"; return MDL_E_ARG; }
    }
    if (!(p->chi > 0) || !(p->cm > 0)) { *why = "chi and cm must be positive"; return MDL_E_ARG; }
    if (!(p->sigma_l >= 0) || !(p->sigma_t >= 0)) { *why = "conductivities must be >= 0"; return MDL_E_ARG; }
    if (!(p->gamma >= 0)) { *why = "gamma must be >= 0"; return MDL_E_ARG; }
    if (p->ionic_model != 0 && p->ionic_model != -1) { *why = "ionic_model must be 0 or -1"; return MDL_E_ARG; }
    if (p->n_stim < 0 || p->n_stim > MDL_MAX_STIM) { *why = "n_stim out of range"; return MDL_E_ARG; }
    if (p->max_refine < 0 || p->max_refine > MDL_MAX_REFINE) { *why = "max_refine out of range"; return MDL_E_ARG; }
    if (p->n_lts_levels < 1 || p->n_lts_levels > 8) { *why = "n_lts_levels must be in [1, 8]"; return MDL_E_ARG; }
    if (!(p->dt_barrier >= 0)) { *why = "dt_barrier must be >= 0"; return MDL_E_ARG; }
    if (p->precision != 32 && p->precision != 64) { *why = "precision must be 32 or 64"; return MDL_E_ARG; }
    if (p->state_integrator != 0 && p->state_integrator != 1) { *why = "state_integrator must be 0 or 1"; return MDL_E_ARG; }
    double roots = 1.0;
    for (int k = 0; k < p->dim; ++k) roots *= p->base[k];
    if (roots * 27.0 > 2.0e9) { *why = "too many roots"; return MDL_E_ARG; }
    if (p->fibre_ref != 0 && p->fibre_ref != 1) { *why = "fibre_ref must be 0 or 1"; return MDL_E_ARG; }
    const char* gw = nullptr;
    if (geo_check(*p, &gw) != MDL_OK) { *why = gw; return MDL_E_ARG; }
    return MDL_OK;
}

}  // namespace mdl

namespace {

mdl::CtxBase* make(const mdl_problem* p) { return mdl::make_ctx(*p); }

}  // namespace

namespace mdl {

CtxBase* make_ctx(const mdl_problem& pr) {
    const mdl_problem* p = &pr;
    const bool f64 = p->precision == 64;
    if (p->dim == 2 && p->order == 1) return f64 ? mdl::make_ctx_f64_2_1() : mdl::make_ctx_f32_2_1();
    if (p->dim == 2 && p->order == 2) return f64 ? mdl::make_ctx_f64_2_2() : mdl::make_ctx_f32_2_2();
    if (p->dim == 3 && p->order == 1) return f64 ? mdl::make_ctx_f64_3_1() : mdl::make_ctx_f32_3_1();
    return f64 ? mdl::make_ctx_f64_3_2() : mdl::make_ctx_f32_3_2();
}

// Device bytes of a freshly created context: per-element arrays at the initial capacity
// (twice the roots, or four times with adaptation, each with its 8-byte leaf key) and the
// probes.
int64_t estimate_footprint(const mdl_problem& p) {
    const int d = p.dim, n1 = p.order + 1;
    const int64_t np0 = d == 2 ? n1 * n1 : n1 * n1 * n1;
    const int64_t np = np0 == 27 ? 28 : np0;   // row stride of the per-DOF arrays (Q2 3D padded)
    const int64_t nf = 2 * d, nsub = 1 << (d - 1);
    int64_t roots = 1;
    for (int k = 0; k < d; ++k) roots *= p.base[k];
    const int64_t cap = std::max<int64_t>(roots * (p.amr_enabled ? 4 : 2), 4096);
    const int64_t r = p.precision == 64 ? 8 : 4;
    const int64_t per_set = 3 * np * r + 8 + 1 + 16;
    const int64_t shared = 2 * np * r + 8 + 8 + 1 + 1 + 8 + 1 + 1 + 4 + 4;
    int64_t tables = 1 + 4 + 4 + 4 * nf + 4 * nf * nsub + 4 + 4 + 4 * p.n_stim + 8;
    if (p.geometry != MDL_GEOMETRY_BOX) {
        // per set: geometric factors, GL masses, signature and stimulus masks of every element;
        // the list of elements whose factors an adaptation recomputes
        const int64_t npf = d == 2 ? n1 : n1 * n1;
        tables += 2 * ((np0 * (d * (d + 1) / 2 + 1) + nf * npf * (d + 2)) * r + np0 * 8 + 4 + 4 * p.n_stim) + 4;
    }
    return cap * (2 * per_set + shared + tables) + roots * np0 * 8 + (1 << 20);
}

}  // namespace mdl

namespace {

thread_local std::string g_create_err;

}  // namespace

#define MDL_GUARD(ctx)                          \
    if (!(ctx) || !(ctx)->impl) return MDL_E_ARG;

#define MDL_CALL(ctx, expr)                     \
    do {                                        \
        MDL_GUARD(ctx);                         \
        try {                                   \
            int rc_ = (ctx)->impl->expr;        \
            if (rc_) (ctx)->err = (ctx)->impl->err; \
            return rc_;                         \
        } catch (const std::bad_alloc&) {       \
            (ctx)->err = "host allocation failed"; \
            return MDL_E_NOMEM;                 \
        } catch (...) {                         \
            (ctx)->err = "internal error";      \
            return MDL_E_STATE;                 \
        }                                       \
    } while (0)

extern "C" {

int mdl_create(const mdl_problem* prob, mdl_ctx** out) {
    if (!out) return MDL_E_ARG;
    *out = nullptr;
    std::string why;
    int rc = mdl::check_problem(prob, &why);
    if (rc) {
        g_create_err = why;
        return rc;
    }
    mdl_ctx* c = nullptr;
    try {
        c = new mdl_ctx();
        c->impl = make(prob);
        rc = c->impl->create(*prob);
    } catch (const std::bad_alloc&) {
        g_create_err = "host allocation failed";
        if (c) { delete c->impl; delete c; }
        return MDL_E_NOMEM;
    }
    if (rc) {
        g_create_err = c->impl->err;
        delete c->impl;
        delete c;
        return rc;
    }
    *out = c;
    return MDL_OK;
}

int mdl_upload_mesh(mdl_ctx* ctx, int64_t n_leaves, const int32_t* root, const int8_t* level,
                    const int32_t* coords) {
    if (n_leaves <= 0 || !level || !coords) return MDL_E_ARG;
    MDL_CALL(ctx, upload_mesh(n_leaves, root, level, coords));
}

int mdl_set_initial(mdl_ctx* ctx, const double* V, const double* s, int64_t n_dof) {
    MDL_CALL(ctx, set_initial(V, s, n_dof));
}

int mdl_set_levels(mdl_ctx* ctx, const int8_t* b_e, int64_t n_e) { MDL_CALL(ctx, set_levels(b_e, n_e)); }

int mdl_set_indicators(mdl_ctx* ctx, const double* eta_s, const double* eta_t, int64_t n_e) {
    MDL_CALL(ctx, set_indicators(eta_s, eta_t, n_e));
}

int mdl_step_to(mdl_ctx* ctx, double t_end) { MDL_CALL(ctx, step_to(t_end)); }

int mdl_step_barriers(mdl_ctx* ctx, int64_t n) {
    if (n < 0) return MDL_E_ARG;
    MDL_CALL(ctx, step_barriers(n));
}

int mdl_get_time(const mdl_ctx* ctx, double* t, int64_t* barrier_tick, double* dt) {
    MDL_GUARD(ctx);
    return ctx->impl->get_time(t, barrier_tick, dt);
}

int mdl_get_sizes(const mdl_ctx* ctx, int64_t* n_e, int64_t* n_dof, int64_t* n_probe) {
    MDL_GUARD(ctx);
    return ctx->impl->get_sizes(n_e, n_dof, n_probe);
}

int mdl_set_initial_f32(mdl_ctx* ctx, const float* V, const float* s, int64_t n_dof) {
    MDL_CALL(ctx, set_initial_f32(V, s, n_dof));
}
int mdl_read_fields_f32(mdl_ctx* ctx, float* V, float* s, int64_t cap, int64_t* n) {
    MDL_CALL(ctx, read_fields_f32(V, s, cap, n));
}
int mdl_read_V(mdl_ctx* ctx, double* out, int64_t cap, int64_t* n) { MDL_CALL(ctx, read_field(0, out, cap, n)); }
int mdl_read_state(mdl_ctx* ctx, double* out, int64_t cap, int64_t* n) { MDL_CALL(ctx, read_field(1, out, cap, n)); }
int mdl_read_activation(mdl_ctx* ctx, double* out, int64_t cap, int64_t* n) {
    MDL_CALL(ctx, read_activation(out, cap, n));
}
int mdl_read_mesh(mdl_ctx* ctx, int32_t* root, int8_t* level, int32_t* coords, int8_t* b_e, int64_t cap,
                  int64_t* n) {
    MDL_CALL(ctx, read_mesh(root, level, coords, b_e, cap, n));
}
int mdl_read_faces(mdl_ctx* ctx, int8_t* kind, int32_t* nbr, int8_t* pos, int64_t cap, int64_t* n) {
    MDL_CALL(ctx, read_faces(kind, nbr, pos, cap, n));
}
int mdl_read_indicators(mdl_ctx* ctx, double* eta_s, double* eta_t, int64_t cap, int64_t* n) {
    MDL_CALL(ctx, read_indicators(eta_s, eta_t, cap, n));
}
int mdl_get_stats(const mdl_ctx* ctx, mdl_stats* out) {
    MDL_GUARD(ctx);
    if (!out) return MDL_E_ARG;
    return ctx->impl->get_stats(out);
}
int mdl_reset_stats(mdl_ctx* ctx) { MDL_CALL(ctx, reset_stats()); }
int mdl_set_timing(mdl_ctx* ctx, int on) { MDL_CALL(ctx, set_timing(on)); }
int mdl_device_view(mdl_ctx* ctx, int which, void** dptr, int64_t* n, void** stream) {
    MDL_CALL(ctx, device_view(which, dptr, n, stream));
}

const char* mdl_last_error(const mdl_ctx* ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

void mdl_destroy(mdl_ctx* ctx) {
    if (!ctx) return;
    delete ctx->impl;
    delete ctx;
}

const char* mdl_version(void) { return "mdl 0.1 sm_103a"; }

}  // extern "C"
