// mdl_ctx.h -- abstract context behind the C ABI; one implementation per (precision, dim, order).
#pragma once

#include <string>

#include "../../include/mdl.h"

namespace mdl {

class CtxBase {
public:
    virtual ~CtxBase() {}
    virtual int create(const mdl_problem& pb) = 0;
    virtual int upload_mesh(int64_t n, const int32_t* root, const int8_t* level, const int32_t* coords) = 0;
    virtual int set_initial(const double* V, const double* s, int64_t n_dof) = 0;
    virtual int set_levels(const int8_t* b, int64_t n) = 0;
    virtual int set_indicators(const double* eta_s, const double* eta_t, int64_t n) = 0;
    virtual int step_barriers(int64_t n) = 0;
    virtual int step_to(double t_end) = 0;
    virtual int get_time(double* t, int64_t* tick, double* dt) const = 0;
    virtual int get_sizes(int64_t* ne, int64_t* ndof, int64_t* nprobe) const = 0;
    virtual int read_field(int which, double* out, int64_t cap, int64_t* n) = 0;
    virtual int set_initial_f32(const float* V, const float* s, int64_t n_dof) = 0;
    virtual int read_fields_f32(float* V, float* s, int64_t cap, int64_t* n) = 0;
    virtual int read_activation(double* out, int64_t cap, int64_t* n) = 0;
    virtual int read_mesh(int32_t* root, int8_t* level, int32_t* coords, int8_t* b, int64_t cap, int64_t* n) = 0;
    virtual int read_faces(int8_t* kind, int32_t* nbr, int8_t* pos, int64_t cap, int64_t* n) = 0;
    virtual int read_indicators(double* eta_s, double* eta_t, int64_t cap, int64_t* n) = 0;
    virtual int get_stats(mdl_stats* s) const = 0;
    virtual int reset_stats() = 0;
    virtual int set_timing(int on) = 0;
    virtual int device_view(int which, void** p, int64_t* n, void** stream) = 0;
    // Asynchronous stepping for batches: launch up to n barriers (no host wait), then
    // wait, handle capacity growth and errors, and report how many completed.
    virtual int begin_barriers(int64_t n) = 0;
    virtual int end_barriers(int64_t* completed) = 0;
    // Launch shape of the sweep kernel (threads per block, resident blocks per SM); results
    // do not depend on it.  Returns MDL_E_ARG for unsupported shapes.
    virtual int set_tick_shape(int threads, int blocks_per_sm) = 0;
    virtual int set_sweep_variant(int variant) = 0;
    // Upper bound on the blocks of the persistent tensor-core sweep (0: the default).
    virtual int set_sweep_blocks(int max_blocks) = 0;
    // Fused batch rounds (mdl_fused.h): launch the phases before the sweep (indicator,
    // adaptation, levels, ordering) of one barrier on the context's stream and write the
    // slot's sweep record (a FusedSlot of the context's precision, shift left 0) and its LTS
    // level count B; after the batch's fused sweep (or after fused_own_sweep(), the
    // context's own sweep variant on its own stream), launch the epilogue.  Several rounds
    // may be issued before end_barriers(), which then completes them as after
    // begin_barriers(rounds).  A context with replayed inputs (set_levels, set_indicators)
    // takes one round per end_barriers(); replaying() says so.
    virtual int fused_begin(void* slot_record, int* B) = 0;
    virtual int fused_own_sweep() = 0;
    virtual int fused_finish() = 0;
    virtual bool replaying() const = 0;
    // A mapped (curved) geometry: its sweep is always its own (the fused kernel has box
    // elements only).
    virtual bool is_mapped() const = 0;
    virtual void* stream_handle() const = 0;
    virtual int precision() const = 0;
    virtual int64_t device_bytes() const = 0;     // device memory held by the context
    virtual double dt_barrier() const = 0;
    std::string err;
};

CtxBase* make_ctx(const mdl_problem& p);
CtxBase* make_ctx_f32_2_1();
CtxBase* make_ctx_f64_2_1();
CtxBase* make_ctx_f32_2_2();
CtxBase* make_ctx_f64_2_2();
CtxBase* make_ctx_f32_3_1();
CtxBase* make_ctx_f64_3_1();
CtxBase* make_ctx_f32_3_2();
CtxBase* make_ctx_f64_3_2();

// Footprint estimate (device bytes) of a problem before it is created.
int64_t estimate_footprint(const mdl_problem& p);
int check_problem(const mdl_problem* p, std::string* why);

}  // namespace mdl

// The opaque handle behind the C ABI.
struct mdl_ctx {
    mdl::CtxBase* impl = nullptr;
    std::string err;
};
