// mdl_batch.cpp -- many resident simulations stepped together on one GPU.
//
// Each slot is an ordinary context with its own stream and captured phase graphs; a
// batch step first launches every unfinished slot's barriers (no host wait), then
// waits for all of them, so their kernels overlap on the device.  Admission is by
// device-memory footprint against the batch's budget.  The sweep kernel's launch shape
// (threads per block, resident blocks per SM) is tuned once per (precision, dim, order)
// class on a temporary copy of the first admitted instance; the shape does not
// change any result, so an instance gives the same values alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <map>
#include <string>
#include <vector>

#include "../../include/mdl.h"
#include "mdl_ctx.h"

struct mdl_batch {
    struct Slot {
        mdl_ctx* ctx = nullptr;
        double t_end = 0;
        int64_t bytes = 0;
        int state = MDL_SLOT_FREE;
        int rc = MDL_OK;
        int64_t barriers_total = 0;
        int64_t barriers_done = 0;
        bool polled = false;
    };
    int64_t budget = 0;
    int64_t used = 0;
    int autotune = 1;
    std::vector<Slot> slots;
    std::map<int, std::pair<int, int>> shapes;   // class -> (threads, blocks per SM)
    std::string err;
    int64_t steps = 0;
};

namespace {

thread_local std::string g_batch_err;

int class_key(const mdl_problem& p) { return p.precision * 100 + p.dim * 10 + p.order; }

int64_t barriers_to(double dt, double t0, double t_end) {
    const double n = std::floor((t_end - t0) / dt + 1e-9);
    return n > 0 ? (int64_t)n : 0;
}

// Time `n` barriers of the context for each candidate sweep launch shape (threads, blocks
// per SM) of its sweep variant and keep the fastest.  The variant itself is not tuned:
// variants round differently, and a slot must give the values it gives alone.
int tune(mdl_ctx* c, int n, std::pair<int, int>* best) {
    static const int cand[][2] = {{128, 16}, {64, 32}, {256, 8}, {128, 8}, {64, 16}};
    double best_ms = 1e300;
    *best = {128, 16};
    mdl::CtxBase* x = c->impl;
    x->set_timing(1);
    for (const auto& s : cand) {
        int rc = x->set_tick_shape(s[0], s[1]);
        if (rc) continue;
        // one untimed barrier captures the graphs
        int64_t done = 0;
        if ((rc = x->begin_barriers(1)) || (rc = x->end_barriers(&done))) return rc;
        mdl_stats s0{}, s1{};
        x->get_stats(&s0);
        for (int i = 0; i < n; ++i)
            if ((rc = x->begin_barriers(1)) || (rc = x->end_barriers(&done))) return rc;
        x->get_stats(&s1);
        const double ms = (s1.sweep_ms - s0.sweep_ms) / std::max<int64_t>(1, s1.timed_barriers - s0.timed_barriers);
        if (ms < best_ms) {
            best_ms = ms;
            *best = {s[0], s[1]};
        }
    }
    x->set_timing(0);
    return x->set_tick_shape(best->first, best->second);
}

}  // namespace

extern "C" {

int mdl_batch_create(int64_t hbm_budget_bytes, int autotune, mdl_batch** out) {
    if (!out) return MDL_E_ARG;
    *out = nullptr;
    mdl_batch* b = new (std::nothrow) mdl_batch();
    if (!b) return MDL_E_NOMEM;
    if (hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            g_batch_err = "cudaMemGetInfo failed";
            delete b;
            return MDL_E_CUDA;
        }
        hbm_budget_bytes = (int64_t)(fr * 0.9);
    }
    b->budget = hbm_budget_bytes;
    b->autotune = autotune ? 1 : 0;
    *out = b;
    return MDL_OK;
}

int mdl_batch_footprint(const mdl_problem* prob, int64_t* bytes) {
    std::string why;
    int rc = mdl::check_problem(prob, &why);
    if (rc) {
        g_batch_err = why;
        return rc;
    }
    if (bytes) *bytes = mdl::estimate_footprint(*prob);
    return MDL_OK;
}

int mdl_batch_admit(mdl_batch* b, const mdl_problem* prob, const double* V0, const double* s0, int64_t n_dof,
                    double t_end, int32_t* slot) {
    if (!b || !prob || !slot) return MDL_E_ARG;
    std::string why;
    int rc = mdl::check_problem(prob, &why);
    if (rc) {
        b->err = why;
        return rc;
    }
    const int64_t est = mdl::estimate_footprint(*prob);
    if (b->used + est > b->budget) {
        b->err = "footprint does not fit the batch budget";
        return MDL_E_NOSPACE;
    }
    mdl_ctx* c = nullptr;
    rc = mdl_create(prob, &c);
    if (rc) {
        b->err = mdl_last_error(nullptr);
        return rc;
    }
    if (V0) {
        rc = c->impl->set_initial(V0, s0, n_dof);
        if (rc) {
            b->err = c->impl->err;
            mdl_destroy(c);
            return rc;
        }
    }
    const int key = class_key(*prob);
    if (b->autotune) {
        auto it = b->shapes.find(key);
        if (it == b->shapes.end()) {
            // tune on a temporary copy of the instance, which is stepped and discarded
            std::pair<int, int> best{128, 16};
            mdl_ctx* tmp = nullptr;
            if (mdl_create(prob, &tmp) == MDL_OK) {
                if (!V0 || tmp->impl->set_initial(V0, s0, n_dof) == MDL_OK) {
                    if (tune(tmp, 3, &best) != MDL_OK) best = {128, 16};
                }
                mdl_destroy(tmp);
            }
            b->shapes[key] = best;
            it = b->shapes.find(key);
        }
        c->impl->set_tick_shape(it->second.first, it->second.second);
    }
    int id = -1;
    for (size_t i = 0; i < b->slots.size(); ++i)
        if (b->slots[i].state == MDL_SLOT_FREE) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        id = (int)b->slots.size();
        b->slots.emplace_back();
    }
    mdl_batch::Slot& s = b->slots[id];
    s = mdl_batch::Slot{};
    s.ctx = c;
    s.t_end = t_end;
    s.bytes = std::max<int64_t>(est, c->impl->device_bytes());
    double t = 0, dt = 0;
    int64_t nb = 0;
    c->impl->get_time(&t, &nb, &dt);
    s.barriers_total = barriers_to(dt, t, t_end);
    s.state = s.barriers_total > 0 ? MDL_SLOT_RUNNING : MDL_SLOT_DONE;
    b->used += s.bytes;
    *slot = id;
    return MDL_OK;
}

int mdl_batch_step(mdl_batch* b, int64_t barriers_per_slot, double wall_budget_s, int64_t* barriers_done) {
    if (!b || barriers_per_slot < 1) return MDL_E_ARG;
    if (barriers_done) *barriers_done = 0;
    const auto t0 = std::chrono::steady_clock::now();
    int64_t total = 0;
    for (;;) {
        std::vector<int> launched;
        for (size_t i = 0; i < b->slots.size(); ++i) {
            mdl_batch::Slot& s = b->slots[i];
            if (s.state != MDL_SLOT_RUNNING) continue;
            double t = 0, dt = 0;
            int64_t nb = 0;
            s.ctx->impl->get_time(&t, &nb, &dt);
            const int64_t rem = barriers_to(dt, t, s.t_end);
            if (rem <= 0) {
                s.state = MDL_SLOT_DONE;
                continue;
            }
            const int rc = s.ctx->impl->begin_barriers(std::min(rem, barriers_per_slot));
            if (rc) {
                s.state = MDL_SLOT_FAILED;
                s.rc = rc;
                continue;
            }
            launched.push_back((int)i);
        }
        for (int i : launched) {
            mdl_batch::Slot& s = b->slots[i];
            int64_t c = 0;
            const int rc = s.ctx->impl->end_barriers(&c);
            total += c;
            s.barriers_done += c;
            if (rc) {
                s.state = MDL_SLOT_FAILED;
                s.rc = rc;
                continue;
            }
            double t = 0, dt = 0;
            int64_t nb = 0;
            s.ctx->impl->get_time(&t, &nb, &dt);
            if (barriers_to(dt, t, s.t_end) <= 0) s.state = MDL_SLOT_DONE;
            s.bytes = std::max<int64_t>(s.bytes, s.ctx->impl->device_bytes());
        }
        b->steps++;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (launched.empty() || wall_budget_s <= 0 || el >= wall_budget_s) break;
    }
    if (barriers_done) *barriers_done = total;
    return MDL_OK;
}

int mdl_batch_poll(mdl_batch* b, int32_t* done_slots, int32_t cap, int32_t* n) {
    if (!b || !n) return MDL_E_ARG;
    int k = 0;
    for (size_t i = 0; i < b->slots.size(); ++i) {
        mdl_batch::Slot& s = b->slots[i];
        if ((s.state == MDL_SLOT_DONE || s.state == MDL_SLOT_FAILED) && !s.polled) {
            if (k < cap && done_slots) {
                done_slots[k] = (int32_t)i;
                s.polled = true;
            }
            ++k;
        }
    }
    *n = std::min(k, cap);
    return MDL_OK;
}

int mdl_batch_slot(mdl_batch* b, int32_t slot, mdl_ctx** ctx, int32_t* state, int32_t* rc) {
    if (!b || slot < 0 || slot >= (int32_t)b->slots.size() || b->slots[slot].state == MDL_SLOT_FREE)
        return MDL_E_ARG;
    const mdl_batch::Slot& s = b->slots[slot];
    if (ctx) *ctx = s.ctx;
    if (state) *state = s.state;
    if (rc) *rc = s.rc;
    return MDL_OK;
}

int mdl_batch_release(mdl_batch* b, int32_t slot) {
    if (!b || slot < 0 || slot >= (int32_t)b->slots.size() || b->slots[slot].state == MDL_SLOT_FREE)
        return MDL_E_ARG;
    mdl_batch::Slot& s = b->slots[slot];
    mdl_destroy(s.ctx);
    b->used -= s.bytes;
    s = mdl_batch::Slot{};
    return MDL_OK;
}

int mdl_batch_usage(const mdl_batch* b, int64_t* used, int64_t* budget, int32_t* resident) {
    if (!b) return MDL_E_ARG;
    if (used) *used = b->used;
    if (budget) *budget = b->budget;
    if (resident) {
        int r = 0;
        for (const auto& s : b->slots)
            if (s.state != MDL_SLOT_FREE) ++r;
        *resident = r;
    }
    return MDL_OK;
}

int mdl_batch_shape(const mdl_batch* b, const mdl_problem* prob, int32_t* threads, int32_t* blocks_per_sm) {
    if (!b || !prob) return MDL_E_ARG;
    auto it = b->shapes.find(class_key(*prob));
    if (it == b->shapes.end()) return MDL_E_STATE;
    if (threads) *threads = it->second.first;
    if (blocks_per_sm) *blocks_per_sm = it->second.second;
    return MDL_OK;
}

const char* mdl_batch_last_error(const mdl_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void mdl_batch_destroy(mdl_batch* b) {
    if (!b) return;
    for (auto& s : b->slots)
        if (s.ctx) mdl_destroy(s.ctx);
    delete b;
}

int mdl_set_tick_shape(mdl_ctx* ctx, int32_t threads, int32_t blocks_per_sm) {
    if (!ctx || !ctx->impl) return MDL_E_ARG;
    const int rc = ctx->impl->set_tick_shape(threads, blocks_per_sm);
    if (rc) ctx->err = ctx->impl->err;
    return rc;
}

int mdl_set_sweep_variant(mdl_ctx* ctx, int32_t variant) {
    if (!ctx || !ctx->impl) return MDL_E_ARG;
    const int rc = ctx->impl->set_sweep_variant(variant);
    if (rc) ctx->err = ctx->impl->err;
    return rc;
}

int mdl_set_sweep_blocks(mdl_ctx* ctx, int32_t max_blocks) {
    if (!ctx || !ctx->impl) return MDL_E_ARG;
    const int rc = ctx->impl->set_sweep_blocks(max_blocks);
    if (rc) ctx->err = ctx->impl->err;
    return rc;
}

}  // extern "C"
