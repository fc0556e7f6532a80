// mdl_batch.cpp -- many resident simulations stepped together on one GPU.
//
// Each slot is an ordinary context with its own stream and captured phase graphs.
// Admission is by device-memory footprint against the batch's budget.  Two ways to step:
//   fused (the default): a round advances every running slot by one barrier step; each
//     slot launches the phases before its sweep on its own stream, then ONE fused sweep
//     (mdl_fused.h) per element class and precision covers the due elements of all the
//     slots of that class, tick by global tick, replayed from a CUDA graph captured for the
//     batch's composition (each class on its own stream, so the classes' sweeps overlap);
//     then each slot's epilogue.  The rounds of one mdl_batch_step run
//     back to back: the host waits for the device once, after the last.  Per class, the
//     first rounds of the batch time every candidate on the batch itself -- launch shapes of
//     the fused kernel (threads per block, due elements per work item) and "own sweeps"
//     (each slot's own sweep variant on its own stream, e.g. the tensor-core sweep of a Q2
//     3D FP32 slot) -- and keep the fastest.  A fused element takes the step of the
//     thread-per-element sweep, so an instance gives the values it gives alone with that
//     sweep up to the FP32 rounding of the two kernels' compilations; with own sweeps it
//     gives the bits it gives alone.
//   streams: every slot launches its own barriers (its own sweep variant) on its own
//     stream before any is waited for, so their kernels overlap on the device; the sweep
//     launch shape is tuned once per class on a temporary copy of the first admitted
//     instance, and an instance gives the same bits alone and in the mix.
#include <cuda_runtime.h>

#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <map>
#include <string>
#include <vector>

#include "../../include/mdl.h"
#include "mdl_ctx.h"
#include "mdl_fused_api.h"

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
        int group = 0;          // fused group: (precision 64) * 4 + element class
        bool own = false;       // this round's sweep: the slot's own (not the fused kernel)
    };
    int64_t budget = 0;
    int64_t used = 0;
    int autotune = 1;
    std::vector<Slot> slots;
    std::map<int, std::pair<int, int>> shapes;   // class -> (threads, blocks per SM)
    std::string err;
    int64_t steps = 0;
    // fused rounds
    int fused = 1;
    std::vector<cudaEvent_t> sev;                 // per slot: phases before the sweep done
    struct Group {                                // slots of one (precision, element class)
        int precision = 32, cls = 0;
        std::vector<int> members;                 // slot ids of the current round
        std::vector<unsigned char> host;          // records of the round (host copy)
        unsigned char* hpin = nullptr;            // pinned staging for uploads
        size_t pin_cap = 0;
        // Uploaded records with the sweep graph captured for them.  Records change only when
        // a slot's state set or capacity does; two entries hold an adapting batch's two sets.
        // A group of more than FUSED_MAX_SLOTS slots sweeps in chunks of that many, one
        // launch sequence per chunk.
        struct Entry {
            std::vector<unsigned char> bytes;
            void* dev = nullptr;
            size_t cap = 0;
            cudaGraphExec_t graph = nullptr;
            std::vector<long long> key;
            int64_t last = -1;
        };
        struct Chunk {
            Entry entry[2];
        };
        std::vector<Chunk> chunks;
        mdl::FusedShape shape{128, 256, 0};
        bool own = false;                         // tuned: each slot's own sweep
        int tuned = 0;                            // candidate rounds timed so far (-1: done)
        std::vector<double> cand_ms;              // measured ms per candidate
        cudaStream_t st = nullptr;                // the group's stream: its fused sweeps
        cudaEvent_t done = nullptr;               // the group's sweep of the round done
        cudaEvent_t t0 = nullptr, t1 = nullptr;   // tuner timing of the current round
        bool timed = false;
        double best_ms = 0, worst_ms = 0, own_ms = 0;
    };
    Group groups[8];                              // (precision 32 / 64) x element class
    int64_t fused_rounds = 0, fused_launches = 0;
    ~mdl_batch() {
        for (auto& g : groups) {
            for (auto& c : g.chunks)
                for (auto& e : c.entry) {
                    if (e.graph) cudaGraphExecDestroy(e.graph);
                    if (e.dev) cudaFree(e.dev);
                }
            if (g.hpin) cudaFreeHost(g.hpin);
            if (g.t0) cudaEventDestroy(g.t0);
            if (g.t1) cudaEventDestroy(g.t1);
            if (g.done) cudaEventDestroy(g.done);
            if (g.st) cudaStreamDestroy(g.st);
        }
        for (auto e : sev)
            if (e) cudaEventDestroy(e);
    }
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

// Candidate launch shapes of the fused sweep: threads per block, due elements per work
// item.  One more candidate follows them: each slot's own sweep on its own stream.
const int kFusedShapes[][2] = {{128, 128}, {128, 512}, {256, 256}, {256, 1024}, {64, 256}, {128, 2048}};
constexpr int kFusedCands = (int)(sizeof(kFusedShapes) / sizeof(kFusedShapes[0]));
constexpr int kOwnCand = kFusedCands;
constexpr int kCands = kFusedCands + 1;
constexpr int kRoundsPerCand = 2;

int sm_count() {
    int dev = 0, n = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

// Finish a slot's barriers after end_barriers-style completion (shared by both modes).
void settle(mdl_batch::Slot& s, int rc, int64_t c, int64_t* total) {
    *total += c;
    s.barriers_done += c;
    if (rc) {
        s.state = MDL_SLOT_FAILED;
        s.rc = rc;
        return;
    }
    double t = 0, dt = 0;
    int64_t nb = 0;
    s.ctx->impl->get_time(&t, &nb, &dt);
    if (barriers_to(dt, t, s.t_end) <= 0) s.state = MDL_SLOT_DONE;
    s.bytes = std::max<int64_t>(s.bytes, s.ctx->impl->device_bytes());
}

#define MDL_BCK(x)                                                  \
    do {                                                            \
        cudaError_t e_ = (x);                                       \
        if (e_ != cudaSuccess) {                                    \
            b->err = std::string(#x) + ": " + cudaGetErrorString(e_); \
            return MDL_E_CUDA;                                      \
        }                                                           \
    } while (0)

bool tuning(const mdl_batch* b) {
    if (!b->autotune) return false;
    for (const auto& g : b->groups)
        if (g.tuned >= 0 && !g.members.empty()) return true;
    return false;
}

// The candidate a group runs this round (-1: its tuned choice).
int candidate(const mdl_batch* b, const mdl_batch::Group& g) {
    return b->autotune && g.tuned >= 0 ? g.tuned / kRoundsPerCand : -1;
}

// Chunk c of the group's fused sweep of this round (records host[0 .. n), already holding
// their shifts) from its captured graph, uploading the records and capturing first when
// they or the launch shape changed.  The group's pinned staging holds every chunk's records
// at the chunk's own offset.
int fused_group_sweep(mdl_batch* b, mdl_batch::Group& g, int c, const unsigned char* host, int n, int Bmax,
                      int threads, int tile, int nsm) {
    const size_t bytes = mdl::fused_slot_bytes(g.precision);
    const size_t nb = (size_t)n * bytes;
    if ((int)g.chunks.size() <= c) g.chunks.resize(c + 1);
    mdl_batch::Group::Chunk& ch = g.chunks[c];
    mdl_batch::Group::Entry* E = nullptr;
    for (auto& e : ch.entry)
        if (e.dev && e.bytes.size() == nb && memcmp(e.bytes.data(), host, nb) == 0) E = &e;
    if (!E) {
        E = ch.entry[0].last <= ch.entry[1].last ? &ch.entry[0] : &ch.entry[1];
        // the entry's buffer and the staging are idle once the group's stream is
        MDL_BCK(cudaStreamSynchronize(g.st));
        if (nb > E->cap) {
            if (E->graph) cudaGraphExecDestroy(E->graph);
            E->graph = nullptr;
            if (E->dev) cudaFree(E->dev);
            E->dev = nullptr;
            E->cap = 0;
            const size_t c = std::max<size_t>(nb * 2, 16 * bytes);
            MDL_BCK(cudaMalloc(&E->dev, c));
            E->cap = c;
        }
        const size_t off = (size_t)c * mdl::FUSED_MAX_SLOTS * bytes;
        if (off + nb > g.pin_cap) {
            if (g.hpin) cudaFreeHost(g.hpin);
            g.hpin = nullptr;
            g.pin_cap = 0;
            const size_t cp = std::max<size_t>((off + nb) * 2, 16 * bytes);
            MDL_BCK(cudaMallocHost((void**)&g.hpin, cp));
            g.pin_cap = cp;
        }
        memcpy(g.hpin + off, host, nb);
        MDL_BCK(cudaMemcpyAsync(E->dev, g.hpin + off, nb, cudaMemcpyHostToDevice, g.st));
        E->bytes.assign(host, host + nb);
    }
    E->last = b->fused_rounds;
    const int blocks = nsm * mdl::fused_blocks_per_sm(g.precision, g.cls, threads);
    const std::vector<long long> key{n, Bmax, threads, tile, blocks, (long long)(uintptr_t)E->dev};
    if (!E->graph || key != E->key) {
        if (E->graph) cudaGraphExecDestroy(E->graph);
        E->graph = nullptr;
        cudaGraph_t graph;
        MDL_BCK(cudaStreamBeginCapture(g.st, cudaStreamCaptureModeThreadLocal));
        const cudaError_t el = mdl::fused_sweep(g.precision, g.cls, E->dev, n, Bmax,
                                                mdl::FusedShape{threads, tile, blocks}, g.st);
        const cudaError_t ec = cudaStreamEndCapture(g.st, &graph);
        MDL_BCK(el);
        MDL_BCK(ec);
        const cudaError_t ei = cudaGraphInstantiate(&E->graph, graph, 0);
        cudaGraphDestroy(graph);
        MDL_BCK(ei);
        E->key = key;
    }
    MDL_BCK(cudaGraphLaunch(E->graph, g.st));
    b->fused_launches += 1 << Bmax;
    return MDL_OK;
}

// Issue one fused round over the running slots `run` (each advances one barrier step);
// completion is left to fused_complete().
int fused_issue(mdl_batch* b, const std::vector<int>& run) {
    while (b->sev.size() < b->slots.size()) {
        cudaEvent_t e = nullptr;
        MDL_BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->sev.push_back(e);
    }
    for (auto& g : b->groups) {
        g.members.clear();
        g.host.clear();
        g.timed = false;
    }
    // the phases before the sweep, each slot on its own stream; a slot of a group tuned to
    // own sweeps goes straight on with its sweep
    std::vector<int> Bs(b->slots.size(), 0);
    std::vector<int> begun;
    std::vector<unsigned char> scratch;
    for (int i : run) {
        mdl_batch::Slot& s = b->slots[i];
        mdl_batch::Group& g = b->groups[s.group];
        const int c = candidate(b, g);
        // a mapped slot always sweeps on its own and is no member of its group
        const bool alone = s.ctx->impl->is_mapped();
        s.own = alone || (c >= 0 ? c == kOwnCand : g.own);
        const size_t bytes = mdl::fused_slot_bytes(g.precision);
        const size_t off = g.host.size();
        unsigned char* rec;
        if (alone) {
            scratch.resize(bytes);
            rec = scratch.data();
        } else {
            g.host.resize(off + bytes);
            rec = g.host.data() + off;
        }
        int rc = s.ctx->impl->fused_begin(rec, &Bs[i]);
        if (!rc && s.own && (c < 0 || alone)) rc = s.ctx->impl->fused_own_sweep();
        if (rc) {
            if (!alone) g.host.resize(off);
            s.state = MDL_SLOT_FAILED;
            s.rc = rc;
            continue;
        }
        MDL_BCK(cudaEventRecord(b->sev[i], (cudaStream_t)s.ctx->impl->stream_handle()));
        if (!alone) g.members.push_back(i);
        begun.push_back(i);
    }
    // per (precision, class) group, on the group's own stream (the groups' sweeps overlap):
    // one fused sweep from its captured graph, or (timed while tuning) the slots' own sweeps.
    // While tuning, the groups' sweeps run one after another so that each is timed alone.
    const int nsm = sm_count();
    const bool serial = tuning(b);
    cudaEvent_t prev = nullptr;
    for (auto& g : b->groups) {
        const int n = (int)g.members.size();
        if (n == 0) continue;
        const int c = candidate(b, g);
        if (c < 0 && g.own) continue;
        if (!g.st) {
            MDL_BCK(cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking));
            MDL_BCK(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
        }
        for (int i : g.members) MDL_BCK(cudaStreamWaitEvent(g.st, b->sev[i], 0));
        if (serial && prev) MDL_BCK(cudaStreamWaitEvent(g.st, prev, 0));
        if (c >= 0) {
            if (!g.t0) {
                MDL_BCK(cudaEventCreate(&g.t0));
                MDL_BCK(cudaEventCreate(&g.t1));
            }
            MDL_BCK(cudaEventRecord(g.t0, g.st));
            g.timed = true;
        }
        if (c == kOwnCand) {
            for (int i : g.members) {
                mdl_batch::Slot& s = b->slots[i];
                cudaStream_t ss = (cudaStream_t)s.ctx->impl->stream_handle();
                MDL_BCK(cudaStreamWaitEvent(ss, g.t0, 0));
                const int rc = s.ctx->impl->fused_own_sweep();
                if (rc) {
                    s.state = MDL_SLOT_FAILED;
                    s.rc = rc;
                }
                MDL_BCK(cudaEventRecord(b->sev[i], ss));
                MDL_BCK(cudaStreamWaitEvent(g.st, b->sev[i], 0));
            }
        } else {
            const size_t bytes = mdl::fused_slot_bytes(g.precision);
            const int threads = c >= 0 ? kFusedShapes[c][0] : g.shape.threads;
            const int tile = c >= 0 ? kFusedShapes[c][1] : g.shape.tile;
            for (int c0 = 0, ci = 0; c0 < n; c0 += mdl::FUSED_MAX_SLOTS, ++ci) {
                const int nc = std::min(n - c0, mdl::FUSED_MAX_SLOTS);
                int Bmax = 0;
                for (int k = c0; k < c0 + nc; ++k) Bmax = std::max(Bmax, Bs[g.members[k]]);
                for (int k = c0; k < c0 + nc; ++k)
                    mdl::fused_set_shift(g.host.data() + k * bytes, g.precision, Bmax - Bs[g.members[k]]);
                const int rc = fused_group_sweep(b, g, ci, g.host.data() + c0 * bytes, nc, Bmax, threads, tile, nsm);
                if (rc) return rc;
            }
        }
        if (c >= 0) MDL_BCK(cudaEventRecord(g.t1, g.st));
        MDL_BCK(cudaEventRecord(g.done, g.st));
        prev = g.done;
    }
    // each slot's epilogue after its sweep
    for (int i : begun) {
        mdl_batch::Slot& s = b->slots[i];
        if (s.state == MDL_SLOT_FAILED) continue;
        if (!s.own) MDL_BCK(cudaStreamWaitEvent((cudaStream_t)s.ctx->impl->stream_handle(), b->groups[s.group].done, 0));
        const int rc = s.ctx->impl->fused_finish();
        if (rc) {
            s.state = MDL_SLOT_FAILED;
            s.rc = rc;
        }
    }
    b->fused_rounds++;
    return MDL_OK;
}

// Wait for the rounds issued since the last completion: complete every slot that took part
// and, while tuning, add the round's timings to the candidates (after the last, keep the best).
int fused_complete(mdl_batch* b, const std::vector<char>& took_part, int64_t* total) {
    for (size_t i = 0; i < b->slots.size(); ++i) {
        mdl_batch::Slot& s = b->slots[i];
        if (!took_part[i] || s.state == MDL_SLOT_FAILED) continue;
        int64_t c = 0;
        const int rc = s.ctx->impl->end_barriers(&c);
        settle(s, rc, c, total);
    }
    for (auto& g : b->groups)
        if (g.st) MDL_BCK(cudaStreamSynchronize(g.st));
    for (auto& g : b->groups) {
        if (!g.timed) continue;
        g.timed = false;
        float ms = 0;
        MDL_BCK(cudaEventElapsedTime(&ms, g.t0, g.t1));
        const int c = g.tuned / kRoundsPerCand;
        if ((int)g.cand_ms.size() < kCands) g.cand_ms.assign(kCands, 0.0);
        g.cand_ms[c] += ms;
        if (++g.tuned == kCands * kRoundsPerCand) {
            int best = 0;
            for (int k = 1; k < kCands; ++k)
                if (g.cand_ms[k] < g.cand_ms[best]) best = k;
            g.own = best == kOwnCand;
            if (!g.own) g.shape = mdl::FusedShape{kFusedShapes[best][0], kFusedShapes[best][1], 0};
            g.best_ms = g.cand_ms[best] / kRoundsPerCand;
            g.worst_ms = *std::max_element(g.cand_ms.begin(), g.cand_ms.end()) / kRoundsPerCand;
            g.own_ms = g.cand_ms[kOwnCand] / kRoundsPerCand;
            g.tuned = -1;
        }
    }
    return MDL_OK;
}

// `rounds` fused rounds (fewer for slots that reach their horizon), issued back to back and
// completed once; while a group is still tuning, each round is completed on its own.
int fused_step(mdl_batch* b, int64_t rounds, int64_t* total) {
    std::vector<int64_t> left(b->slots.size(), 0);
    for (size_t i = 0; i < b->slots.size(); ++i) {
        mdl_batch::Slot& s = b->slots[i];
        if (s.state != MDL_SLOT_RUNNING) continue;
        double t = 0, dt = 0;
        int64_t nb = 0;
        s.ctx->impl->get_time(&t, &nb, &dt);
        left[i] = std::min(rounds, barriers_to(dt, t, s.t_end));
        if (left[i] <= 0) s.state = MDL_SLOT_DONE;
    }
    std::vector<char> took(b->slots.size(), 0);
    bool pending = false;
    for (int64_t r = 0; r < rounds; ++r) {
        std::vector<int> run;
        for (size_t i = 0; i < b->slots.size(); ++i) {
            mdl_batch::Slot& s = b->slots[i];
            if (s.state != MDL_SLOT_RUNNING || left[i] <= 0) continue;
            // replayed inputs hold for one barrier: such a slot takes one round per completion
            if (took[i] && s.ctx->impl->replaying()) continue;
            run.push_back((int)i);
        }
        if (run.empty()) break;
        const bool sync_each = tuning(b);
        int rc = fused_issue(b, run);
        for (int i : run) {
            took[i] = 1;
            --left[i];
        }
        pending = true;
        if (rc) {
            fused_complete(b, took, total);
            return rc;
        }
        if (sync_each || tuning(b)) {
            if ((rc = fused_complete(b, took, total))) return rc;
            std::fill(took.begin(), took.end(), 0);
            pending = false;
            // horizons and failures as of this completion
            for (size_t i = 0; i < b->slots.size(); ++i)
                if (b->slots[i].state != MDL_SLOT_RUNNING) left[i] = 0;
        }
    }
    if (pending) return fused_complete(b, took, total);
    return MDL_OK;
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
    for (int gi = 0; gi < 8; ++gi) {
        b->groups[gi].precision = gi >= 4 ? 64 : 32;
        b->groups[gi].cls = gi & 3;
        b->groups[gi].tuned = b->autotune ? 0 : -1;
    }
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
    if (b->autotune && !b->fused) {
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
    s.group = (prob->precision == 64 ? 4 : 0) + mdl::fused_class(prob->dim, prob->order);
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
    if (b->fused) {
        for (;;) {
            const int rc = fused_step(b, barriers_per_slot, &total);
            if (rc) {
                if (barriers_done) *barriers_done = total;
                return rc;
            }
            b->steps++;
            bool any = false;
            for (const auto& s : b->slots) any = any || s.state == MDL_SLOT_RUNNING;
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (!any || wall_budget_s <= 0 || el >= wall_budget_s) break;
        }
        if (barriers_done) *barriers_done = total;
        return MDL_OK;
    }
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
            settle(s, rc, c, &total);
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

int mdl_batch_set_fused(mdl_batch* b, int32_t on) {
    if (!b) return MDL_E_ARG;
    b->fused = on ? 1 : 0;   // (a batch step completes its rounds before it returns)
    return MDL_OK;
}

int mdl_batch_fused_info(const mdl_batch* b, int32_t precision, int32_t dim, int32_t order, int32_t* own,
                         int32_t* threads, int32_t* tile, double* best_ms, double* worst_ms, double* own_ms,
                         int64_t* rounds, int64_t* launches) {
    if (!b || (precision != 32 && precision != 64) || (dim != 2 && dim != 3) || (order != 1 && order != 2))
        return MDL_E_ARG;
    if (rounds) *rounds = b->fused_rounds;
    if (launches) *launches = b->fused_launches;
    const mdl_batch::Group& g = b->groups[(precision == 64 ? 4 : 0) + mdl::fused_class(dim, order)];
    if (g.tuned != -1) return MDL_E_STATE;
    if (own) *own = g.own ? 1 : 0;
    if (threads) *threads = g.shape.threads;
    if (tile) *tile = g.shape.tile;
    if (best_ms) *best_ms = g.best_ms;
    if (worst_ms) *worst_ms = g.worst_ms;
    if (own_ms) *own_ms = g.own_ms;
    return MDL_OK;
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
