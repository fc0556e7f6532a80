// mdl_ctx_impl.cuh -- context implementation for one (precision R, dim, order).
//
// A barrier step (Alg. 1) is a fixed sequence of kernel launches on the context's
// stream, in four phases that are captured once as CUDA graphs and replayed
// (indicator / adaptation + levels + ordering / sweep / epilogue); element counts, due
// counts per tick, the barrier counter and errors live in device memory (DevMeta), so
// the host never waits inside a barrier:
//   [AMR]  k_eta_s, k_amr_mark, k_amr_close x max_refine, k_amr_family, k_scan_blocks,
//          k_scan_top (commit), k_scan_emit (coordinates into the other state set),
//          k_leaf_keys + k_mesh_tables + k_lat_refresh (in place, only if the mesh changed),
//          k_transfer (state into the other set)
//   levels k_levels_count, k_order_top, k_order_scatter
//   sweep  2^B launches of k_tick (each reads its due count from DevMeta)
//   end    k_epilogue (eta^t, parities, int V by a last-block reduction, counters)
// The state (V slots, v, eta^t, levels, coordinates) is double-buffered across an
// adaptation; the mesh tables are single copies rebuilt in place.
// The host reads DevMeta once at the end of each stepping call.  A capacity overflow
// makes every later kernel skip; the host then grows the buffers and resumes at the
// failed barrier, so results do not depend on the capacity.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <type_traits>
#include <vector>

#include "mdl_amr.cuh"
#include "mdl_ctx.h"
#include "mdl_fused.h"
#include "mdl_kernels.cuh"
#include "mdl_geometry.h"
#include "mdl_mapped.cuh"
#include "mdl_mesh.h"
#include "mdl_tables.h"
#include "mdl_tc.cuh"

namespace mdl {

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t cap = 0;
    // (Re)allocate for n elements; contents are not preserved.
    cudaError_t ensure(size_t n) {
        if (n <= cap && p) return cudaSuccess;
        release();
        const size_t c = n > 0 ? n : 1;
        cudaError_t e = cudaMalloc((void**)&p, c * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            cap = 0;
            return e;
        }
        cap = c;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

#define MDL_CK(x)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess) {                                                    \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? MDL_E_NOMEM : MDL_E_CUDA;      \
        }                                                                           \
    } while (0)

#define MDL_LAUNCHED()                                                              \
    do {                                                                            \
        stats.kernel_launches++;                                                    \
        MDL_CK(cudaGetLastError());                                                 \
    } while (0)

__global__ void k_fill_inf(double* p, int64_t n);

template <typename R, int DIM, int P>
class Ctx : public CtxBase {
    using S = Shape<DIM, P>;
    static constexpr int N1 = S::N1, NP = S::NP, NF = S::NF, NSUB = S::NSUB, NC = 1 << DIM, NPS = S::NPS;

    // State of one mesh (double-buffered across an adaptation).
    struct Set {
        DBuf<R> V0, V1, v;
        DBuf<double> eta_t;
        DBuf<uint8_t> lvl;
        DBuf<int4> coord;
        // mapped meshes: each element's geometric factors, GL masses, signature (face kinds,
        // level, b^CFL) and stimulus masks, which follow the element through adaptations
        DBuf<R> gvol, gface;
        DBuf<double> mq;
        DBuf<uint32_t> fsig;
        DBuf<uint32_t> fsm[MDL_MAX_STIM];
        void release() {
            V0.release(); V1.release(); v.release(); eta_t.release(); lvl.release(); coord.release();
            gvol.release(); gface.release(); mq.release(); fsig.release();
            for (auto& m : fsm) m.release();
        }
    };

    mdl_problem pb{};
    Tables<double> Td{};
    Phys<double> phd{};
    Tables<R> T{};
    Phys<R> ph{};
    Grid grid_{};
    StimBoxes sboxes{};
    StimArgs stim{};
    double dt = 0;
    int B = 0;
    int nsm = 1;
    int64_t cap = 0;          // element capacity of every per-element array
    int64_t ne = 0;           // host copy of the element count (valid after sync)
    int64_t nbar = 0;         // host copy of the barrier count (valid after sync)
    int64_t n_probe = 0;
    cudaStream_t st = nullptr;
    Set sets[2];
    int cs = 0;
    DBuf<R> Ia, ga;
    DBuf<double> acc, eta_s, lat, partial, scratch;
    DBuf<float> fscratch;   // FP32 field transfers
    DBuf<R> cview;          // compact copy handed out by device_view for padded rows
    DBuf<uint8_t> r, c0, class_b;
    DBuf<int32_t> bcnt, psrc;
    DBuf<uint64_t> lkey;      // sort key of every leaf (neighbour search of the mesh tables)
    DBuf<int64_t> bsum;
    // mesh tables (single copies)
    DBuf<uint8_t> bcfl;
    DBuf<uint32_t> info, loc;
    DBuf<int32_t> nbr, hang, root, order;
    DBuf<uint32_t> smask[MDL_MAX_STIM];
    DBuf<int8_t> pkind, pbits, lvl_ovr;
    DBuf<int32_t> ftodo;   // curved meshes: elements whose factors an adaptation recomputes
    DBuf<double> eta_t_ovr;
    DBuf<double> mtab;   // FP64 GL mass w_q det J per (level, node); mapped: per (element, node)
    DBuf<R> qvol, qface, qkelly;   // Q1 class blocks
    bool mapped = false;           // curved mesh (mdl_geometry.h): per-element factors in the sets
    MapArgs margs{};               // its map, diffusion, GL nodes and stimulus boxes for k_mapped_factors
    DBuf<uint16_t> tcB;            // Q2 3D FP32: level-0 operator of the tensor-core sweep (FP16 hi/lo)
    float tc_unscale = 1.0f;       // 2^-t: undoes the scaling of the operator by 2^t
    DBuf<float> tcC;               // Q2 3D FP32: level-0 correction blocks of non-regular faces
    DBuf<DevMeta> meta;
    DBuf<Tables<R>> dT;       // device copies of the tables and physics (fused batch sweeps)
    DBuf<Phys<R>> dph;
    int fused_cur = 0;        // state set the fused sweep of the barrier in flight updates
    bool fused_own = false;   // this round's sweep is the context's own (fused_own_sweep)
    DevMeta* hmeta = nullptr;
    bool ovr_levels = false, ovr_eta_s = false, ovr_eta_t = false;
    bool timing = false;
    std::vector<cudaEvent_t> evpool;
    size_t ev_used = 0;
    struct EvSet {
        cudaEvent_t a, b, c, d;
    };
    std::vector<EvSet> pending_ev;
    mdl_stats stats{};
    // captured phase graphs, per phase and state set (an adapting barrier swaps sets)
    cudaGraphExec_t gexec[4][2] = {};
    int64_t gcap[4][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
    int64_t glaunch[4][2] = {};
    int64_t gticks[4][2] = {};
    bool use_graphs = true;
    int tick_threads = 128, tick_bpsm = 16;   // sweep launch shape
    bool coop_sweep = false;                  // ticks + epilogue in one cooperative launch
    bool group_tick = false;                  // Q1: a group of (p+1)^d lanes per element
    bool tensor_tick = false;                 // Q2 3D FP32: element residual on the tensor cores
    int sweep_blocks = 0;                     // bound on the tensor sweep's blocks (0: default)
    bool pdl = true;                          // programmatic dependent launch between kernels
    int64_t inflight = 0, inflight_start = 0; // barriers launched by begin_barriers

    static int div_up(int64_t n, int64_t b) { return (int)((n + b - 1) / b); }
    // Launch a barrier-step kernel on the context's stream.  With pdl set, the launch
    // allows programmatic dependent launch: the kernel's blocks may be scheduled while
    // its predecessor drains, and every such kernel starts with pdl_enter(), which waits
    // for the predecessor to complete (its writes visible) before touching any data.
    template <typename... KP, typename... Args>
    cudaError_t launch_k(void (*k)(KP...), int grid, int block, Args&&... args) {
        return launch_kx(pdl, k, grid, block, std::forward<Args>(args)...);
    }

    template <typename... KP, typename... Args>
    cudaError_t launch_kx(bool overlap, void (*k)(KP...), int grid, int block, Args&&... args) {
        return launch_kxs(overlap, 0, k, grid, block, std::forward<Args>(args)...);
    }

    template <typename... KP, typename... Args>
    cudaError_t launch_kxs(bool overlap, size_t dyn_smem, void (*k)(KP...), int grid, int block, Args&&... args) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)block);
        cfg.dynamicSmemBytes = dyn_smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = overlap ? 1 : 0;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
    }

    int persistent_blocks(int threads) const {
        const int64_t need = div_up(std::max<int64_t>(cap, 1), threads);
        return (int)std::min<int64_t>(need, (int64_t)nsm * (2048 / threads));
    }

    static constexpr bool tensor_capable = std::is_same<R, float>::value && DIM == 3 && P == 2;

    DevArrays<R> arrays(int s) {
        DevArrays<R> d{};
        Set& x = sets[s];
        d.V0 = x.V0.p; d.V1 = x.V1.p; d.v = x.v.p; d.eta_t = x.eta_t.p; d.lvl = x.lvl.p;
        d.Ia = Ia.p; d.ga = ga.p; d.acc = acc.p; d.eta_s = eta_s.p; d.lat = lat.p;
        d.partial = partial.p; d.bcfl = bcfl.p; d.info = info.p; d.nbr = nbr.p; d.hang = hang.p;
        d.order = order.p; d.root = root.p; d.loc = loc.p;
        for (int k = 0; k < MDL_MAX_STIM; ++k) d.smask[k] = smask[k].p;
        d.meta = meta.p;
        d.qvol = qvol.p;
        d.qface = qface.p;
        d.qkelly = qkelly.p;
        d.gvol = x.gvol.p;
        d.gface = x.gface.p;
        d.mq = mapped ? x.mq.p : nullptr;
        return d;
    }

    // ------------------------------------------------------------------
    // Allocation.  Growing keeps the current set's contents.
    static constexpr int MAP_VOL = NP * (DIM * (DIM + 1) / 2 + 1);      // factor values per element
    static constexpr int MAP_FACE = NF * (DIM == 2 ? N1 : N1 * N1) * (DIM + 2);

    int alloc_set(Set& x, int64_t c) {
        MDL_CK(x.V0.ensure((size_t)c * NPS));
        MDL_CK(x.V1.ensure((size_t)c * NPS));
        MDL_CK(x.v.ensure((size_t)c * NPS));
        MDL_CK(x.eta_t.ensure(c));
        MDL_CK(x.lvl.ensure(c));
        MDL_CK(x.coord.ensure(c));
        if (mapped) {
            MDL_CK(x.gvol.ensure((size_t)c * MAP_VOL));
            MDL_CK(x.gface.ensure((size_t)c * MAP_FACE));
            MDL_CK(x.mq.ensure((size_t)c * NP));
            MDL_CK(x.fsig.ensure(c));
            for (int s = 0; s < pb.n_stim; ++s) MDL_CK(x.fsm[s].ensure(c));
        }
        return MDL_OK;
    }

    int alloc_tables(int64_t c) {
        MDL_CK(bcfl.ensure(c));
        MDL_CK(info.ensure(c));
        MDL_CK(loc.ensure(c));
        MDL_CK(nbr.ensure((size_t)c * NF));
        MDL_CK(hang.ensure((size_t)c * NF * NSUB));
        MDL_CK(root.ensure(c));
        MDL_CK(order.ensure(c));
        MDL_CK(lkey.ensure(c));
        for (int s = 0; s < pb.n_stim; ++s) MDL_CK(smask[s].ensure(c));
        return MDL_OK;
    }

    int alloc_shared(int64_t c) {
        MDL_CK(Ia.ensure((size_t)c * NPS));
        MDL_CK(ga.ensure((size_t)c * NPS));
        MDL_CK(acc.ensure(c));
        MDL_CK(eta_s.ensure(c));
        MDL_CK(r.ensure(c));
        MDL_CK(c0.ensure(c));
        MDL_CK(bsum.ensure(div_up(c, SCAN_CHUNK) + 1));
        MDL_CK(bcnt.ensure((size_t)(div_up(c, ORD_THREADS) + 1) * 8 + 8));
        MDL_CK(pkind.ensure(c));
        MDL_CK(pbits.ensure(c));
        MDL_CK(psrc.ensure(c));
        if (mapped) MDL_CK(ftodo.ensure(c));
        MDL_CK(partial.ensure((size_t)nsm * 16 + 1024));
        return MDL_OK;
    }

    template <class T2>
    int grow_copy(DBuf<T2>& b, size_t n_new, size_t n_keep) {
        DBuf<T2> nb;
        MDL_CK(nb.ensure(n_new));
        if (n_keep && b.p) MDL_CK(cudaMemcpyAsync(nb.p, b.p, n_keep * sizeof(T2), cudaMemcpyDeviceToDevice, st));
        MDL_CK(cudaStreamSynchronize(st));
        b.release();
        b.p = nb.p;
        b.cap = nb.cap;
        nb.p = nullptr;
        nb.cap = 0;
        return MDL_OK;
    }

    int grow(int64_t need) {
        const int64_t c = std::max<int64_t>(need + need / 2, cap * 2);
        Set& x = sets[cs];
        int rc;
#define MDL_GROW(buf, per) if ((rc = grow_copy(buf, (size_t)c * (per), (size_t)ne * (per)))) return rc
        MDL_GROW(x.V0, NPS); MDL_GROW(x.V1, NPS); MDL_GROW(x.v, NPS); MDL_GROW(x.eta_t, 1);
        MDL_GROW(x.lvl, 1); MDL_GROW(x.coord, 1);
        if (mapped) {
            MDL_GROW(x.gvol, MAP_VOL); MDL_GROW(x.gface, MAP_FACE); MDL_GROW(x.mq, NP); MDL_GROW(x.fsig, 1);
            for (int s = 0; s < pb.n_stim; ++s) MDL_GROW(x.fsm[s], 1);
        }
        MDL_GROW(bcfl, 1); MDL_GROW(info, 1); MDL_GROW(loc, 1); MDL_GROW(nbr, NF); MDL_GROW(hang, NF * NSUB);
        MDL_GROW(root, 1); MDL_GROW(order, 1); MDL_GROW(lkey, 1);
        for (int s = 0; s < pb.n_stim; ++s) MDL_GROW(smask[s], 1);
        MDL_GROW(eta_s, 1);
#undef MDL_GROW
        sets[cs ^ 1].release();
        if ((rc = alloc_set(sets[cs ^ 1], c))) return rc;
        Ia.release(); ga.release(); acc.release(); r.release(); c0.release();
        bsum.release(); bcnt.release(); pkind.release(); pbits.release(); psrc.release(); ftodo.release();
        if ((rc = alloc_shared(c))) return rc;
        if (lvl_ovr.p && (rc = grow_copy(lvl_ovr, (size_t)c, (size_t)ne))) return rc;
        if (eta_t_ovr.p && (rc = grow_copy(eta_t_ovr, (size_t)c, (size_t)ne))) return rc;
        cap = c;
        drop_graphs();
        return MDL_OK;
    }

    // ------------------------------------------------------------------
    int sync_meta() {
        MDL_CK(cudaMemcpyAsync(hmeta, meta.p, sizeof(DevMeta), cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        ne = hmeta->ne;
        nbar = hmeta->nbar;
        cs = (int)hmeta->cur_set;
        stats.n_elements = ne;
        stats.integral_V = hmeta->integral;
        stats.element_updates = hmeta->elem_updates;
        stats.dof_updates = hmeta->elem_updates * NP;
        stats.amr_rebuilds = hmeta->rebuilds;
        stats.factor_updates = hmeta->fac_updates;
        for (int b = 0; b < 8; ++b) stats.level_counts[b] = hmeta->cnt[b];
        return MDL_OK;
    }

    // Build the mesh tables from the coordinates of set s (device), given ne in DevMeta;
    // unless forced, only when this barrier's adaptation changed the mesh.
    int build_tables(int s, int force) {
        Set& x = sets[s];
        const int gb = persistent_blocks(256);
        MDL_CK(launch_k((k_leaf_keys<DIM>), persistent_blocks(256), 256, x.coord.p, lkey.p, grid_, meta.p, force));
        MDL_LAUNCHED();
        MDL_CK(launch_k((k_mesh_tables<R, DIM, P>), persistent_blocks(128), 128, 
            x.coord.p, lkey.p, grid_, info.p, nbr.p, hang.p, root.p, loc.p, bcfl.p, class_b.p,
            smask[0].p, smask[1].p, smask[2].p, smask[3].p, sboxes, phd, meta.p, force));
        MDL_LAUNCHED();
        return MDL_OK;
    }

    // Upload a (validated, sorted) host mesh into the current set and reset the state.
    int load_mesh(const Mesh& mh) {
        const int64_t n = mh.n();
        if (n > cap) {
            const int64_t c = std::max<int64_t>(n * 2, 4096);
            sets[0].release();
            sets[1].release();
            int rc = alloc_set(sets[0], c);
            if (!rc) rc = alloc_set(sets[1], c);
            if (!rc) rc = alloc_shared(c);
            if (!rc) rc = alloc_tables(c);
            if (rc) return rc;
            cap = c;
            drop_graphs();
        }
        std::vector<int4> hc(n);
        for (int64_t i = 0; i < n; ++i) {
            const Leaf& lf = mh.leaves[i];
            hc[i] = make_int4(lf.c[0], lf.c[1], DIM == 3 ? lf.c[2] : 0, lf.level);
        }
        Set& x = sets[cs];
        MDL_CK(cudaMemcpyAsync(x.coord.p, hc.data(), n * sizeof(int4), cudaMemcpyHostToDevice, st));
        DevMeta init{};
        init.ne = n;
        init.nbar = nbar;
        init.cur_set = (unsigned)cs;
        MDL_CK(cudaMemcpyAsync(meta.p, &init, sizeof(DevMeta), cudaMemcpyHostToDevice, st));
        int rc = build_tables(cs, 1);
        if (rc) return rc;
        ne = n;
        MDL_CK(cudaMemsetAsync(x.V0.p, 0, (size_t)n * NPS * sizeof(R), st));
        MDL_CK(cudaMemsetAsync(x.V1.p, 0, (size_t)n * NPS * sizeof(R), st));
        MDL_CK(cudaMemsetAsync(x.v.p, 0, (size_t)n * NPS * sizeof(R), st));
        MDL_CK(cudaMemsetAsync(x.eta_t.p, 0, n * sizeof(double), st));
        MDL_CK(cudaMemsetAsync(x.lvl.p, 0, n, st));
        MDL_CK(cudaMemsetAsync(eta_s.p, 0, n * sizeof(double), st));
        k_fill_inf<<<div_up(n_probe, 256), 256, 0, st>>>(lat.p, n_probe);
        MDL_LAUNCHED();
        k_lat_refresh<R, DIM, P><<<persistent_blocks(128), 128, 0, st>>>(arrays(cs), T, ph, (double)nbar * dt, 0, 1);
        MDL_LAUNCHED();
        rc = sync_meta();   // the host staging buffer hc must outlive the copy
        if (rc) return rc;
        if (hmeta->err) {
            err = "mesh tables: inconsistent mesh";
            return MDL_E_STATE;
        }
        return MDL_OK;
    }

    // ------------------------------------------------------------------
    cudaEvent_t next_event() {
        if (ev_used == evpool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            evpool.push_back(e);
        }
        return evpool[ev_used++];
    }

    // A barrier step is four phases, each launched directly or replayed from a captured graph:
    //   0 indicator (k_eta_s), 1 adaptation + levels + ordering, 2 sweep ticks, 3 epilogue.
    // Phase 0 only runs with adaptation and no replayed eta^s.  No host synchronisation.
    static constexpr int NPHASE = 4;

    int launch_phase(int ph_, int o) {
        const int g256 = persistent_blocks(256), g128 = persistent_blocks(128);
        if (ph_ == 0) {
            if (mapped) MDL_CK(launch_k((k_eta_s_mapped<R, DIM, P>), g128, 128, arrays(o), T));
            else MDL_CK(launch_k((k_eta_s<R, DIM, P>), g128, 128, arrays(o), T, ph));
            MDL_LAUNCHED();
            return MDL_OK;
        }
        if (ph_ == 1) {
            int cur = o;
            if (pb.amr_enabled) {
                const int n = o ^ 1;
                Set& so = sets[o];
                Set& sn = sets[n];
                MDL_CK(launch_k((k_amr_mark<DIM>), g256, 256, so.coord.p, eta_s.p, r.p, c0.p, meta.p, pb.tau_refine,
                                                      pb.max_refine));
                MDL_LAUNCHED();
                for (int i = 0; i < pb.max_refine; ++i) {
                    MDL_CK(launch_k((k_amr_close<DIM>), g256, 256, info.p, nbr.p, r.p, meta.p));
                    MDL_LAUNCHED();
                }
                MDL_CK(launch_k((k_amr_family<DIM>), g256, 256, so.coord.p, info.p, nbr.p, eta_s.p, r.p, c0.p, meta.p,
                                                        pb.tau_coarsen));
                MDL_LAUNCHED();
                const int nsb = div_up(cap, SCAN_CHUNK);
                MDL_CK(launch_k((k_scan_blocks<DIM>), nsb, SCAN_THREADS, so.coord.p, r.p, c0.p, bsum.p, meta.p));
                MDL_LAUNCHED();
                MDL_CK(launch_k((k_scan_top), 1, 1024, bsum.p, meta.p, cap));
                MDL_LAUNCHED();
                MDL_CK(launch_k((k_scan_emit<DIM>), nsb, SCAN_THREADS, so.coord.p, r.p, c0.p, bsum.p, sn.coord.p,
                                                               pkind.p, psrc.p, pbits.p, meta.p));
                MDL_LAUNCHED();
                DevArrays<R> od = arrays(o);
                int rc = build_tables(n, 0);
                if (rc) return rc;
                if (mapped) {
                    // factors of the new set: copied for elements kept with the same face kinds,
                    // computed for the rest (every barrier: the sets alternate)
                    MDL_CK(launch_k((k_mapped_keep<R, DIM, P>), persistent_blocks(256), 256, info.p, margs.nstim,
                                    sn.gvol.p, sn.gface.p, sn.mq.p, sn.fsig.p, sn.fsm[0].p, sn.fsm[1].p, sn.fsm[2].p,
                                    sn.fsm[3].p, bcfl.p, smask[0].p, smask[1].p, smask[2].p, smask[3].p, so.gvol.p,
                                    so.gface.p, so.mq.p, so.fsig.p, so.fsm[0].p, so.fsm[1].p, so.fsm[2].p,
                                    so.fsm[3].p, (const int8_t*)pkind.p, (const int32_t*)psrc.p, ftodo.p, meta.p));
                    MDL_LAUNCHED();
                    MDL_CK(launch_k((k_mapped_factors<R, DIM, P>), nsm * 8, 64, sn.coord.p, info.p, margs, Td,
                                    sn.gvol.p, sn.gface.p, sn.mq.p, sn.fsig.p, sn.fsm[0].p, sn.fsm[1].p, sn.fsm[2].p,
                                    sn.fsm[3].p, bcfl.p, smask[0].p, smask[1].p, smask[2].p, smask[3].p,
                                    (const int32_t*)ftodo.p, meta.p));
                    MDL_LAUNCHED();
                }
                MDL_CK(launch_k((k_transfer<R, DIM, P>), g128, 128, od, arrays(n), pkind.p, psrc.p, pbits.p, T));
                MDL_LAUNCHED();
                MDL_CK(launch_k((k_lat_refresh<R, DIM, P>), g128, 128, arrays(n), T, ph, 0.0, 0, 0));
                MDL_LAUNCHED();
                cur = n;
            }
            int bcell = 0;
            if (pb.dt_bar_cell > 0) {
                bcell = b_from_bound(dt, pb.dt_bar_cell);
                if (bcell < 0) bcell = 15;
            }
            const double* et = ovr_eta_t ? eta_t_ovr.p : sets[cur].eta_t.p;
            const int nob = div_up(cap, ORD_THREADS);
            MDL_CK(launch_k((k_levels_count<R>), nob, ORD_THREADS, arrays(cur), ovr_levels ? lvl_ovr.p : nullptr, et,
                                                           pb.tau_cell, bcell, B, pb.lts_enabled, bcnt.p));
            MDL_LAUNCHED();
            MDL_CK(launch_k((k_order_top), 1, 1024, bcnt.p, meta.p, B));
            MDL_LAUNCHED();
            MDL_CK(launch_k((k_order_scatter), nob, ORD_THREADS, sets[cur].lvl.p, bcnt.p, order.p, meta.p));
            MDL_LAUNCHED();
            return MDL_OK;
        }
        if (ph_ == 2) {
            TickArgs<R> ta = tick_args(o);
            const int nt = 1 << B;
            if (coop_sweep) {
                // all ticks + epilogue in one cooperative launch (every block resident)
                int occ = 0;
                MDL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep<R, DIM, P>, tick_threads, 0));
                const int per_sm = std::max(1, std::min(occ, tick_bpsm));
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3((unsigned)(nsm * per_sm));
                cfg.blockDim = dim3((unsigned)tick_threads);
                cfg.stream = st;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeCooperative;
                attr[0].val.cooperative = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, gbar), 0, sizeof(unsigned int), st));
                MDL_CK(cudaLaunchKernelEx(&cfg, k_sweep<R, DIM, P>, ta, T, ph, (const double*)mtab.p));
                MDL_LAUNCHED();
                stats.tick_launches += nt;
                return MDL_OK;
            }
            if (mapped) {
                const int gm = (int)std::min<int64_t>(div_up(std::max<int64_t>(cap, 1), 128), (int64_t)nsm * 16);
                for (int i = 0; i < nt; ++i) {
                    ta.tick = i;
                    MDL_CK(launch_kx(pdl && i > 0, (k_tick_mapped<R, DIM, P>), gm, 128, ta, T, ph));
                    MDL_LAUNCHED();
                    stats.tick_launches++;
                }
                return MDL_OK;
            }
            const int lanes = (P == 1 && group_tick) ? NP : 1;
            const int gt = (int)std::min<int64_t>(div_up(std::max<int64_t>(cap, 1) * lanes, tick_threads),
                                                  (int64_t)nsm * tick_bpsm);
            if constexpr (tensor_capable) {
                if (tensor_tick) {
                    // persistent: two blocks per SM walk the tiles of 64 due elements; no more
                    // blocks than the capacity has tiles (a small instance leaves the other SMs
                    // to the batch's other slots)
                    const int nfit = (int)std::min<int64_t>(div_up(std::max<int64_t>(cap, 1), tc::M), 2 * nsm);
                    const int nblk = sweep_blocks > 0 ? std::min(sweep_blocks, 2 * nsm) : nfit;
                    for (int i = 0; i < nt; ++i) {
                        ta.tick = i;
                        MDL_CK(launch_kxs(pdl && i > 0, (size_t)tc::SMEM_BYTES, (k_tick_tc<DIM, P>), nblk, tc::THREADS,
                                          ta, T, ph, (const uint16_t*)tcB.p, tc_unscale, (const float*)tcC.p));
                        MDL_LAUNCHED();
                        stats.tick_launches++;
                    }
                    return MDL_OK;
                }
            }
            for (int i = 0; i < nt; ++i) {
                ta.tick = i;
                if constexpr (P == 1) {
                    if (group_tick) MDL_CK(launch_k((k_tick_group<R, DIM>), gt, tick_threads, ta, ph, T));
                    else MDL_CK(launch_kx(pdl && i > 0, (k_tick<R, DIM, P>), gt, tick_threads, ta, T, ph));
                } else {
                    MDL_CK(launch_kx(pdl && i > 0, (k_tick<R, DIM, P>), gt, tick_threads, ta, T, ph));
                }
                MDL_LAUNCHED();
                stats.tick_launches++;
            }
            return MDL_OK;
        }
        {
            int ex = 0;
            const double fr = frexp(dt, &ex);
            MDL_CK(launch_k((k_epilogue<R, DIM, P>), g256, 256, arrays(o), mapped ? sets[o].mq.p : mtab.p, dt,
                            1.0 / dt, fr == 0.5 ? 1 : 0, mapped ? 1 : 0));
        }
        MDL_LAUNCHED();
        return MDL_OK;
    }

    // Arguments of the sweep ticks on state set o (the tick is set per launch).
    TickArgs<R> tick_args(int o) {
        TickArgs<R> ta{};
        ta.d = arrays(o);
        ta.dt = dt;
        ta.B = B;
        ta.tscale = ldexp(dt, -B);
        for (int b = 0; b < 8; ++b) {
            ta.dte[b] = ldexp(dt, -b);
            ta.dteR[b] = (R)ta.dte[b];
        }
        ta.stim = stim;
        return ta;
    }

    // Run phase ph_ on set o: replay its captured graph (capturing it first) unless inputs
    // are replayed this barrier, in which case launch directly.
    int run_phase(int ph_, int o, bool direct) {
        if (direct || !use_graphs) return launch_phase(ph_, o);
        cudaGraphExec_t& ge = gexec[ph_][o];
        if (!ge || gcap[ph_][o] != cap) {
            if (ge) cudaGraphExecDestroy(ge);
            ge = nullptr;
            const int64_t kl0 = stats.kernel_launches, tl0 = stats.tick_launches;
            cudaGraph_t graph;
            MDL_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            int rc = launch_phase(ph_, o);
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (rc) {
                if (ec == cudaSuccess) cudaGraphDestroy(graph);
                return rc;
            }
            MDL_CK(ec);
            ec = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            MDL_CK(ec);
            glaunch[ph_][o] = stats.kernel_launches - kl0;
            gticks[ph_][o] = stats.tick_launches - tl0;
            stats.kernel_launches = kl0;
            stats.tick_launches = tl0;
            gcap[ph_][o] = cap;
        }
        MDL_CK(cudaGraphLaunch(ge, st));
        stats.kernel_launches += glaunch[ph_][o];
        stats.tick_launches += gticks[ph_][o];
        return MDL_OK;
    }

    // One barrier step; events around the indicator and the sweep when timing.
    int run_barrier() {
        const bool direct = ovr_levels || ovr_eta_s || ovr_eta_t;
        const int o = cs;
        int rc;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
        // the spatial indicator: for the adaptation, and on a mapped mesh (which does not
        // adapt) as the barrier's diagnostic
        if ((pb.amr_enabled || mapped) && !ovr_eta_s) {
            if (timing && (e2 = next_event())) MDL_CK(cudaEventRecord(e2, st));
            if ((rc = run_phase(0, o, direct))) return rc;
            if (timing && (e3 = next_event())) MDL_CK(cudaEventRecord(e3, st));
        }
        if ((rc = run_phase(1, o, direct))) return rc;
        const int cur = pb.amr_enabled ? (o ^ 1) : o;
        if (timing && (e0 = next_event())) MDL_CK(cudaEventRecord(e0, st));
        if ((rc = run_phase(2, cur, direct))) return rc;
        if (timing && (e1 = next_event())) MDL_CK(cudaEventRecord(e1, st));
        if (!coop_sweep && (rc = run_phase(3, cur, direct))) return rc;
        if (timing) pending_ev.push_back({e0, e1, e2, e3});
        cs = cur;
        return MDL_OK;
    }

    void drop_graphs() {
        for (int p = 0; p < NPHASE; ++p)
            for (int i = 0; i < 2; ++i) {
                if (gexec[p][i]) cudaGraphExecDestroy(gexec[p][i]);
                gexec[p][i] = nullptr;
                gcap[p][i] = -1;
            }
    }

    void collect_timing() {
        for (auto& x : pending_ev) {
            float ms = 0;
            if (x.a && x.b && cudaEventElapsedTime(&ms, x.a, x.b) == cudaSuccess) stats.sweep_ms += ms;
            if (x.c && x.d && cudaEventElapsedTime(&ms, x.c, x.d) == cudaSuccess) stats.indicator_ms += ms;
        }
        pending_ev.clear();
        ev_used = 0;
        (void)cudaGetLastError();   // a failed elapsed-time query must not leak into later calls
    }

public:
    ~Ctx() override {
        if (st) cudaStreamSynchronize(st);
        drop_graphs();
        for (auto& s : sets) s.release();
        Ia.release(); ga.release(); acc.release(); eta_s.release(); lat.release(); partial.release();
        scratch.release(); fscratch.release(); cview.release(); r.release(); c0.release(); class_b.release(); lkey.release();
        bcnt.release(); psrc.release(); bsum.release(); pkind.release(); pbits.release();
        bcfl.release(); info.release(); loc.release(); nbr.release(); hang.release(); root.release();
        order.release();
        for (auto& m : smask) m.release();
        lvl_ovr.release(); eta_t_ovr.release(); meta.release(); mtab.release(); dT.release(); dph.release();
        qvol.release(); qface.release(); qkelly.release(); tcB.release(); tcC.release();
        if (hmeta) cudaFreeHost(hmeta);
        for (auto e : evpool) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
    }

    int create(const mdl_problem& p) override {
        pb = p;
        mapped = pb.geometry != MDL_GEOMETRY_BOX;
        // Q2 3D FP32: the tensor-core sweep is the default (box elements)
        tensor_tick = tensor_capable && !mapped;
        B = pb.lts_enabled ? pb.n_lts_levels - 1 : 0;
        make_tables(P, &Td);
        make_phys(pb, Td, &phd);
        convert_tables<R>(Td, &T);
        convert_phys<R>(phd, &ph);
        MappedFactors mf;
        if (mapped) {
            const int rc = mapped_factors(pb, Td, &mf, &err);
            if (rc) return rc;
        }
        if (pb.dt_barrier > 0) {
            dt = pb.dt_barrier;
        } else if (mapped) {
            // the largest 2^-k ms with dt 2^-B below every element's bound (the mesh is fixed)
            double cmin = INFINITY;
            for (double c : mf.cfl) cmin = std::min(cmin, c);
            int k = -20;
            while (ldexp(1.0, -k - B) > cmin) ++k;
            dt = ldexp(1.0, -k);
        } else {
            dt = auto_dt_barrier(Td, phd, DIM, P, pb.max_refine, B);
        }
        int dev = 0;
        MDL_CK(cudaGetDevice(&dev));
        MDL_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        MDL_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        MDL_CK(cudaMallocHost((void**)&hmeta, sizeof(DevMeta)));
        memset(hmeta, 0, sizeof(DevMeta));
        MDL_CK(meta.ensure(1));
        for (int k = 0; k < 3; ++k) {
            grid_.base[k] = (k < DIM) ? pb.base[k] : 1;
            grid_.fine[k] = (k < DIM) ? ((int64_t)pb.base[k] << pb.max_refine) : 1;
        }
        grid_.L = pb.max_refine;
        grid_.dim = DIM;
        // stimulus boxes (inclusion slack applied here, once) and time windows
        sboxes.n = pb.n_stim;
        stim.n = pb.n_stim;
        for (int s = 0; s < pb.n_stim; ++s) {
            for (int k = 0; k < 3; ++k) {
                sboxes.lo[s][k] = pb.stim[s].lo[k] - 1e-12;
                sboxes.hi[s][k] = pb.stim[s].hi[k] + 1e-12;
            }
            stim.t0[s] = pb.stim[s].t0;
            stim.t1[s] = pb.stim[s].t1;
            stim.amp[s] = pb.stim[s].amplitude;
        }
        if (P == 1) {
            sboxes.xi[0] = -1.0 / sqrt(3.0);
            sboxes.xi[1] = 1.0 / sqrt(3.0);
        } else {
            sboxes.xi[0] = -sqrt(0.6);
            sboxes.xi[1] = 0.0;
            sboxes.xi[2] = sqrt(0.6);
        }
        // b^CFL of every (level, face configuration) class
        const size_t per = (size_t)1 << (2 * NF);
        std::vector<uint8_t> hcb((size_t)(pb.max_refine + 1) * per, 0);
        if (pb.lts_enabled) {
            std::vector<double> vol, face;
            for (int l = 0; l <= pb.max_refine; ++l) {
                level_blocks(Td, phd, DIM, P, l, &vol, &face);
                for (size_t cfg = 0; cfg < per; ++cfg) {
                    bool valid = true;
                    for (int f = 0; f < NF; ++f) {
                        const unsigned kd = (cfg >> (2 * f)) & 3u;
                        if ((kd == 2 && l == 0) || (kd == 3 && l == pb.max_refine)) valid = false;
                    }
                    if (!valid) continue;
                    const double c = class_cfl_from_blocks(Td, phd, DIM, P, l, (unsigned)cfg, vol, face);
                    int b = b_from_bound(dt, c);
                    if (b < 0 || b > 15) b = 15;
                    hcb[l * per + cfg] = (uint8_t)b;
                }
            }
        }
        std::vector<double> hm(8 * NP);
        for (int l = 0; l < 8; ++l)
            for (int q = 0; q < NP; ++q) {
                double w = phd.Wvol[l];
                for (int k = 0; k < DIM; ++k) w *= Td.w[digit<N1>(q, k)];
                hm[l * NP + q] = w;
            }
        if (P == 1) {
            std::vector<double> bv, bf, bk;
            q1_blocks(Td, phd, DIM, pb.max_refine, &bv, &bf, &bk);
            std::vector<R> rv(bv.begin(), bv.end()), rf(bf.begin(), bf.end()), rk(bk.begin(), bk.end());
            MDL_CK(qvol.ensure(rv.size()));
            MDL_CK(qface.ensure(rf.size()));
            MDL_CK(qkelly.ensure(rk.size()));
            MDL_CK(cudaMemcpy(qvol.p, rv.data(), rv.size() * sizeof(R), cudaMemcpyHostToDevice));
            MDL_CK(cudaMemcpy(qface.p, rf.data(), rf.size() * sizeof(R), cudaMemcpyHostToDevice));
            MDL_CK(cudaMemcpy(qkelly.p, rk.data(), rk.size() * sizeof(R), cudaMemcpyHostToDevice));
        }
        if constexpr (tensor_capable) {
            std::vector<uint16_t> hb;
            const int t = q2_tensor_blocks(Td, phd, &hb);
            tc_unscale = (float)ldexp(1.0, -t);
            // as the image of the kernel's swizzled shared-memory operand (B_hi, then B_lo)
            std::vector<uint16_t> img((size_t)2 * tc::B_BYTES / 2, 0);
            for (int part = 0; part < 2; ++part)
                for (int n = 0; n < tc::N; ++n)
                    for (int k = 0; k < tc::K; ++k)
                        img[((size_t)part * tc::B_BYTES + tc::sw128h(n, k, tc::N)) / 2] =
                            hb[((size_t)part * tc::N + n) * tc::K + k];
            MDL_CK(tcB.ensure(img.size()));
            MDL_CK(cudaMemcpy(tcB.p, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
            std::vector<float> hc;
            q2_correction_blocks(Td, phd, &hc);
            MDL_CK(tcC.ensure(hc.size()));
            MDL_CK(cudaMemcpy(tcC.p, hc.data(), hc.size() * sizeof(float), cudaMemcpyHostToDevice));
            MDL_CK(cudaFuncSetAttribute((k_tick_tc<DIM, P>), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        tc::SMEM_BYTES));
        }
        MDL_CK(dT.ensure(1));
        MDL_CK(dph.ensure(1));
        MDL_CK(cudaMemcpy(dT.p, &T, sizeof(Tables<R>), cudaMemcpyHostToDevice));
        MDL_CK(cudaMemcpy(dph.p, &ph, sizeof(Phys<R>), cudaMemcpyHostToDevice));
        MDL_CK(mtab.ensure(hm.size()));
        MDL_CK(cudaMemcpyAsync(mtab.p, hm.data(), hm.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        MDL_CK(class_b.ensure(hcb.size()));
        MDL_CK(cudaMemcpyAsync(class_b.p, hcb.data(), hcb.size(), cudaMemcpyHostToDevice, st));
        Mesh mh;
        mh.init(DIM, pb.base, pb.max_refine);
        n_probe = mh.n() * NP;
        MDL_CK(lat.ensure(n_probe));
        MDL_CK(cudaStreamSynchronize(st));
        int rc = load_mesh(mh);
        if (rc || !mapped) return rc;
        return load_mapped(mf);
    }

    // Mapped meshes: the factors, GL masses, b^CFL and stimulus masks of every element of the
    // current mesh, computed on the device (replacing the box tables of the mesh build).
    int load_mapped(const MappedFactors& mf) {
        if (mf.ne != ne) {
            err = "mapped geometry: factor count does not match the mesh";
            return MDL_E_STATE;
        }
        margs.g = geo_args(pb);
        double wg[3];
        gl_nodes(P, margs.xg, wg);
        for (int k = 0; k < 3; ++k) margs.h0[k] = k < DIM ? pb.extent[k] / pb.base[k] : 1.0;
        margs.nstim = pb.n_stim;
        for (int s = 0; s < pb.n_stim; ++s)
            for (int k = 0; k < 3; ++k) {
                margs.slo[s][k] = pb.stim[s].lo[k] - 1e-12;
                margs.shi[s][k] = pb.stim[s].hi[k] + 1e-12;
            }
        margs.dt = dt;
        margs.B = B;
        margs.lts = pb.lts_enabled;
        Set& x = sets[cs];
        MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, nfac), 0, sizeof(unsigned int), st));
        const int nb = (int)std::min<int64_t>(div_up(std::max<int64_t>(ne, 1), 256), (int64_t)nsm * 8);
        k_mapped_keep<R, DIM, P><<<nb, 256, 0, st>>>(
            info.p, margs.nstim, x.gvol.p, x.gface.p, x.mq.p, x.fsig.p, x.fsm[0].p, x.fsm[1].p, x.fsm[2].p,
            x.fsm[3].p, bcfl.p, smask[0].p, smask[1].p, smask[2].p, smask[3].p, nullptr, nullptr, nullptr, nullptr,
            nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, ftodo.p, meta.p);
        MDL_LAUNCHED();
        k_mapped_factors<R, DIM, P><<<nsm * 8, 64, 0, st>>>(
            x.coord.p, info.p, margs, Td, x.gvol.p, x.gface.p, x.mq.p, x.fsig.p, x.fsm[0].p, x.fsm[1].p,
            x.fsm[2].p, x.fsm[3].p, bcfl.p, smask[0].p, smask[1].p, smask[2].p, smask[3].p, ftodo.p, meta.p);
        MDL_LAUNCHED();
        MDL_CK(cudaStreamSynchronize(st));
        drop_graphs();
        return MDL_OK;
    }

    int upload_mesh(int64_t n, const int32_t* rt, const int8_t* level, const int32_t* coords) override {
        if (mapped) {
            err = "upload_mesh: a mapped geometry runs on its root mesh";
            return MDL_E_STATE;
        }
        std::vector<Leaf> lv(n);
        for (int64_t i = 0; i < n; ++i) {
            lv[i].level = level[i];
            lv[i].c[0] = lv[i].c[1] = lv[i].c[2] = 0;
            for (int k = 0; k < DIM; ++k) lv[i].c[k] = coords[i * DIM + k];
            if (level[i] < 0 || level[i] > pb.max_refine) {
                err = "leaf level out of range";
                return MDL_E_ARG;
            }
        }
        Mesh m2;
        m2.init_params(DIM, pb.base, pb.max_refine);
        for (int64_t i = 0; i < n; ++i)
            if (rt && m2.root_id(lv[i]) != rt[i]) {
                err = "root id does not match coordinates";
                return MDL_E_ARG;
            }
        std::string e2;
        if (!m2.set_leaves(lv, &e2)) {
            err = "upload_mesh: " + e2;
            return MDL_E_ARG;
        }
        return load_mesh(m2);
    }

    int set_initial(const double* V, const double* s, int64_t n_dof) override {
        if (n_dof != ne * NP || !V) {
            err = "set_initial: n_dof must be n_elements * (p+1)^d";
            return MDL_E_ARG;
        }
        MDL_CK(scratch.ensure((size_t)2 * n_dof));
        MDL_CK(cudaMemcpyAsync(scratch.p, V, n_dof * 8, cudaMemcpyHostToDevice, st));
        if (s) MDL_CK(cudaMemcpyAsync(scratch.p + n_dof, s, n_dof * 8, cudaMemcpyHostToDevice, st));
        k_scatter_initial<R, NP, NPS, double><<<div_up(ne * NPS, 256), 256, 0, st>>>(
            arrays(cs), ne, scratch.p, s ? scratch.p + n_dof : nullptr);
        MDL_LAUNCHED();
        MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, err), 0, sizeof(unsigned int), st));
        k_lat_refresh<R, DIM, P><<<persistent_blocks(128), 128, 0, st>>>(arrays(cs), T, ph, (double)nbar * dt, 1, 1);
        MDL_LAUNCHED();
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int set_levels(const int8_t* b, int64_t n) override {
        if (n != ne || !b) {
            err = "set_levels: size mismatch";
            return MDL_E_ARG;
        }
        for (int64_t i = 0; i < n; ++i)
            if (b[i] < 0 || b[i] > B) {
                err = "set_levels: level outside [0, n_lts_levels)";
                return MDL_E_ARG;
            }
        MDL_CK(lvl_ovr.ensure(cap));
        MDL_CK(cudaMemcpyAsync(lvl_ovr.p, b, n, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaStreamSynchronize(st));
        ovr_levels = true;
        return MDL_OK;
    }

    int set_indicators(const double* es, const double* et, int64_t n) override {
        if (n != ne) {
            err = "set_indicators: size mismatch";
            return MDL_E_ARG;
        }
        if (es) {
            MDL_CK(cudaMemcpyAsync(eta_s.p, es, n * 8, cudaMemcpyHostToDevice, st));
            ovr_eta_s = true;
        }
        if (et) {
            MDL_CK(eta_t_ovr.ensure(cap));
            MDL_CK(cudaMemcpyAsync(eta_t_ovr.p, et, n * 8, cudaMemcpyHostToDevice, st));
            ovr_eta_t = true;
        }
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int step_barriers(int64_t n) override {
        int64_t done = 0;
        int retries = 0;
        while (done < n) {
            const int64_t start = nbar;
            // replayed indicators/levels apply to exactly one barrier: run it alone
            const bool ovr = ovr_levels || ovr_eta_s || ovr_eta_t;
            const int64_t chunk = ovr ? 1 : (n - done);
            for (int64_t i = 0; i < chunk; ++i) {
                int rc = run_barrier();
                if (rc) return rc;
            }
            int rc = sync_meta();
            if (rc) return rc;
            if (timing) {
                stats.timed_barriers += (int64_t)pending_ev.size();
                collect_timing();
            }
            done += nbar - start;
            if (nbar > start) ovr_levels = ovr_eta_s = ovr_eta_t = false;   // consumed by a completed barrier
            const unsigned e = hmeta->err;
            if (e & ERR_CAPACITY) {
                if (++retries > 8) {
                    err = "element capacity could not be grown";
                    return MDL_E_NOMEM;
                }
                rc = grow(hmeta->need);
                if (rc) return rc;
                MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, err), 0, sizeof(unsigned int), st));
                MDL_CK(cudaStreamSynchronize(st));
                hmeta->err = 0;
                continue;
            }
            if (e & ERR_NONFINITE) {
                err = "V or the state is not finite";
                return MDL_E_NONFINITE;
            }
            if (e & ERR_CFL) {
                err = "an element needs more LTS levels than n_lts_levels allows";
                MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, err), 0, sizeof(unsigned int), st));
                MDL_CK(cudaStreamSynchronize(st));
                return MDL_E_CFL;
            }
            if (e & ERR_WAIT) {
                err = "a bounded wait of the sweep gave up (tensor-core mbarrier or cooperative grid barrier)";
                return MDL_E_TIMEOUT;
            }
            if (e & ERR_MESH) {
                err = "internal: adapted mesh is not 2:1 balanced";
                return MDL_E_STATE;
            }
        }
        stats.barriers = nbar;
        return MDL_OK;
    }

    int begin_barriers(int64_t n) override {
        if (inflight) {
            err = "begin_barriers: barriers already in flight";
            return MDL_E_STATE;
        }
        inflight_start = nbar;
        // replayed inputs apply to exactly one barrier
        if (ovr_levels || ovr_eta_s || ovr_eta_t) n = std::min<int64_t>(n, 1);
        for (int64_t i = 0; i < n; ++i) {
            int rc = run_barrier();
            if (rc) return rc;
        }
        inflight = n;
        return MDL_OK;
    }

    int end_barriers(int64_t* completed) override {
        if (completed) *completed = 0;
        int rc = sync_meta();
        if (rc) return rc;
        inflight = 0;
        if (timing) {
            stats.timed_barriers += (int64_t)pending_ev.size();
            collect_timing();
        }
        const int64_t done = nbar - inflight_start;
        if (completed) *completed = done;
        if (done > 0) ovr_levels = ovr_eta_s = ovr_eta_t = false;
        stats.barriers = nbar;
        const unsigned e = hmeta->err;
        if (e & ERR_CAPACITY) {
            rc = grow(hmeta->need);
            if (rc) return rc;
            MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, err), 0, sizeof(unsigned int), st));
            MDL_CK(cudaStreamSynchronize(st));
            hmeta->err = 0;
            return MDL_OK;   // the barriers after the overflow were skipped; the caller relaunches
        }
        if (e & ERR_NONFINITE) {
            err = "V or the state is not finite";
            return MDL_E_NONFINITE;
        }
        if (e & ERR_CFL) {
            err = "an element needs more LTS levels than n_lts_levels allows";
            MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, err), 0, sizeof(unsigned int), st));
            MDL_CK(cudaStreamSynchronize(st));
            return MDL_E_CFL;
        }
        if (e & ERR_WAIT) {
            err = "a bounded wait of the sweep gave up (tensor-core mbarrier or cooperative grid barrier)";
            return MDL_E_TIMEOUT;
        }
        if (e & ERR_MESH) {
            err = "internal: adapted mesh is not 2:1 balanced";
            return MDL_E_STATE;
        }
        return MDL_OK;
    }

    int set_tick_shape(int threads, int blocks_per_sm) override {
        if ((threads != 64 && threads != 128 && threads != 256) || blocks_per_sm < 1 || blocks_per_sm > 32 ||
            threads * blocks_per_sm > 2048) {
            err = "set_tick_shape: threads in {64,128,256}, threads * blocks_per_sm <= 2048";
            return MDL_E_ARG;
        }
        if (threads != tick_threads || blocks_per_sm != tick_bpsm) {
            tick_threads = threads;
            tick_bpsm = blocks_per_sm;
            drop_graphs();
        }
        return MDL_OK;
    }

    int set_sweep_variant(int variant) override {
        if (variant < MDL_SWEEP_THREAD || variant > MDL_SWEEP_TENSOR) {
            err = "set_sweep_variant: variant in {0, 1, 2, 3}";
            return MDL_E_ARG;
        }
        if (mapped && variant != MDL_SWEEP_THREAD) {
            err = "set_sweep_variant: a mapped geometry has the thread-per-element sweep only";
            return MDL_E_ARG;
        }
        if (variant == MDL_SWEEP_TENSOR && !tensor_capable) {
            err = "set_sweep_variant: the tensor-core sweep needs a Q2 3D FP32 context";
            return MDL_E_ARG;
        }
        const bool co = variant == MDL_SWEEP_COOP, gr = variant == MDL_SWEEP_GROUP, tn = variant == MDL_SWEEP_TENSOR;
        if (co != coop_sweep || gr != group_tick || tn != tensor_tick) {
            coop_sweep = co;
            group_tick = gr;
            tensor_tick = tn;
            drop_graphs();
        }
        return MDL_OK;
    }

    int set_sweep_blocks(int max_blocks) override {
        if (max_blocks < 0) {
            err = "set_sweep_blocks: max_blocks must be >= 0";
            return MDL_E_ARG;
        }
        if (max_blocks != sweep_blocks) {
            sweep_blocks = max_blocks;
            drop_graphs();
        }
        return MDL_OK;
    }

    int fused_begin(void* slot_record, int* Bout) override {
        const bool direct = ovr_levels || ovr_eta_s || ovr_eta_t;
        if (inflight && direct) {
            err = "fused_begin: replayed inputs apply to one barrier per completion";
            return MDL_E_STATE;
        }
        if (!inflight) inflight_start = nbar;
        fused_own = false;
        const int o = cs;
        int rc;
        if ((pb.amr_enabled || mapped) && !ovr_eta_s && (rc = run_phase(0, o, direct))) return rc;
        if ((rc = run_phase(1, o, direct))) return rc;
        fused_cur = pb.amr_enabled ? (o ^ 1) : o;
        FusedSlot<R>* fs = static_cast<FusedSlot<R>*>(slot_record);
        fs->ta = tick_args(fused_cur);
        fs->T = dT.p;
        fs->ph = dph.p;
        fs->cls = DIM == 2 ? (P == 1 ? FC_2_1 : FC_2_2) : (P == 1 ? FC_3_1 : FC_3_2);
        fs->shift = 0;
        if (Bout) *Bout = B;
        return MDL_OK;
    }

    int fused_own_sweep() override {
        const bool direct = ovr_levels || ovr_eta_s || ovr_eta_t;
        int rc = run_phase(2, fused_cur, direct);
        if (rc) return rc;
        fused_own = true;
        return MDL_OK;
    }

    int fused_finish() override {
        const bool direct = ovr_levels || ovr_eta_s || ovr_eta_t;
        // the cooperative sweep runs the epilogue itself
        if (!(fused_own && coop_sweep)) {
            int rc = run_phase(3, fused_cur, direct);
            if (rc) return rc;
        }
        cs = fused_cur;
        inflight += 1;
        return MDL_OK;
    }

    bool replaying() const override { return ovr_levels || ovr_eta_s || ovr_eta_t; }
    bool is_mapped() const override { return mapped; }

    void* stream_handle() const override { return (void*)st; }
    int precision() const override { return sizeof(R) == 8 ? 64 : 32; }

    int64_t device_bytes() const override {
        int64_t b = 0;
        auto add = [&](size_t n, size_t sz) { b += (int64_t)(n * sz); };
        for (const auto& x : sets) {
            add(x.V0.cap + x.V1.cap + x.v.cap, sizeof(R));
            add(x.eta_t.cap, 8); add(x.lvl.cap, 1); add(x.coord.cap, sizeof(int4));
        }
        add(Ia.cap + ga.cap, sizeof(R));
        add(acc.cap + eta_s.cap + lat.cap + partial.cap + scratch.cap + eta_t_ovr.cap + mtab.cap, 8);
        add(fscratch.cap, 4);
        add(cview.cap, sizeof(R));
        for (const auto& x : sets) {
            add(x.gvol.cap + x.gface.cap, sizeof(R));
            add(x.mq.cap, 8);
            add(x.fsig.cap, 4);
            for (const auto& m : x.fsm) add(m.cap, 4);
        }
        add(r.cap + c0.cap + class_b.cap + bcfl.cap + pkind.cap + pbits.cap + lvl_ovr.cap, 1);
        add(bcnt.cap + psrc.cap + ftodo.cap + nbr.cap + hang.cap + root.cap + order.cap + info.cap + loc.cap, 4);
        add(lkey.cap, 8);
        for (const auto& m : smask) add(m.cap, 4);
        add(bsum.cap, 8);
        return b;
    }

    double dt_barrier() const override { return dt; }

    int step_to(double t_end) override {
        const double nn = floor((t_end - (double)nbar * dt) / dt + 1e-9);
        if (nn <= 0) return MDL_OK;
        return step_barriers((int64_t)nn);
    }

    int get_time(double* t, int64_t* tick, double* d) const override {
        if (t) *t = (double)nbar * dt;
        if (tick) *tick = nbar;
        if (d) *d = dt;
        return MDL_OK;
    }

    int get_sizes(int64_t* n_e, int64_t* ndof, int64_t* np) const override {
        if (n_e) *n_e = ne;
        if (ndof) *ndof = ne * NP;
        if (np) *np = n_probe;
        return MDL_OK;
    }

    int read_field(int which, double* out, int64_t cap_, int64_t* n) override {
        const int64_t nd = ne * NP;
        if (n) *n = nd;
        if (cap_ < nd || !out) {
            err = "read: capacity too small";
            return MDL_E_ARG;
        }
        MDL_CK(scratch.ensure(2 * nd));
        k_gather<R, NP, NPS, double><<<div_up(nd, 256), 256, 0, st>>>(arrays(cs), ne, which, scratch.p);
        MDL_LAUNCHED();
        MDL_CK(cudaMemcpyAsync(out, scratch.p, nd * 8, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    // The device address of a page-locked host buffer mapped into the device's address space
    // (cudaHostAlloc / pinned memory), or null for any other pointer (which is then staged
    // through a device copy).
    static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }   // null counts as aligned
    static const void* mapped_host(const void* p) {
        if (!p) return nullptr;
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
    }

    int set_initial_f32(const float* V, const float* s, int64_t n_dof) override {
        if (n_dof != ne * NP || !V) {
            err = "set_initial_f32: n_dof must be n_elements * (p+1)^d";
            return MDL_E_ARG;
        }
        // page-locked host buffers are read by the layout kernel itself over the host link;
        // others go through one device copy first
        const float* dV = static_cast<const float*>(mapped_host(V));
        const float* dS = s ? static_cast<const float*>(mapped_host(s)) : nullptr;
        if (!dV || (s && !dS)) {
            MDL_CK(fscratch.ensure((size_t)2 * n_dof));
            MDL_CK(cudaMemcpyAsync(fscratch.p, V, n_dof * sizeof(float), cudaMemcpyHostToDevice, st));
            if (s) MDL_CK(cudaMemcpyAsync(fscratch.p + n_dof, s, n_dof * sizeof(float), cudaMemcpyHostToDevice, st));
            dV = fscratch.p;
            dS = s ? fscratch.p + n_dof : nullptr;
        }
        if (dV != fscratch.p && aligned16(dV) && aligned16(dS)) {
            const int64_t nt = std::max<int64_t>(div_up(n_dof, 4), ne);
            k_scatter_initial_x4<R, NP, NPS><<<div_up(nt, 256), 256, 0, st>>>(arrays(cs), ne, dV, dS);
        } else {
            k_scatter_initial<R, NP, NPS, float><<<div_up(ne * NPS, 256), 256, 0, st>>>(arrays(cs), ne, dV, dS);
        }
        MDL_LAUNCHED();
        MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, err), 0, sizeof(unsigned int), st));
        k_lat_refresh<R, DIM, P><<<persistent_blocks(128), 128, 0, st>>>(arrays(cs), T, ph, (double)nbar * dt, 1, 1);
        MDL_LAUNCHED();
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int read_fields_f32(float* V, float* s, int64_t cap_, int64_t* n) override {
        const int64_t nd = ne * NP;
        if (n) *n = nd;
        if (cap_ < nd || (!V && !s)) {
            err = "read_fields_f32: capacity too small";
            return MDL_E_ARG;
        }
        // page-locked host buffers are written by the layout kernel itself; others through a
        // device copy
        float* dV = V ? static_cast<float*>(const_cast<void*>(mapped_host(V))) : nullptr;
        float* dS = s ? static_cast<float*>(const_cast<void*>(mapped_host(s))) : nullptr;
        if ((V && !dV) || (s && !dS)) {
            MDL_CK(fscratch.ensure((size_t)2 * nd));
            k_gather_f32<R, NP, NPS><<<div_up(nd, 256), 256, 0, st>>>(arrays(cs), ne, fscratch.p, fscratch.p + nd);
            MDL_LAUNCHED();
            if (V) MDL_CK(cudaMemcpyAsync(V, fscratch.p, nd * sizeof(float), cudaMemcpyDeviceToHost, st));
            if (s) MDL_CK(cudaMemcpyAsync(s, fscratch.p + nd, nd * sizeof(float), cudaMemcpyDeviceToHost, st));
        } else if (aligned16(dV) && aligned16(dS)) {
            k_gather_f32x4<R, NP, NPS><<<div_up(div_up(nd, 4), 256), 256, 0, st>>>(arrays(cs), ne, dV, dS);
            MDL_LAUNCHED();
        } else {
            k_gather_f32<R, NP, NPS><<<div_up(nd, 256), 256, 0, st>>>(arrays(cs), ne, dV, dS);
            MDL_LAUNCHED();
        }
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int read_activation(double* out, int64_t cap_, int64_t* n) override {
        if (n) *n = n_probe;
        if (cap_ < n_probe || !out) {
            err = "read_activation: capacity too small";
            return MDL_E_ARG;
        }
        MDL_CK(cudaMemcpyAsync(out, lat.p, n_probe * 8, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int read_mesh(int32_t* rt, int8_t* level, int32_t* coords, int8_t* b, int64_t cap_, int64_t* n) override {
        if (n) *n = ne;
        if (cap_ < ne) {
            err = "read_mesh: capacity too small";
            return MDL_E_ARG;
        }
        std::vector<int4> hc(ne);
        std::vector<int32_t> hr(ne);
        std::vector<uint8_t> hl(ne);
        MDL_CK(cudaMemcpyAsync(hc.data(), sets[cs].coord.p, ne * sizeof(int4), cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaMemcpyAsync(hr.data(), root.p, ne * 4, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaMemcpyAsync(hl.data(), sets[cs].lvl.p, ne, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        for (int64_t i = 0; i < ne; ++i) {
            if (rt) rt[i] = hr[i];
            if (level) level[i] = (int8_t)hc[i].w;
            if (coords) {
                const int c[3] = {hc[i].x, hc[i].y, hc[i].z};
                for (int k = 0; k < DIM; ++k) coords[i * DIM + k] = c[k];
            }
            if (b) b[i] = (int8_t)(hl[i] & 7);
        }
        return MDL_OK;
    }

    int read_faces(int8_t* kind, int32_t* nb, int8_t* pos, int64_t cap_, int64_t* n) override {
        if (n) *n = ne;
        if (cap_ < ne) {
            err = "read_faces: capacity too small";
            return MDL_E_ARG;
        }
        std::vector<uint32_t> hi(ne);
        std::vector<int32_t> hn((size_t)ne * NF), hh((size_t)ne * NF * NSUB);
        MDL_CK(cudaMemcpyAsync(hi.data(), info.p, ne * 4, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaMemcpyAsync(hn.data(), nbr.p, (size_t)ne * NF * 4, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaMemcpyAsync(hh.data(), hang.p, (size_t)ne * NF * NSUB * 4, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        for (int64_t e = 0; e < ne; ++e)
            for (int f = 0; f < NF; ++f) {
                const int64_t i = e * NF + f;
                const int kd = (hi[e] >> (4 * f)) & 3;
                const int ps = (hi[e] >> (4 * f + 2)) & 3;
                if (kind) kind[i] = (int8_t)kd;
                if (pos) pos[i] = (kd == F_COARSER) ? (int8_t)ps : 0;
                if (nb) {
                    for (int j = 0; j < NSUB; ++j) nb[i * NSUB + j] = -1;
                    if (kd == F_SAME || kd == F_COARSER) nb[i * NSUB] = hn[i];
                    else if (kd == F_FINER)
                        for (int j = 0; j < NSUB; ++j) nb[i * NSUB + j] = hh[hn[i] + j];
                }
            }
        return MDL_OK;
    }

    int read_indicators(double* es, double* et, int64_t cap_, int64_t* n) override {
        if (n) *n = ne;
        if (cap_ < ne) {
            err = "read_indicators: capacity too small";
            return MDL_E_ARG;
        }
        if (es) MDL_CK(cudaMemcpyAsync(es, eta_s.p, ne * 8, cudaMemcpyDeviceToHost, st));
        if (et) MDL_CK(cudaMemcpyAsync(et, sets[cs].eta_t.p, ne * 8, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int get_stats(mdl_stats* s) const override {
        *s = stats;
        return MDL_OK;
    }
    int reset_stats() override {
        MDL_CK(cudaMemsetAsync((char*)meta.p + offsetof(DevMeta, elem_updates), 0, 3 * sizeof(int64_t), st));
        MDL_CK(cudaStreamSynchronize(st));
        stats = mdl_stats{};
        stats.n_elements = ne;
        stats.barriers = nbar;
        return MDL_OK;
    }
    int set_timing(int on) override {
        timing = on != 0;
        return MDL_OK;
    }
    int device_view(int which, void** p, int64_t* n, void** stream) override {
        if (stream) *stream = (void*)st;
        switch (which) {
            case 0: {
                // normalise: current values into slot 0 with the parities reset
                std::vector<double> tmp(ne * NP);
                int64_t nn;
                int rc = read_field(0, tmp.data(), ne * NP, &nn);
                if (rc) return rc;
                MDL_CK(scratch.ensure(2 * ne * NP));
                MDL_CK(cudaMemcpyAsync(scratch.p, tmp.data(), ne * NP * 8, cudaMemcpyHostToDevice, st));
                k_scatter_initial<R, NP, NPS, double><<<div_up(ne * NPS, 256), 256, 0, st>>>(
                    arrays(cs), ne, scratch.p, (const double*)nullptr);
                MDL_LAUNCHED();
                if (NPS != NP) {
                    // padded rows: hand out a compact copy ((p+1)^d values per element)
                    MDL_CK(cview.ensure((size_t)ne * NP));
                    k_gather<R, NP, NPS, R><<<div_up(ne * NP, 256), 256, 0, st>>>(arrays(cs), ne, 0, cview.p);
                    MDL_LAUNCHED();
                }
                MDL_CK(cudaStreamSynchronize(st));
                if (p) *p = NPS != NP ? (void*)cview.p : (void*)sets[cs].V0.p;
                if (n) *n = ne * NP;
                return MDL_OK;
            }
            case 1: {
                if (NPS != NP) {
                    MDL_CK(cview.ensure((size_t)ne * NP));
                    k_gather<R, NP, NPS, R><<<div_up(ne * NP, 256), 256, 0, st>>>(arrays(cs), ne, 1, cview.p);
                    MDL_LAUNCHED();
                    MDL_CK(cudaStreamSynchronize(st));
                }
                if (p) *p = NPS != NP ? (void*)cview.p : (void*)sets[cs].v.p;
                if (n) *n = ne * NP;
                return MDL_OK;
            }
            case 2: if (p) *p = lat.p; if (n) *n = n_probe; return MDL_OK;
            case 3: if (p) *p = sets[cs].eta_t.p; if (n) *n = ne; return MDL_OK;
            default: err = "device_view: unknown array"; return MDL_E_ARG;
        }
    }
};

}  // namespace mdl
