// mdl_ctx_impl.cuh -- context implementation for one (precision R, dim, order).
//
// Per barrier step (Alg. 1):
//   1. [AMR] eta^s on the device (k_eta_s), refine/coarsen mark counts (k_marks);
//      only if a change is possible, eta^s goes to the host, the forest adapts,
//      the new mesh tables go up and k_transfer remaps V, v and eta^t.
//   2. levels b_e on the device (k_levels) from the class CFL level b^CFL and eta^t;
//      the host re-sorts the element order only when some b_e changed.
//   3. 2^B ticks of k_tick over the due prefix of the order.
//   4. k_epilogue + k_reduce_partials: eta^t, parities, non-finite flag, int V.
// The host crosses to the device at most twice per barrier (status reads) plus
// the mesh upload when the forest changed.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <unordered_map>
#include <vector>

#include "mdl_ctx.h"
#include "mdl_kernels.cuh"
#include "mdl_mesh.h"
#include "mdl_tables.h"

namespace mdl {

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t n) {
        if (n <= cap && p) return cudaSuccess;
        release();
        const size_t c = n + n / 4 + 64;
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

__global__ void k_fill_inf(double* p, int64_t n);

template <typename R, int DIM, int P>
class Ctx : public CtxBase {
    using S = Shape<DIM, P>;
    static constexpr int N1 = S::N1, NP = S::NP, NF = S::NF, NSUB = S::NSUB;

    struct StateSet {
        DBuf<R> V0, V1, v;
        DBuf<double> eta_t;
        DBuf<uint8_t> lvl;
        void release() {
            V0.release(); V1.release(); v.release(); eta_t.release(); lvl.release();
        }
    };

    mdl_problem pb{};
    Mesh mesh;
    Tables<double> Td{};
    Phys<double> phd{};
    Tables<R> T{};
    Phys<R> ph{};
    double dt = 0;
    int B = 0;
    int64_t nbar = 0;
    int64_t n_probe = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    StateSet sets[2];
    int cs = 0;
    DBuf<R> Ia, ga;
    DBuf<double> acc, eta_s, lat, partial, scratch;
    DBuf<uint32_t> info, loc;
    DBuf<int32_t> nbr, hang, order, root;
    DBuf<uint8_t> bcfl;
    DBuf<uint32_t> smask[MDL_MAX_STIM];
    DBuf<int8_t> lvl_ovr, pkind, pbits;
    DBuf<int32_t> psrc;
    DBuf<double> eta_t_ovr;
    DBuf<DevStatus> status;
    DevStatus* hst = nullptr;
    std::vector<int32_t> h_order;
    std::vector<uint8_t> h_lvl;
    unsigned int cnt[8] = {0};
    bool need_order = true;
    bool ovr_levels = false, ovr_eta_s = false, ovr_eta_t = false;
    bool timing = false;
    std::unordered_map<uint32_t, int> bcache;
    mdl_stats stats{};

    // ------------------------------------------------------------------
    DevArrays<R> arrays(int set) {
        DevArrays<R> d{};
        StateSet& s = sets[set];
        d.V0 = s.V0.p; d.V1 = s.V1.p; d.v = s.v.p; d.eta_t = s.eta_t.p; d.lvl = s.lvl.p;
        d.Ia = Ia.p; d.ga = ga.p; d.acc = acc.p; d.eta_s = eta_s.p; d.lat = lat.p;
        d.partial = partial.p; d.bcfl = bcfl.p; d.info = info.p; d.nbr = nbr.p; d.hang = hang.p;
        d.order = order.p; d.root = root.p; d.loc = loc.p;
        for (int s2 = 0; s2 < MDL_MAX_STIM; ++s2) d.smask[s2] = smask[s2].p;
        d.status = status.p;
        d.ne = mesh.n();
        return d;
    }

    static int grid(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

    int class_b(int level, unsigned cls) {
        if (!pb.lts_enabled) return 0;
        const uint32_t key = ((uint32_t)level << 16) | cls;
        auto it = bcache.find(key);
        if (it != bcache.end()) return it->second;
        const double c = class_cfl(Td, phd, DIM, P, level, cls);
        int b = b_from_bound(dt, c);
        if (b < 0 || b > 15) b = 15;
        bcache[key] = b;
        return b;
    }

    // Upload the mesh tables of `mesh` (info, neighbours, classes, probes, stimulus masks).
    int upload_tables() {
        const int64_t ne = mesh.n();
        std::vector<uint32_t> h_info(ne), h_loc(ne);
        std::vector<int32_t> h_root(ne);
        std::vector<uint8_t> h_b(ne);
        std::vector<std::vector<uint32_t>> h_sm(pb.n_stim, std::vector<uint32_t>(ne, 0));
        double xi[3];
        for (int a = 0; a < N1; ++a) xi[a] = 0;
        {
            // GL nodes from the tables' weights are not stored; recompute closed form
            if (P == 1) { xi[0] = -1.0 / sqrt(3.0); xi[1] = -xi[0]; }
            else { xi[0] = -sqrt(0.6); xi[1] = 0.0; xi[2] = sqrt(0.6); }
        }
        for (int64_t e = 0; e < ne; ++e) {
            const Leaf& lf = mesh.leaves[e];
            uint32_t inf = 0;
            for (int f = 0; f < NF; ++f) {
                const uint32_t kd = (uint32_t)mesh.kind[e * NF + f] & 3u;
                const uint32_t ps = (uint32_t)mesh.pos[e * NF + f] & 3u;
                inf |= (kd | (ps << 2)) << (4 * f);
            }
            inf |= (uint32_t)lf.level << 24;
            bool stim = false;
            for (int s = 0; s < pb.n_stim; ++s) {
                uint32_t m = 0;
                for (int q = 0; q < NP; ++q) {
                    bool in = true;
                    for (int k = 0; k < DIM; ++k) {
                        const double h = phd.h[lf.level][k];
                        const double x = lf.c[k] * h + (xi[digit<N1>(q, k)] + 1.0) * 0.5 * h;
                        if (x < pb.stim[s].lo[k] - 1e-12 || x > pb.stim[s].hi[k] + 1e-12) in = false;
                    }
                    if (in) m |= 1u << q;
                }
                h_sm[s][e] = m;
                if (m) stim = true;
            }
            if (stim) inf |= INFO_STIM;
            h_info[e] = inf;
            const int64_t rid = mesh.root_id(lf);
            h_root[e] = (int32_t)rid;
            uint32_t lc = (uint32_t)lf.level << 24;
            for (int k = 0; k < DIM; ++k) {
                const int32_t r = lf.c[k] >> lf.level;
                lc |= (uint32_t)(lf.c[k] - (r << lf.level)) << (8 * k);
            }
            h_loc[e] = lc;
            h_b[e] = (uint8_t)class_b(lf.level, mesh.cls[e]);
        }
        MDL_CK(info.ensure(ne));
        MDL_CK(loc.ensure(ne));
        MDL_CK(root.ensure(ne));
        MDL_CK(bcfl.ensure(ne));
        MDL_CK(order.ensure(ne));
        MDL_CK(nbr.ensure((size_t)ne * NF));
        MDL_CK(hang.ensure(mesh.hang.size() + 1));
        MDL_CK(cudaMemcpyAsync(info.p, h_info.data(), ne * 4, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaMemcpyAsync(loc.p, h_loc.data(), ne * 4, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaMemcpyAsync(root.p, h_root.data(), ne * 4, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaMemcpyAsync(bcfl.p, h_b.data(), ne, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaMemcpyAsync(nbr.p, mesh.nbr.data(), (size_t)ne * NF * 4, cudaMemcpyHostToDevice, st));
        if (!mesh.hang.empty())
            MDL_CK(cudaMemcpyAsync(hang.p, mesh.hang.data(), mesh.hang.size() * 4, cudaMemcpyHostToDevice, st));
        for (int s = 0; s < pb.n_stim; ++s) {
            MDL_CK(smask[s].ensure(ne));
            MDL_CK(cudaMemcpyAsync(smask[s].p, h_sm[s].data(), ne * 4, cudaMemcpyHostToDevice, st));
        }
        MDL_CK(Ia.ensure((size_t)ne * NP));
        MDL_CK(ga.ensure((size_t)ne * NP));
        MDL_CK(acc.ensure(ne));
        MDL_CK(eta_s.ensure(ne));
        MDL_CK(partial.ensure(grid(ne, 256) + 1));
        // host copies must stay alive until the async copies ran
        MDL_CK(cudaStreamSynchronize(st));
        need_order = true;
        return MDL_OK;
    }

    int ensure_set(int s, int64_t ne) {
        StateSet& S_ = sets[s];
        MDL_CK(S_.V0.ensure((size_t)ne * NP));
        MDL_CK(S_.V1.ensure((size_t)ne * NP));
        MDL_CK(S_.v.ensure((size_t)ne * NP));
        MDL_CK(S_.eta_t.ensure(ne));
        MDL_CK(S_.lvl.ensure(ne));
        return MDL_OK;
    }

    int reset_state() {
        const int64_t ne = mesh.n();
        int rc = ensure_set(cs, ne);
        if (rc) return rc;
        StateSet& S_ = sets[cs];
        MDL_CK(cudaMemsetAsync(S_.V0.p, 0, (size_t)ne * NP * sizeof(R), st));
        MDL_CK(cudaMemsetAsync(S_.V1.p, 0, (size_t)ne * NP * sizeof(R), st));
        MDL_CK(cudaMemsetAsync(S_.v.p, 0, (size_t)ne * NP * sizeof(R), st));
        MDL_CK(cudaMemsetAsync(S_.eta_t.p, 0, ne * sizeof(double), st));
        MDL_CK(cudaMemsetAsync(S_.lvl.p, 0, ne, st));
        MDL_CK(cudaMemsetAsync(eta_s.p, 0, ne * sizeof(double), st));
        MDL_CK(cudaMemsetAsync(status.p, 0, sizeof(DevStatus), st));
        k_fill_inf<<<grid(n_probe, 256), 256, 0, st>>>(lat.p, n_probe);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        k_lat_refresh<R, DIM, P><<<grid(ne, 128), 128, 0, st>>>(arrays(cs), T, ph, time_now(), 0);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    double time_now() const { return (double)nbar * dt; }
    double tick_time(int i) const {
        const double nt = (double)(1 << B);
        return ((double)nbar * nt + (double)i) * dt / nt;
    }

    int read_status() {
        MDL_CK(cudaMemcpyAsync(hst, status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }
    int zero_counters() {
        MDL_CK(cudaMemsetAsync(status.p, 0, offsetof(DevStatus, nonfinite), st));
        MDL_CK(cudaMemsetAsync((char*)status.p + offsetof(DevStatus, n_refine), 0, 2 * sizeof(unsigned int), st));
        return MDL_OK;
    }

    // ------------------------------------------------------------------
    int amr_step() {
        const int64_t ne = mesh.n();
        if (!ovr_eta_s) {
            if (timing) MDL_CK(cudaEventRecord(ev[2], st));
            k_eta_s<R, DIM, P><<<grid(ne, 128), 128, 0, st>>>(arrays(cs), T, ph);
            stats.kernel_launches++;
            MDL_CK(cudaGetLastError());
            if (timing) MDL_CK(cudaEventRecord(ev[3], st));
        }
        ovr_eta_s = false;
        int rc = zero_counters();
        if (rc) return rc;
        k_marks<R, DIM><<<grid(ne, 256), 256, 0, st>>>(arrays(cs), pb.tau_refine, pb.tau_coarsen, pb.max_refine);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        rc = read_status();
        if (rc) return rc;
        if (timing) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ev[2], ev[3]) == cudaSuccess) stats.indicator_ms += ms;
        }
        const bool possible = hst->n_refine > 0 || hst->n_coarsen > 0;
        if (!possible) return MDL_OK;
        auto t0 = std::chrono::steady_clock::now();
        std::vector<double> h_eta(ne);
        MDL_CK(cudaMemcpyAsync(h_eta.data(), eta_s.p, ne * sizeof(double), cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        Mesh next;
        std::vector<int8_t> pk, pbits_h;
        std::vector<int32_t> ps;
        std::string e2;
        const bool changed = adapt(mesh, h_eta.data(), pb.tau_refine, pb.tau_coarsen, &next, &pk, &ps,
                                   &pbits_h, &e2);
        if (!e2.empty()) {
            err = "adapt: " + e2;
            return MDL_E_STATE;
        }
        auto t1 = std::chrono::steady_clock::now();
        stats.amr_host_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
        if (!changed) return MDL_OK;
        // transfer into the other state set
        const int ns = cs ^ 1;
        const int64_t nn = next.n();
        rc = ensure_set(ns, nn);
        if (rc) return rc;
        MDL_CK(pkind.ensure(nn));
        MDL_CK(pbits.ensure(nn));
        MDL_CK(psrc.ensure(nn));
        MDL_CK(cudaMemcpyAsync(pkind.p, pk.data(), nn, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaMemcpyAsync(pbits.p, pbits_h.data(), nn, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaMemcpyAsync(psrc.p, ps.data(), nn * 4, cudaMemcpyHostToDevice, st));
        DevArrays<R> od = arrays(cs);
        std::swap(mesh, next);
        rc = upload_tables();
        if (rc) return rc;
        DevArrays<R> nd = arrays(ns);
        k_transfer<R, DIM, P><<<grid(nn, 128), 128, 0, st>>>(od, nd, pkind.p, psrc.p, pbits.p, T);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        cs = ns;
        k_lat_refresh<R, DIM, P><<<grid(nn, 128), 128, 0, st>>>(arrays(cs), T, ph, time_now(), 0);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        MDL_CK(cudaStreamSynchronize(st));
        auto t2 = std::chrono::steady_clock::now();
        stats.transfer_ms += std::chrono::duration<double, std::milli>(t2 - t1).count();
        stats.amr_rebuilds++;
        return MDL_OK;
    }

    int build_order() {
        const int64_t ne = mesh.n();
        h_lvl.resize(ne);
        MDL_CK(cudaMemcpyAsync(h_lvl.data(), sets[cs].lvl.p, ne, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        int64_t off[9] = {0};
        for (int b = B; b >= 0; --b) off[B - b + 1] = off[B - b] + cnt[b];
        h_order.resize(ne);
        int64_t pos[8];
        for (int b = 0; b <= B; ++b) pos[b] = off[B - b];
        for (int64_t e = 0; e < ne; ++e) h_order[pos[h_lvl[e] & 7]++] = (int32_t)e;
        MDL_CK(cudaMemcpyAsync(order.p, h_order.data(), ne * 4, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaStreamSynchronize(st));
        need_order = false;
        return MDL_OK;
    }

    int barrier() {
        int rc;
        if (pb.amr_enabled) {
            rc = amr_step();
            if (rc) return rc;
        }
        const int64_t ne = mesh.n();
        rc = zero_counters();
        if (rc) return rc;
        const double tau_cell = pb.tau_cell;
        int bcell = 0;
        if (pb.dt_bar_cell > 0) {
            bcell = b_from_bound(dt, pb.dt_bar_cell);
            if (bcell < 0) bcell = 15;
        }
        const double* et = ovr_eta_t ? eta_t_ovr.p : sets[cs].eta_t.p;
        k_levels<R><<<grid(ne, 256), 256, 0, st>>>(arrays(cs), ovr_levels ? lvl_ovr.p : nullptr, et, tau_cell,
                                                    bcell, B, pb.lts_enabled);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        const bool was_ovr = ovr_levels;
        ovr_levels = false;
        ovr_eta_t = false;
        rc = read_status();
        if (rc) return rc;
        if (hst->nonfinite) {
            err = "V or the state is not finite";
            return MDL_E_NONFINITE;
        }
        if (hst->cfl_err) {
            err = was_ovr ? "replayed level out of range" : "an element needs more LTS levels than allowed";
            need_order = true;
            return MDL_E_CFL;
        }
        for (int b = 0; b < 8; ++b) cnt[b] = hst->cnt[b];
        if (hst->changed || need_order) {
            rc = build_order();
            if (rc) return rc;
        }
        const int nt = 1 << B;
        TickArgs<R> ta{};
        ta.d = arrays(cs);
        ta.dt = dt;
        ta.B = B;
        ta.stim.n = pb.n_stim;
        for (int s = 0; s < pb.n_stim; ++s) {
            ta.stim.t0[s] = pb.stim[s].t0;
            ta.stim.t1[s] = pb.stim[s].t1;
            ta.stim.amp[s] = pb.stim[s].amplitude;
        }
        if (timing) MDL_CK(cudaEventRecord(ev[0], st));
        int64_t elem_upd = 0;
        for (int i = 0; i < nt; ++i) {
            int64_t na = 0;
            if (i == 0) na = ne;
            else {
                int tz = 0;
                while (((i >> tz) & 1) == 0) ++tz;
                for (int b = B - tz; b <= B; ++b) na += cnt[b];
            }
            if (na == 0) continue;
            ta.tick = i;
            ta.n_act = (int)na;
            ta.t_i = tick_time(i);
            k_tick<R, DIM, P><<<grid(na, 128), 128, 0, st>>>(ta, T, ph);
            stats.kernel_launches++;
            MDL_CK(cudaGetLastError());
            elem_upd += na;
            stats.tick_launches++;
        }
        if (timing) MDL_CK(cudaEventRecord(ev[1], st));
        const int nb = grid(ne, 256);
        k_epilogue<R, DIM, P><<<nb, 256, 0, st>>>(arrays(cs), T, ph, dt);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        k_reduce_partials<<<1, 256, 0, st>>>(partial.p, nb, &status.p->integral);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        if (timing) {
            MDL_CK(cudaEventSynchronize(ev[1]));
            float ms = 0;
            MDL_CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            stats.sweep_ms += ms;
        }
        nbar++;
        stats.barriers++;
        stats.element_updates += elem_upd;
        stats.dof_updates += elem_upd * NP;
        for (int b = 0; b < 8; ++b) stats.level_counts[b] = cnt[b];
        stats.n_elements = ne;
        return MDL_OK;
    }

public:
    ~Ctx() override {
        if (st) cudaStreamSynchronize(st);
        for (auto& s : sets) s.release();
        Ia.release(); ga.release(); acc.release(); eta_s.release(); lat.release(); partial.release();
        scratch.release(); info.release(); loc.release(); nbr.release(); hang.release(); order.release();
        root.release(); bcfl.release(); lvl_ovr.release(); pkind.release(); pbits.release(); psrc.release();
        eta_t_ovr.release(); status.release();
        for (auto& m : smask) m.release();
        if (hst) cudaFreeHost(hst);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
    }

    int create(const mdl_problem& p) override {
        pb = p;
        B = pb.lts_enabled ? pb.n_lts_levels - 1 : 0;
        make_tables(P, &Td);
        make_phys(pb, Td, &phd);
        convert_tables<R>(Td, &T);
        convert_phys<R>(phd, &ph);
        dt = pb.dt_barrier > 0 ? pb.dt_barrier : auto_dt_barrier(Td, phd, DIM, P, pb.max_refine, B);
        MDL_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        for (auto& e : ev) MDL_CK(cudaEventCreate(&e));
        MDL_CK(cudaMallocHost((void**)&hst, sizeof(DevStatus)));
        MDL_CK(status.ensure(1));
        MDL_CK(cudaMemsetAsync(status.p, 0, sizeof(DevStatus), st));
        mesh.init(DIM, pb.base, pb.max_refine);
        n_probe = (int64_t)mesh.n() * NP;
        MDL_CK(lat.ensure(n_probe));
        int rc = upload_tables();
        if (rc) return rc;
        return reset_state();
    }

    int upload_mesh(int64_t n, const int32_t* rt, const int8_t* level, const int32_t* coords) override {
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
        std::swap(mesh, m2);
        int rc = upload_tables();
        if (rc) return rc;
        return reset_state();
    }

    int set_initial(const double* V, const double* s, int64_t n_dof) override {
        const int64_t ne = mesh.n();
        if (n_dof != ne * NP || !V) {
            err = "set_initial: n_dof must be n_elements * (p+1)^d";
            return MDL_E_ARG;
        }
        MDL_CK(scratch.ensure((size_t)2 * n_dof));
        MDL_CK(cudaMemcpyAsync(scratch.p, V, n_dof * 8, cudaMemcpyHostToDevice, st));
        if (s) MDL_CK(cudaMemcpyAsync(scratch.p + n_dof, s, n_dof * 8, cudaMemcpyHostToDevice, st));
        k_scatter_initial<R, NP><<<grid(n_dof, 256), 256, 0, st>>>(arrays(cs), scratch.p, s ? scratch.p + n_dof : nullptr);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        MDL_CK(cudaMemsetAsync((char*)status.p + offsetof(DevStatus, nonfinite), 0, sizeof(unsigned int), st));
        k_lat_refresh<R, DIM, P><<<grid(ne, 128), 128, 0, st>>>(arrays(cs), T, ph, time_now(), 1);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int set_levels(const int8_t* b, int64_t n) override {
        if (n != mesh.n() || !b) {
            err = "set_levels: size mismatch";
            return MDL_E_ARG;
        }
        for (int64_t i = 0; i < n; ++i)
            if (b[i] < 0 || b[i] > B) {
                err = "set_levels: level outside [0, n_lts_levels)";
                return MDL_E_ARG;
            }
        MDL_CK(lvl_ovr.ensure(n));
        MDL_CK(cudaMemcpyAsync(lvl_ovr.p, b, n, cudaMemcpyHostToDevice, st));
        MDL_CK(cudaStreamSynchronize(st));
        ovr_levels = true;
        return MDL_OK;
    }

    int set_indicators(const double* es, const double* et, int64_t n) override {
        if (n != mesh.n()) {
            err = "set_indicators: size mismatch";
            return MDL_E_ARG;
        }
        if (es) {
            MDL_CK(cudaMemcpyAsync(eta_s.p, es, n * 8, cudaMemcpyHostToDevice, st));
            ovr_eta_s = true;
        }
        if (et) {
            MDL_CK(eta_t_ovr.ensure(n));
            MDL_CK(cudaMemcpyAsync(eta_t_ovr.p, et, n * 8, cudaMemcpyHostToDevice, st));
            ovr_eta_t = true;
        }
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int step_barriers(int64_t n) override {
        for (int64_t i = 0; i < n; ++i) {
            int rc = barrier();
            if (rc) return rc;
        }
        int rc = read_status();
        if (rc) return rc;
        stats.integral_V = hst->integral;
        if (hst->nonfinite) {
            err = "V or the state is not finite";
            return MDL_E_NONFINITE;
        }
        return MDL_OK;
    }

    int step_to(double t_end) override {
        const double nn = floor((t_end - time_now()) / dt + 1e-9);
        if (nn <= 0) return MDL_OK;
        return step_barriers((int64_t)nn);
    }

    int get_time(double* t, int64_t* tick, double* d) const override {
        if (t) *t = time_now();
        if (tick) *tick = nbar;
        if (d) *d = dt;
        return MDL_OK;
    }

    int get_sizes(int64_t* ne, int64_t* ndof, int64_t* np) const override {
        if (ne) *ne = mesh.n();
        if (ndof) *ndof = mesh.n() * NP;
        if (np) *np = n_probe;
        return MDL_OK;
    }

    int read_field(int which, double* out, int64_t cap, int64_t* n) override {
        const int64_t nd = mesh.n() * NP;
        if (n) *n = nd;
        if (cap < nd || !out) {
            err = "read: capacity too small";
            return MDL_E_ARG;
        }
        MDL_CK(scratch.ensure(2 * nd));
        k_gather<R, NP><<<grid(nd, 256), 256, 0, st>>>(arrays(cs), which, scratch.p);
        stats.kernel_launches++;
        MDL_CK(cudaGetLastError());
        MDL_CK(cudaMemcpyAsync(out, scratch.p, nd * 8, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int read_activation(double* out, int64_t cap, int64_t* n) override {
        if (n) *n = n_probe;
        if (cap < n_probe || !out) {
            err = "read_activation: capacity too small";
            return MDL_E_ARG;
        }
        MDL_CK(cudaMemcpyAsync(out, lat.p, n_probe * 8, cudaMemcpyDeviceToHost, st));
        MDL_CK(cudaStreamSynchronize(st));
        return MDL_OK;
    }

    int read_mesh(int32_t* rt, int8_t* level, int32_t* coords, int8_t* b, int64_t cap, int64_t* n) override {
        const int64_t ne = mesh.n();
        if (n) *n = ne;
        if (cap < ne) {
            err = "read_mesh: capacity too small";
            return MDL_E_ARG;
        }
        for (int64_t i = 0; i < ne; ++i) {
            const Leaf& lf = mesh.leaves[i];
            if (rt) rt[i] = (int32_t)mesh.root_id(lf);
            if (level) level[i] = (int8_t)lf.level;
            if (coords)
                for (int k = 0; k < DIM; ++k) coords[i * DIM + k] = lf.c[k];
        }
        if (b) {
            h_lvl.resize(ne);
            MDL_CK(cudaMemcpyAsync(h_lvl.data(), sets[cs].lvl.p, ne, cudaMemcpyDeviceToHost, st));
            MDL_CK(cudaStreamSynchronize(st));
            for (int64_t i = 0; i < ne; ++i) b[i] = (int8_t)(h_lvl[i] & 7);
        }
        return MDL_OK;
    }

    int read_faces(int8_t* kind, int32_t* nb, int8_t* pos, int64_t cap, int64_t* n) override {
        const int64_t ne = mesh.n();
        if (n) *n = ne;
        if (cap < ne) {
            err = "read_faces: capacity too small";
            return MDL_E_ARG;
        }
        for (int64_t e = 0; e < ne; ++e)
            for (int f = 0; f < NF; ++f) {
                const int64_t i = e * NF + f;
                const int kd = mesh.kind[i];
                if (kind) kind[i] = (int8_t)kd;
                if (pos) pos[i] = (kd == F_COARSER) ? mesh.pos[i] : 0;
                if (nb) {
                    for (int j = 0; j < NSUB; ++j) nb[i * NSUB + j] = -1;
                    if (kd == F_SAME || kd == F_COARSER) nb[i * NSUB] = mesh.nbr[i];
                    else if (kd == F_FINER)
                        for (int j = 0; j < NSUB; ++j) nb[i * NSUB + j] = mesh.hang[mesh.nbr[i] + j];
                }
            }
        return MDL_OK;
    }

    int read_indicators(double* es, double* et, int64_t cap, int64_t* n) override {
        const int64_t ne = mesh.n();
        if (n) *n = ne;
        if (cap < ne) {
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
        stats = mdl_stats{};
        return MDL_OK;
    }
    int set_timing(int on) override {
        timing = on != 0;
        return MDL_OK;
    }
    int device_view(int which, void** p, int64_t* n, void** stream) override {
        const int64_t ne = mesh.n();
        if (stream) *stream = (void*)st;
        switch (which) {
            case 0: {
                // normalise: current values into slot 0
                std::vector<double> tmp(ne * NP);
                int64_t nn;
                int rc = read_field(0, tmp.data(), ne * NP, &nn);
                if (rc) return rc;
                if (p) *p = sets[cs].V0.p;
                // write back as slot 0 with parity reset
                MDL_CK(scratch.ensure(2 * ne * NP));
                MDL_CK(cudaMemcpyAsync(scratch.p, tmp.data(), ne * NP * 8, cudaMemcpyHostToDevice, st));
                k_scatter_initial<R, NP><<<grid(ne * NP, 256), 256, 0, st>>>(arrays(cs), scratch.p, nullptr);
                stats.kernel_launches++;
                MDL_CK(cudaGetLastError());
                MDL_CK(cudaStreamSynchronize(st));
                if (n) *n = ne * NP;
                return MDL_OK;
            }
            case 1: if (p) *p = sets[cs].v.p; if (n) *n = ne * NP; return MDL_OK;
            case 2: if (p) *p = lat.p; if (n) *n = n_probe; return MDL_OK;
            case 3: if (p) *p = sets[cs].eta_t.p; if (n) *n = ne; return MDL_OK;
            default: err = "device_view: unknown array"; return MDL_E_ARG;
        }
    }
};

}  // namespace mdl
