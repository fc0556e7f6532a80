// mdl_fused.h -- one fused sweep over the due elements of many resident simulations.
//
// A batch round advances every running slot by one barrier step (Alg. 1).  Each slot runs
// its own indicator, adaptation, level and ordering phases and its own epilogue on its own
// stream; the sweep between them is fused: for every global tick g = 0 .. 2^Bmax - 1 one
// persistent kernel launch per element class (2D/3D, Q1/Q2) and precision covers the due
// elements of every slot of that class whose tick grid contains g
// (a slot with B LTS levels above level 0 takes its tick g 2^(B - Bmax) when 2^(Bmax - B)
// divides g), walking work items of `tile` consecutive due elements of one slot.  Each
// element takes the same element step as the slot's own thread-per-element sweep.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mdl_fused_api.h"
#include "mdl_kernels.cuh"

namespace mdl {

// Element classes of the fused sweep (dim, order).
enum FusedClass : int32_t { FC_2_1 = 0, FC_2_2 = 1, FC_3_1 = 2, FC_3_2 = 3 };

// One slot of a fused round, in device memory (filled on the host by the slot's context).
template <typename R>
struct FusedSlot {
    TickArgs<R> ta;           // the state set the sweep updates, time step, LTS levels, stimuli
    const Tables<R>* T;       // device copies of the slot's basis tables and physics
    const Phys<R>* ph;
    int32_t cls;              // FusedClass
    int32_t shift;            // Bmax - B: the slot takes part in global ticks divisible by 2^shift
};

}  // namespace mdl
