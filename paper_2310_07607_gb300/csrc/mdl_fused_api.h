// mdl_fused_api.h -- host-side interface of the fused multi-simulation sweep (mdl_fused.h
// has the device-side records and the kernel).  Slot records are opaque byte blocks here.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace mdl {

constexpr int FUSED_MAX_SLOTS = 256;

// Launch shape of the fused sweep: threads per block, due elements per work item, blocks.
struct FusedShape {
    int threads;
    int tile;
    int blocks;
};

// Bytes of one slot record of the given precision (32 or 64).
size_t fused_slot_bytes(int precision);
// Write the record's shift (Bmax - B: the slot takes part in global ticks divisible by 2^shift).
void fused_set_shift(void* record, int precision, int shift);
// Element family of an order: 1 (Q1, 2D and 3D) or 2 (Q2).  One fused kernel serves each
// family: one kernel for all four element classes would take the register budget of the Q2
// element step (255 registers, spilling) for the Q1 elements too.
int fused_family(int order);
// Resident blocks per SM of the family's fused kernel at `threads` per block (occupancy API).
int fused_blocks_per_sm(int precision, int family, int threads);
// Launch the 2^Bmax global ticks of one fused round of a family on `st` (d_slots: nslot
// records of that family in device memory).  Returns a CUDA error code; each slot's own
// errors stay in its device bookkeeping.
cudaError_t fused_sweep(int precision, int family, const void* d_slots, int nslot, int Bmax, FusedShape shape,
                        cudaStream_t st);

}  // namespace mdl
