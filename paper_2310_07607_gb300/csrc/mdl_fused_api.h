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
// Element class of a (dimension, order): 0 (2D Q1), 1 (2D Q2), 2 (3D Q1), 3 (3D Q2).  One
// fused kernel serves each class, so each compiles with its own element step's register
// budget (the 3D Q2 step takes 255 registers; the 2D Q1 step about half of that).
int fused_class(int dim, int order);
// Resident blocks per SM of the class's fused kernel at `threads` per block (occupancy API).
int fused_blocks_per_sm(int precision, int cls, int threads);
// Launch the 2^Bmax global ticks of one fused round of a class on `st` (d_slots: nslot
// records of that class in device memory).  Returns a CUDA error code; each slot's own
// errors stay in its device bookkeeping.
cudaError_t fused_sweep(int precision, int cls, const void* d_slots, int nslot, int Bmax, FusedShape shape,
                        cudaStream_t st);

}  // namespace mdl
