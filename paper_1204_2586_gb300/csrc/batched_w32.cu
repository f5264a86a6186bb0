// batched_w32.cu -- the multi-RHS PCG for blocks of 32 columns.
#include "batched_impl.cuh"

PK_BATCHED_WIDTH(32)
