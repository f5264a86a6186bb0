// batched_w64.cu -- the multi-RHS PCG for blocks of 64 columns.
#include "batched_impl.cuh"

PK_BATCHED_WIDTH(64)
