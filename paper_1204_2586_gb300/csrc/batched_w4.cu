// batched_w4.cu -- the multi-RHS PCG for blocks of 4 columns.
#include "batched_impl.cuh"

PK_BATCHED_WIDTH(4)
