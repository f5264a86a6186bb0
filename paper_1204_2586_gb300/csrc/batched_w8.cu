// batched_w8.cu -- the multi-RHS PCG for blocks of 8 columns.
#include "batched_impl.cuh"

PK_BATCHED_WIDTH(8)
