// batched_w16.cu -- the multi-RHS PCG for blocks of 16 columns.
#include "batched_impl.cuh"

PK_BATCHED_WIDTH(16)
