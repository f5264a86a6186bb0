// batched_w48.cu -- the multi-RHS PCG for blocks of 48 columns.
#include "batched_impl.cuh"

PK_BATCHED_WIDTH(48)
