// Batched chain kernels for clusters of 2, 4 or 8 CTAs (and of 1 with cluster
// barriers); the code is in chain_batch.cuh.
#define FILARK_BATCH_SOLO 0
#include "chain_batch.cuh"
