// Batched chain kernels for clusters of one CTA, with block barriers in the
// body; the code is in chain_batch.cuh.
#define FILARK_BATCH_SOLO 1
#include "chain_batch.cuh"
