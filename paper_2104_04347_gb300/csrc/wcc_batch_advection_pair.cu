// Batched two-half-step kernels of the advection system.
#define WCC_SYSTEM ::wcc::ADVECTION
#define WCC_BATCH_PART 1
#include "wcc_batch_kernels.inc"
