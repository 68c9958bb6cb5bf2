// Batched kernels for the advection system.
#define WCC_SYSTEM ::wcc::ADVECTION
#define WCC_BATCH_PART 0
#include "wcc_batch_kernels.inc"
