// Batched kernels for the advection system.
#define WCC_SYSTEM ::wcc::ADVECTION
#include "wcc_batch_kernels.inc"
