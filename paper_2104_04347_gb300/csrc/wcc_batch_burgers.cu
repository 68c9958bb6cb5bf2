// Batched kernels for the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#define WCC_BATCH_PART 0
#include "wcc_batch_kernels.inc"
