// Batched two-half-step kernels of the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#define WCC_BATCH_PART 1
#include "wcc_batch_kernels.inc"
