// Batched kernels for the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#include "wcc_batch_kernels.inc"
