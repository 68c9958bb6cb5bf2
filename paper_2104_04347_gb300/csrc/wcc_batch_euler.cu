// Batched kernels for the euler system.
#define WCC_SYSTEM ::wcc::EULER
#include "wcc_batch_kernels.inc"
