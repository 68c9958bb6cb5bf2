// Batched kernels for the euler system.
#define WCC_SYSTEM ::wcc::EULER
#define WCC_BATCH_PART 0
#include "wcc_batch_kernels.inc"
