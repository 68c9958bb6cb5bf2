// Batched two-half-step kernels of the euler system.
#define WCC_SYSTEM ::wcc::EULER
#define WCC_BATCH_PART 1
#include "wcc_batch_kernels.inc"
