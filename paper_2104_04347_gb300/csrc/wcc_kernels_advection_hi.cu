// FP32-variant kernels of the advection system at P = 5, 6.
#define WCC_SYSTEM ::wcc::ADVECTION
#define WCC_KERNELS_PART 3
#include "wcc_kernels.inc"
