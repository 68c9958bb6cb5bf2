// FP32-variant kernels of the burgers system at P = 5, 6.
#define WCC_SYSTEM ::wcc::BURGERS
#define WCC_KERNELS_PART 3
#include "wcc_kernels.inc"
