// FP32-variant kernels of the euler system at P = 5, 6.
#define WCC_SYSTEM ::wcc::EULER
#define WCC_KERNELS_PART 3
#include "wcc_kernels.inc"
