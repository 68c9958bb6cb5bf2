// Two-half-step kernels of the euler system.
#define WCC_SYSTEM ::wcc::EULER
#define WCC_KERNELS_PART 2
#include "wcc_kernels.inc"
