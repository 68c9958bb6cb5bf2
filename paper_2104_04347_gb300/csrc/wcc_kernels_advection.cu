// FP64 half-step kernels, the stage bound and the dispatcher of the advection system.
#define WCC_SYSTEM ::wcc::ADVECTION
#define WCC_KERNELS_PART 0
#include "wcc_kernels.inc"
