// FP64 half-step kernels, the stage bound and the dispatcher of the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#define WCC_KERNELS_PART 0
#include "wcc_kernels.inc"
