// FP32-variant half-step kernels and the FP32 stage set-up of the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#define WCC_KERNELS_PART 1
#include "wcc_kernels.inc"
