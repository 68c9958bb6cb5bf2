// Two-half-step kernels of the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#define WCC_KERNELS_PART 2
#include "wcc_kernels.inc"
