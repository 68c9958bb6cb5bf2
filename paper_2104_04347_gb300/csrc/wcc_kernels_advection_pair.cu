// Two-half-step kernels of the advection system.
#define WCC_SYSTEM ::wcc::ADVECTION
#define WCC_KERNELS_PART 2
#include "wcc_kernels.inc"
