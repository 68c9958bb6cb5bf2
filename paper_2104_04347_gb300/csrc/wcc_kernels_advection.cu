// Kernels for the advection system.
#define WCC_SYSTEM ::wcc::ADVECTION
#include "wcc_kernels.inc"
