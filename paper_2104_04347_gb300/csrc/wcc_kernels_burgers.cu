// Kernels for the burgers system.
#define WCC_SYSTEM ::wcc::BURGERS
#include "wcc_kernels.inc"
