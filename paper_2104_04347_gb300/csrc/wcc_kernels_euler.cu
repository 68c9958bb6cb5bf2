// Kernels for the euler system.
#define WCC_SYSTEM ::wcc::EULER
#include "wcc_kernels.inc"
