// The FP32 hot kernels (k_track, k_step_ext for MS_F32) again, with exp2 and
// log2 evaluated as polynomials on the FMA pipe instead of the SFU
// (ms_device.cuh, fma_ex2 / fma_lg2; MS_FLAG_FMA_TRANSCENDENTALS).  The
// paper moves its transcendentals to the FMA units (Sec. 3.3); this variant
// measures that choice on GB300, where the SFU and the instruction issue
// share the bound.  It exports launch_track_fma and launch_step_ext_fma.
#define MS_FMA_TRANSCENDENTALS 1
#include "ms_kernels.cu"
