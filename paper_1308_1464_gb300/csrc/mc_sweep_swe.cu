// mc_sweep_swe.cu -- fused wave-propagation step instantiated for the
// swe Riemann solver (FP32 and FP64).
#include "mc_sweep_impl.cuh"

MC_DEFINE_SOLVER_LAUNCHERS(swe, mc::SweRP)
