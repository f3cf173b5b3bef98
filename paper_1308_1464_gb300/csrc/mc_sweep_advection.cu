// mc_sweep_advection.cu -- fused wave-propagation step instantiated for the
// constant-velocity advection solver (FP32 and FP64).
#include "mc_sweep_impl.cuh"

MC_DEFINE_SOLVER_LAUNCHERS(advection, mc::AdvectionRP)
