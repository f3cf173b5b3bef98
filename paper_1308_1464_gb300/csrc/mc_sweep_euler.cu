// mc_sweep_euler.cu -- fused wave-propagation step instantiated for the
// euler Riemann solver (FP32 and FP64).
#include "mc_sweep_impl.cuh"

MC_DEFINE_SOLVER_LAUNCHERS(euler, mc::EulerRP)
