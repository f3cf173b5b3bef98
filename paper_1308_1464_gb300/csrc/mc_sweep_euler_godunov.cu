// mc_sweep_euler_godunov.cu -- fused wave-propagation step instantiated for
// the Euler equations with the exact-solution (Godunov) normal solve (FP32
// and FP64).
#include "mc_sweep_impl.cuh"

MC_DEFINE_SOLVER_LAUNCHERS(euler_godunov, mc::EulerGodunovRP)
