// mc_sweep_acoustics.cu -- fused wave-propagation step instantiated for the
// acoustics Riemann solver (FP32 and FP64).
#include "mc_sweep_impl.cuh"

MC_DEFINE_SOLVER_LAUNCHERS(acoustics, mc::AcousticsRP)
