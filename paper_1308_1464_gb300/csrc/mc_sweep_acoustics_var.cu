// mc_sweep_acoustics_var.cu -- fused wave-propagation step instantiated for
// variable-coefficient acoustics (FP32 and FP64).
#include "mc_sweep_impl.cuh"

MC_DEFINE_SOLVER_LAUNCHERS(acoustics_var, mc::AcousticsVarRP)
