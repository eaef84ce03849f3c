// FP32 residual instantiations (every n in 2..9, 1D/3D scalar and 3D Navier-Stokes).
#include "sd_launch.cuh"

sd_status sdi_residual_f32(sd_ctx* c, const float* U, float* R) {
    return sdk::residual_dispatch<float>(c, U, R);
}
