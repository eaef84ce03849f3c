// FP64 residual instantiations (every n in 2..9, 1D/3D scalar and 3D Navier-Stokes).
#include "sd_launch.cuh"

sd_status sdi_residual_f64(sd_ctx* c, const double* U, double* R) {
    return sdk::residual_dispatch<double>(c, U, R);
}
