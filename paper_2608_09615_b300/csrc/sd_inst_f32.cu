// FP32 residual instantiations (every n in 2..9, 1D/3D scalar and 3D Navier-Stokes) and
// the upload of this translation unit's constant operator tables.
#include "sd_launch.cuh"

sd_status sdi_residual_f32(sd_ctx* c, const float* U, float* R, int offset_in) {
    return sdk::residual_dispatch<float>(c, U, R, offset_in);
}

sd_status sdi_residual_phase_f32(sd_ctx* c, const float* U, float* R, int phase, int e_begin, int e_end,
                                 cudaStream_t stream) {
    return sdk::phase_dispatch<float>(c, U, R, 0, phase, e_begin, e_end, stream);
}

sd_status sdi_upload_f32(const sd_ctx* c) { return sdk::upload_dispatch<float>(c); }

sd_status sdi_closure_data_f32(sd_ctx* c, const float* U, float* X, double* means) {
    return sdk::closure_data_dispatch<float>(c, U, X, means, 0);
}
