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

// The SSPRK(5,4) stage of an FP32 context with the stage update fused into the flux kernel:
// gradient, interface-flux and flux phases of the stage input U (offsets removed; its traces
// already in c->Tu), the flux kernel applying stage `so->k` (sdk::StageOut)
sd_status sdi_fused_stage_f32(sd_ctx* c, const float* U, const void* so) {
    const sdk::StageOut* st = static_cast<const sdk::StageOut*>(so);
    sd_status s;
    if (c->closure_on && c->nvar == 5 && (s = sdk::closure_dispatch<float>(c, U, 1)) != SD_OK) return s;
    for (int ph : {SDI_PH_GRAD, SDI_PH_FACE})
        if ((s = sdk::phase_dispatch<float>(c, U, nullptr, 1, ph, 0, c->nelem, c->stream)) != SD_OK) return s;
    return sdk::phase_dispatch<float>(c, U, nullptr, 1, SDI_PH_FLUX, 0, c->nelem, c->stream, st);
}

// traces of a stage input (offsets removed) into c->Tu
sd_status sdi_stage_traces_f32(sd_ctx* c, const float* U) {
    return sdk::phase_dispatch<float>(c, U, nullptr, 1, SDI_PH_TRACE, 0, c->nelem, c->stream);
}

sd_status sdi_upload_f32(const sd_ctx* c) { return sdk::upload_dispatch<float>(c); }

sd_status sdi_closure_data_f32(sd_ctx* c, const float* U, float* X, double* means) {
    return sdk::closure_data_dispatch<float>(c, U, X, means, 0);
}
