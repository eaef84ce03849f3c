// Library-internal context and dispatch declarations (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "sd.h"

#define SD_MAX_N 9

#define SDI_MAX_SLABS 16   // slabs of the pipelined host-buffer residual

struct sd_ctx {
    // problem
    int dim;
    int ne[3];
    int nelem;
    int p, n;
    int nvar;
    int ngrad;               // gradient components exchanged per face (1 scalar, 9 NS)
    sd_scheme scheme;
    sd_physics phys;
    sd_precision prec;
    cudaStream_t stream;
    int device;
    double lo[3], hi[3], h[3];
    double J;                // prod_d h_d / 2
    // 1D operators (host, FP64), built by the library itself
    double xs[SD_MAX_N], ws[SD_MAX_N], xf[SD_MAX_N + 1];
    double L[(SD_MAX_N + 1) * SD_MAX_N];     // L[f*n + i]
    double M[SD_MAX_N * (SD_MAX_N + 1)];     // M[i*(n+1) + f]
    double D[SD_MAX_N * SD_MAX_N];           // D = M L
    double LD[(SD_MAX_N + 1) * SD_MAX_N];    // LD[f*n + i] = (L D)[f][i]: derivative of the interpolant at flux point f
    double LM0[SD_MAX_N + 1], LMN[SD_MAX_N + 1];   // (L M)[f][0], (L M)[f][n]: weights of the face corrections
    double alpha, beta;
    // sizes
    size_t npts;             // points per variable = nelem * n^dim
    size_t nstate;           // nvar * npts
    size_t ntu, ntg, nfh;    // trace and interface-flux buffer sizes (values)
    size_t esize;            // bytes per value of the residual precision
    // scratch owned by the context
    void* Tu;                // face traces of u        [nelem][2dim][F] ([nvar][n^(dim-1)] padded to F, a multiple of 4)
    void* Tg;                // face gradient values    [nelem][2dim][G] ([ngrad][n^(dim-1)] padded to G)
    void* Fh;                // interface fluxes        [dim][nelem][F] (+d face of each element)
    double* Tu64;            // FP64 traces for diagnostics (== Tu when prec is F64)
    void* S;                 // stage input of the residual precision
    void* K;                 // stage residual of the residual precision
    // Runge-Kutta registers, in the residual precision: FP64 contexts keep full stage
    // states, FP32 contexts keep stage increments (the state itself accumulates in FP64)
    void *rA, *rB, *rC;
    void* rX;                // FP32 contexts: the step's start state minus the offsets
    // FP32 contexts in SD_RK_STAGES_F64 mode: FP64 stage registers (allocated on first use)
    sd_rk_stages rk_stages;
    double *rA64, *rB64, *rC64;
    double* dW;              // Gauss weights (device, n values)
    double* partial;         // diagnostics block partials
    double* partial2;        // second-level partials (DIAG_L1 x NDIAG)
    double* dsum;            // diagnostics totals (device)
    int diag_blocks;
    void* hU;                // device staging of the host-buffer residual path
    void* hR;
    // host-buffer path in slabs (3D): copy streams and per-slab events, created with the
    // context; null when the path is not used
    cudaStream_t s_h2d, s_d2h;
    cudaEvent_t ev_in[SDI_MAX_SLABS], ev_out[SDI_MAX_SLABS], ev_start;
    // extra per-element flux added by the residual ([nelem][15] FP32, tau[e][3 v + d]),
    // caller-owned or the closure's own buffer; NULL: none
    const float* tau;
    // learned closure attached with sd_closure_enable (buffers owned by the context)
    int closure_on;
    double* cl_tmode;        // Legendre modal transform T[m][i] and the points xi (features)
    float* cl_X;             // features [nelem][64]
    void* cl_Xb;             // standardised BF16 input [nelem][64]
    float* cl_Y;             // network output [nelem][15]
    void* cl_H;              // activation cache [2][nelem][128] BF16
    float* cl_tau;           // closure flux [nelem][15]
    const void* cl_Wb;       // caller-owned network: BF16 weights, FP32 parameters,
    const float* cl_P;       //   input and output standardisation
    const float *cl_mux, *cl_sgx, *cl_mut, *cl_sgt;
    // curvilinear grids (periodic trilinear hexahedra), set up by sd_init_curvilinear
    int curv;
    void* cgeo;              // map coefficients c1..c7 [nelem][24] in the residual precision
    double* cgeo64;          // the same in FP64 (diagnostics; == cgeo when prec is F64)
    void* cih;               // interior-penalty 1/h of the -d face of each element [nelem][3]
    void* cvs;               // v^S [nelem][nvar][3][n^3]
    void* cTg;               // own interface gradients [nelem][6][nvar][3][n^2]
    double curv_volume;      // volume of the periodic domain (sum of the element volumes)
    // owned box of a sub-domain context (sd_set_owned_box): the diagnostics sum over it only
    int own_set;
    int own_lo[3], own_hi[3];
    int diag_nb;             // rows of `partial` written by the last diagnostics launch
    // profiling and launch accounting
    long long launches;
    int prof_on;
    int prof_n[SD_K_COUNT];                   // recorded event pairs per kernel class
    cudaEvent_t* prof_ev[SD_K_COUNT];         // 2 * SDI_PROF_CAP events per class
    double prof_ms[SD_K_COUNT];
    long long prof_count[SD_K_COUNT];
};

#define SDI_PROF_CAP 512

// bracket one kernel launch of class k (no-op unless profiling is enabled)
void sdi_prof_begin(sd_ctx* c, int k);
void sdi_prof_end(sd_ctx* c, int k);

// dispatch entry points (one translation unit per residual precision)
// offset_in != 0: U already has the reference offsets removed (Runge-Kutta stage copies)
sd_status sdi_residual_f32(sd_ctx* c, const float* U, float* R, int offset_in);
sd_status sdi_residual_f64(sd_ctx* c, const double* U, double* R, int offset_in);
// one phase of the residual over elements [e_begin, e_end) on `stream` (host pipeline)
enum { SDI_PH_TRACE = 0, SDI_PH_GRAD = 1, SDI_PH_FACE = 2, SDI_PH_FLUX = 3 };
sd_status sdi_residual_phase_f32(sd_ctx* c, const float* U, float* R, int phase, int e_begin, int e_end,
                                 cudaStream_t stream);
sd_status sdi_residual_phase_f64(sd_ctx* c, const double* U, double* R, int phase, int e_begin, int e_end,
                                 cudaStream_t stream);
// curvilinear grids: set-up from the corner nodes, residual, diagnostics partial sums
sd_status sdi_curv_setup(sd_ctx* c, const double* nodes);
sd_status sdi_curv_residual_f32(sd_ctx* c, const float* U, float* R, int offset_in);
sd_status sdi_curv_residual_f64(sd_ctx* c, const double* U, double* R, int offset_in);
sd_status sdi_curv_diag_partials(sd_ctx* c, const double* U64);
sd_status sdi_upload_f32(const sd_ctx* c);
sd_status sdi_upload_f64(const sd_ctx* c);
// closure data of a state: features X [nelem][64] and/or flux means [nelem][15] (either NULL)
sd_status sdi_closure_data_f32(sd_ctx* c, const float* U, float* X, double* means);
sd_status sdi_closure_data_f64(sd_ctx* c, const double* U, float* X, double* means);
// closure network on the context's feature buffer -> c->cl_tau
sd_status sdi_closure_network(sd_ctx* c);
sd_status sdi_diag(sd_ctx* c, const double* U64, double* host_out);
sd_status sdi_check_smem(sd_ctx* c);
void sdi_set_error(const char* fmt, ...);
void sdi_build_operators(sd_ctx* c);
// validate a problem and fill the problem fields, operators and scratch sizes of c
// (no CUDA call, no allocation; c is overwritten)
sd_status sdi_setup(const sd_mesh* mesh, int p, sd_scheme scheme, const sd_physics* phys, sd_precision prec,
                    void* stream, sd_ctx* c);

// size of the static scratch of sd_residual_f32_noalloc (FP32 values, 36 MiB)
#define SD_NOALLOC_SCRATCH_FLOATS (9 * 1024 * 1024)
