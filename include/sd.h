/*
 * sd.h -- C ABI of the B300 Spectral Difference (SD) residual library.
 *
 * The library evaluates the SD semi-discrete residual dU/dt of Lodato & Tonicello,
 * "A novel compact scheme for second-order fluxes applied to the Spectral Difference
 * method", on periodic, uniform, tensor-product Cartesian grids (1D segments or 3D
 * hexahedra), with the viscous terms built from the auxiliary gradient v = grad u either
 * by the standard BR1 scheme (Sec. 2.1) or by the compact one-sided scheme (Secs. 2.2,
 * 2.3). Physics: linear diffusion (Sec. 3 / 4.1), the porous medium equation (Sec. 4.3,
 * Eq. pme) and the compressible Navier-Stokes equations (Sec. 4.4).
 *
 * Data layout (every state / residual array, device or host):
 *     U[var][E_{dim-1}]...[E_0][n]...[n]
 * variable-major, then the element grid with x fastest, then the n^dim solution points
 * of each element with the x point index fastest; n = p + 1. In 3D this is
 * U[var][ez][ey][ex][k][j][i]. The points are the n Gauss-Legendre points of each
 * element (Sec. 2). NS variables: rho, rho u, rho v, rho w, rho E. Scalar: u.
 *
 * Ownership: the caller owns every state/residual buffer it passes. The context owns
 * all scratch (face-trace buffers, Runge-Kutta registers, staging buffers), allocated in
 * sd_init and freed in sd_destroy; afterwards only the calls that say so allocate
 * (sd_closure_enable, sd_set_rk_stages), each once.
 * Errors: every call returns an sd_status; nothing throws across the ABI. On error the
 * outputs are unspecified and sd_last_error() describes the failure (thread-local).
 * Streams: all device work is enqueued on the context's stream (sd_init / sd_set_stream).
 * Calls returning SD_OK have only enqueued work unless stated otherwise.
 */
#ifndef SD_H
#define SD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SD_OK = 0,
    SD_EINVAL = 1,          /* bad argument (null pointer, size, enum, aliasing)      */
    SD_ENOMEM = 2,          /* device or host allocation failed (allocating calls)    */
    SD_ECUDA = 3,           /* a CUDA runtime call failed                             */
    SD_EUNSUPPORTED = 4,    /* valid but not supported here (p, dim, shared memory)   */
    SD_ENONFINITE = 5,      /* sd_diagnostics found a NaN/Inf in the state            */
    SD_ETIMEOUT = 6         /* reserved: a bounded device-side wait gave up           */
} sd_status;

typedef enum { SD_BR1 = 0, SD_COMPACT = 1 } sd_scheme;            /* Secs. 2.1 / 2.2-2.3 */
typedef enum { SD_HEAT = 0, SD_PME = 1, SD_NS = 2 } sd_physics_kind;
typedef enum { SD_ROE = 0, SD_RUSANOV = 1 } sd_riemann;           /* NS inviscid flux    */
typedef enum { SD_F64 = 0, SD_F32 = 1 } sd_precision;            /* residual arithmetic */
typedef enum { SD_RK4 = 0, SD_SSPRK54 = 1, SD_LSRK54 = 2 } sd_rk;

/* Periodic uniform Cartesian grid: dim in {1, 3}; ne[d] elements along direction d
 * (x first; unused entries ignored); the domain is prod_d [lo[d], hi[d]). */
typedef struct {
    int dim;
    int ne[3];
    double lo[3];
    double hi[3];
} sd_mesh;

/* Physics parameters.
 *  SD_HEAT: du/dt = nu lap u                                  (uses nu)
 *  SD_PME : du/dt = div(m |u|^(m-1) grad u), the factor taken from the solution at the
 *           flux points (Sec. 4.3)                            (uses m_pme)
 *  SD_NS  : Sec. 4.4. mu0 = rho0 u0 L / Re, p0 = rho0 (u0/Ma)^2 / gamma,
 *           e0 = p0/((gamma-1) rho0); kappa grad T = (mu gamma/Pr) grad e; lambda = 0;
 *           sutherland != 0: mu = mu0 (e/e0)^(3/2) (1 + suth_s)/(e/e0 + suth_s),
 *           suth_s = S/T0 (0.368 for S = 110.4 K, T0 = 300 K); otherwise mu = mu0.
 *           Interfaces: Roe (Harten fix on the acoustic waves, delta = harten * c_Roe)
 *           or Rusanov, minus the interface viscous flux.
 *  All kinds: eta_ip >= 0 adds the interior-penalty term to the interface gradient.
 *  Interface viscous (diffusive) flux, Sec. 2.1 step 4: viscous_flux = SD_VISC_STATE_AVG
 *  (option (a), the flux of the averaged state and averaged gradient; the paper's choice)
 *  or SD_VISC_FLUX_AVG (option (b), the average of the two sides' fluxes, each from its
 *  own trace and own interface gradient; the penalty term is added to both sides'
 *  normal gradients). */
typedef enum { SD_VISC_STATE_AVG = 0, SD_VISC_FLUX_AVG = 1 } sd_viscous_flux;
/* Porous medium diffusivity m |u|^(m-1) (Sec. 4.3): SD_PME_COEF_FLUX evaluates it at the
 * flux points from the extrapolated solution (the paper's results); SD_PME_COEF_SOLUTION
 * evaluates it at the solution points and extrapolates it like any field (the variant the
 * paper mentions); at an interface option (a) uses the average of the two sides'
 * extrapolated values, option (b) each side's own. Ignored for the other kinds. */
typedef enum { SD_PME_COEF_FLUX = 0, SD_PME_COEF_SOLUTION = 1 } sd_pme_coef;
typedef struct {
    sd_physics_kind kind;
    double nu;
    double m_pme;
    double gamma, Pr, Re, Ma, rho0, u0, L;
    int sutherland;
    double suth_s;
    sd_riemann riemann;
    double harten;
    double eta_ip;      /* interior penalty (Sec. 3): the interface average of the normal
                           gradient gains eta_ip (p+1)^2 / h_d (u_R - u_L); 0 = off */
    sd_viscous_flux viscous_flux;
    sd_pme_coef pme_coef;
} sd_physics;

/* Volume diagnostics (Sec. 4.4), FP64, Gauss quadrature over every element.
 * NS: ke = 1/2 int u.u, ke_rho = 1/2 int rho u.u, enstrophy = int |curl u|^2 (velocity
 * gradient from the conservative auxiliary gradient at the solution points), mass,
 * mom[3], energy = int rho E. Scalar: mass = int u, l2sq = int u^2. volume = |Omega|.
 * nonfinite != 0 when any state value is NaN or Inf. */
typedef struct {
    double t;
    double ke, ke_rho, enstrophy;
    double mass, mom[3], energy;
    double l2sq, volume;
    int nonfinite;
} sd_diag;

typedef struct sd_ctx sd_ctx;

/* Create a context for one grid, polynomial degree p, scheme, physics and residual
 * precision; all scratch is allocated here on the current CUDA device.
 *   p: 1..8 (n = p + 1 points per direction). dim: 1 or 3 (NS: 3 only).
 *   stream: a cudaStream_t (NULL = legacy default stream).
 * Returns SD_EINVAL / SD_EUNSUPPORTED / SD_ENOMEM / SD_ECUDA, else SD_OK and *out. */
sd_status sd_init(const sd_mesh* mesh, int p, sd_scheme scheme, const sd_physics* phys,
                  sd_precision prec, void* stream, sd_ctx** out);

/* Create a context on a periodic grid of curved (trilinear) hexahedra: the element map of
 * Sec. 2 with K = 8 corner nodes, the transformed equations Eqs. ns:mapped / adj:f and the
 * steps of Sec. 2.3 with the metric terms taken point by point (row d of S = adj(dx/dxi)
 * at the flux points of family d, J^-1 at the solution points).
 *   mesh: dim must be 3; ne gives the element counts; lo / hi are ignored.
 *   nodes: host array of 3 * (ne[2]+1) * (ne[1]+1) * (ne[0]+1) doubles, read only during
 *     the call: nodes[((c*(nz+1) + k)*(ny+1) + j)*(nx+1) + i] is component c (x, y, z) of
 *     corner node (i, j, k). Element (ex, ey, ez) has the corners (ex+a, ey+b, ez+c), a, b, c
 *     in {0, 1}; xi runs along i, eta along j, zeta along k. The last node along each axis is
 *     the periodic image of the first: node(nx, j, k) - node(0, j, k) must be the same
 *     vector for every j, k (likewise along y and z), else SD_EINVAL.
 *   Every element needs a positive Jacobian at its solution points, else SD_EINVAL.
 * The other arguments are those of sd_init. State layout, sd_residual, sd_residual_host,
 * sd_rk_step and sd_diagnostics (Gauss quadrature with weights J w_i w_j w_k; volume =
 * the domain's) work as on a Cartesian grid. The interior penalty uses, per interface,
 * 1/h = |A_f| / min(V_{e-}, V_{e+}) (A_f: integral of the area vector over the face,
 * V: element volumes) along the face's unit normal (Sec. 3). Not available here
 * (SD_EUNSUPPORTED): the learned closure and per-element fluxes, and the porous-medium
 * diffusivity at the solution points. */
sd_status sd_init_curvilinear(const sd_mesh* mesh, const double* nodes, int p, sd_scheme scheme,
                              const sd_physics* phys, sd_precision prec, void* stream, sd_ctx** out);

/* 1 if the context was made by sd_init_curvilinear, else 0. */
int sd_is_curvilinear(const sd_ctx* ctx);

void sd_destroy(sd_ctx* ctx);
sd_status sd_set_stream(sd_ctx* ctx, void* stream);

/* Number of values in one state array: nvar * prod(ne) * n^dim. */
size_t sd_state_size(const sd_ctx* ctx);
int sd_nvar(const sd_ctx* ctx);

/* 1D solution points xi_i in [-1, 1] (n values) and Gauss weights (n values), as the
 * library computed them (Newton iteration on the Legendre recurrence). Host pointers. */
sd_status sd_points(const sd_ctx* ctx, double* xi, double* w);

/* R = dU/dt (Sec. 2.3 steps 1-5). U, R: device arrays in the layout above, of the
 * context's precision (float for SD_F32, double for SD_F64), sd_state_size values each;
 * they must not overlap. Asynchronous on the context stream. */
sd_status sd_residual(sd_ctx* ctx, const void* U, void* R);

/* The same residual through host memory: copies U_host to the device, evaluates R and
 * copies it back into R_host, on the context stream, and synchronises the stream before
 * returning. U_host / R_host: host arrays of the context's precision (pinned memory
 * gives full copy bandwidth; pageable memory works). */
sd_status sd_residual_host(sd_ctx* ctx, const void* U_host, void* R_host);

/* One explicit time step of the FP64 state U64 (device, sd_state_size doubles), in place:
 * U64 <- U64 + dt-integral of R, with the Runge-Kutta scheme rk (Sec. 4.4 integrates in
 * time with the five-stage, fourth-order strong-stability-preserving scheme of Spiteri and
 * Ruuth, SD_SSPRK54; SD_RK4 is the classical scheme; SD_LSRK54 the two-register low-storage
 * scheme of Carpenter and Kennedy). t is the time at the start of the step (the residual
 * is autonomous; t is recorded only). Asynchronous on the context stream.
 * How the stages are held depends on the context's precision and stage mode:
 *   SD_F64 contexts: FP64 residual, FP64 stage states and registers.
 *   SD_F32 contexts, SD_RK_STAGES_F32 (the default): within a step every stage state is
 *     U + d_j, U the FP64 state at the start of the step. The increments d_j = O(dt) and
 *     the stage registers are FP32; each stage's FP32 residual is evaluated on X + d_j,
 *     X = U minus the reference offsets rounded to FP32 once per step. U itself is updated
 *     in FP64 once per step (U <- U + d_s).
 *   SD_F32 contexts, SD_RK_STAGES_F64 (sd_set_rk_stages): FP64 stage states and registers
 *     as in SD_F64 contexts; only each stage's residual is FP32, evaluated on the FP64 stage
 *     state (offsets removed) rounded to FP32. */
sd_status sd_rk_step(sd_ctx* ctx, double* U64, double t, double dt, sd_rk rk);

/* Stage arithmetic of sd_rk_step on an SD_F32 context (see sd_rk_step). Selecting
 * SD_RK_STAGES_F64 allocates three FP64 state-sized registers the first time (the one call
 * besides sd_init and sd_closure_enable that allocates; SD_ENOMEM if that fails). On an SD_F64
 * context only SD_RK_STAGES_F64 is accepted (SD_EUNSUPPORTED otherwise). */
typedef enum { SD_RK_STAGES_F32 = 0, SD_RK_STAGES_F64 = 1 } sd_rk_stages;
sd_status sd_set_rk_stages(sd_ctx* ctx, sd_rk_stages mode);

/* sd_rk_step one stage at a time, for callers that must act between stages (a decomposed
 * grid refreshes the ghost elements of every stage input from its neighbours). sd_rk_prepare
 * writes the first stage input from U64 and returns it in *input (a device array owned by
 * the context: sd_state_size values of the residual precision, offsets removed from rho and
 * rho E for Navier-Stokes). sd_rk_stage(k) evaluates the residual of the current stage input,
 * applies stage k of rk and returns the next stage input in *input (NULL after the last
 * stage, which updates U64). k runs 0 .. 3 (SD_RK4) or 0 .. 4; sd_rk_prepare followed by all
 * stages is exactly sd_rk_step. Asynchronous on the context stream. */
sd_status sd_rk_prepare(sd_ctx* ctx, double* U64, void** input);
sd_status sd_rk_stage(sd_ctx* ctx, double* U64, int k, double dt, sd_rk rk, void** input);

/* ---- Sub-domains of a decomposed grid (Secs. 2.1-2.3: the residual of an element reads
 * the elements of its stencil only: compact max|d| <= 1 and |d|_1 <= 2, BR1 |d|_1 <= 2).
 * A sub-domain context is an sd_init context over the owned block extended by ghost layers;
 * its residual is exact on the owned block once the ghosts hold the neighbours' data. These
 * calls move that data; the caller decides which elements go where (paper_2608_09615_b300.decomp
 * builds the lists and runs the exchanges). Element and face index lists are device int32
 * arrays; indices outside the context's grid are skipped, never accessed. Asynchronous. */

/* buf[v][k][p] = U[v][elems[k]][p] for k < count (whole elements, every variable), and the
 * inverse. U: a state in the context's layout whose values are value_bytes (4 or 8) wide (the
 * residual precision's stage inputs, or an FP64 state on any context); buf: count * nvar * n^dim
 * such values. The values are copied as raw words. */
sd_status sd_pack_elements(sd_ctx* ctx, const void* U, int value_bytes, const int* elems, int count, void* buf);
sd_status sd_unpack_elements(sd_ctx* ctx, const void* buf, int value_bytes, const int* elems, int count,
                             void* U);

/* Values in one face block of the context's own-interface-gradient buffer (0 on curved grids). */
size_t sd_face_gradient_size(const sd_ctx* ctx);
/* Face blocks (elems[k], faces[k]) of the own-interface-gradient buffer written by
 * sd_residual_begin, gathered into buf (count * sd_face_gradient_size values), and the
 * inverse: the BR1 scheme's second exchange (Eq. v:e), between sd_residual_begin and
 * sd_residual_end. Faces: 2 d for the -d face, 2 d + 1 for the +d face. Cartesian grids. */
sd_status sd_pack_face_gradients(sd_ctx* ctx, const int* elems, const int* faces, int count, void* buf);
sd_status sd_unpack_face_gradients(sd_ctx* ctx, const void* buf, const int* elems, const int* faces,
                                   int count);

/* sd_residual in two halves: begin = the traces and each element's own interface gradients
 * (Sec. 2.3 steps 1-4 up to the interface values); end = the common interface fluxes and the
 * divergence (steps 4-5), reading what begin left in the context. sd_residual_begin followed
 * by sd_residual_end equals sd_residual. Cartesian grids, without the learned closure. */
sd_status sd_residual_begin(sd_ctx* ctx, const void* U);
sd_status sd_residual_end(sd_ctx* ctx, const void* U, void* R);

/* Restrict sd_diagnostics to the elements [lo[d], hi[d]) along each axis (a sub-domain's
 * owned block; the reported volume is the block's); lo = hi = NULL removes the restriction. */
sd_status sd_set_owned_box(sd_ctx* ctx, const int* lo, const int* hi);

/* FP64 volume diagnostics of the FP64 device state U64 at time t. Synchronises the
 * context stream and writes *out (host). Returns SD_ENONFINITE (with *out filled)
 * when the state holds a NaN or Inf. */
sd_status sd_diagnostics(sd_ctx* ctx, const double* U64, double t, sd_diag* out);

/* Profiling (CUDA events on the context stream). While enabled, every kernel launch of
 * the context is bracketed by two events; sd_profile_read synchronises the stream and
 * returns, per kernel class (SD_K_TRACE, SD_K_GRAD, SD_K_FLUX, SD_K_OTHER, SD_K_FACE), the summed
 * device time in ms and the launch count since the last read, then resets them.
 * Enabling creates the events (no device memory); disabling destroys them. */
enum { SD_K_TRACE = 0, SD_K_GRAD = 1, SD_K_FLUX = 2, SD_K_OTHER = 3, SD_K_FACE = 4, SD_K_COUNT = 5 };
sd_status sd_profile_enable(sd_ctx* ctx, int on);
sd_status sd_profile_read(sd_ctx* ctx, double* ms, long long* launches);

/* Total number of kernels the context has launched since sd_init. */
long long sd_launch_count(const sd_ctx* ctx);

/* ---- Per-element MLP closure network (64 -> 128 -> 128 -> 15, ReLU hidden layers) ----
 * The paper has no learned component; this network is the sub-grid closure of the
 * coarse Taylor-Green runs (features and targets are defined in the library's closure
 * functions). BF16 operands on the tensor cores with FP32 accumulation; FP32 biases,
 * FP32 master parameters and Adam moments. All buffers are device buffers owned by the
 * caller; these calls allocate nothing and run asynchronously on `stream`.
 * Parameter vector (FP32, sd_mlp_param_count() values, packed): W1[128][64], b1[128],
 * W2[128][128], b2[128], W3[16][128] (row 15 zero), b3[16] (entry 15 zero). Wb: the BF16
 * copy of the same vector (biases unused). X: BF16 [M][64]. Y, T, dY: FP32 [M][15].
 * H: BF16 activation cache [2][M][128] written by the forward pass, read by backward. */
int sd_mlp_param_count(void);
/* Wb <- BF16(P). */
sd_status sd_mlp_cast(const float* P, void* Wb, void* stream);
/* Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for the M rows of X; fills H. */
sd_status sd_mlp_forward(const void* X, int M, const void* Wb, const float* P, float* Y,
                         void* H, void* stream);
/* Mean-squared error over the M x 15 outputs: *loss (device FP64) and dY = dL/dY.
 * part: device FP64 scratch of 64 values (block partial sums). */
sd_status sd_mlp_loss(const float* Y, const float* T, int M, float* dY, double* part,
                      double* loss, void* stream);
/* Parameter gradient grad (FP32, packed like P) of the loss whose output gradient is dY.
 * part: device FP32 scratch of ceil(M/64) * sd_mlp_param_count() values (per-block partial
 * gradients, summed in a fixed order). */
sd_status sd_mlp_backward(const void* X, const void* H, const float* dY, int M, const void* Wb,
                          float* part, float* grad, void* stream);
/* One Adam step (step = 1, 2, ...) on the masters P with moments m1, m2; refreshes Wb. */
sd_status sd_mlp_adam(float* P, float* m1, float* m2, const float* grad, void* Wb, int step,
                      float lr, float b1, float b2, float eps, void* stream);

/* ---- Learned sub-grid closure of coarse Navier-Stokes runs (no counterpart in the paper;
 * see the closure definitions in the oracle's closure module: L2-projection filter,
 * sub-grid flux targets, 64 element features, per-element flux injection). ---- */

/* Extra per-element flux added by sd_residual / sd_rk_step: tau (device FP32,
 * [nelem][15], tau[e][3 v + d] for variable v and direction d) is added to F at the
 * element's interior flux points, and the average of the two elements' values at each
 * interface. NULL removes it. The buffer stays the caller's; it is read at every residual. */
sd_status sd_set_flux_tau(sd_ctx* ctx, const float* tau);

/* Closure data of the state U (device, context precision, Navier-Stokes): X = the 64
 * element features [nelem][64] FP32 and/or means = the Gauss means of the physical flux
 * F = F_c - F_v at the solution points, [nelem][15] FP64 (either pointer may be NULL).
 * Uses the context's trace buffer; asynchronous. */
sd_status sd_closure_data(sd_ctx* ctx, const void* U, float* X, double* means);

/* The 1D L2 projection from r fine elements of degree pf onto one coarse element of degree
 * pc (host, row-major (pc+1) x (r (pf+1))): coarse nodal value a from the fine values. */
sd_status sd_filter_matrix(int pf, int pc, int r, double* P);

/* Box filter: L2 projection of the fine FP64 state Uf (nv variables) onto the nested coarse
 * grid of ne_coarse[3] elements (r fine elements per coarse element and axis) -> Uc (FP64).
 * P: the device copy of sd_filter_matrix(nf - 1, nc - 1, r). */
sd_status sd_filter_project(const double* Uf, double* Uc, const double* P, int nv,
                            const int* ne_coarse, int r, int nf, int nc, void* stream);

/* Sub-grid flux targets tau[ec][k] = mean over the r^3 children of fine_means[ef][k] -
 * coarse_means[ec][k] (FP32 out, [nelem_coarse][15]). */
sd_status sd_closure_targets(const double* fine_means, const double* coarse_means, float* tau,
                             const int* ne_coarse, int r, void* stream);

/* Column statistics and standardisation of row-major FP32 tables (device). */
sd_status sd_colstats(const float* A, int rows, int cols, float* mu, float* sigma, void* stream);
sd_status sd_standardise(const float* A, int rows, int cols, const float* mu, const float* sigma,
                         void* out_bf16, float* out_f32, void* stream);
sd_status sd_unstandardise(const float* Y, int rows, int cols, const float* mu, const float* sigma,
                           float* out, void* stream);

/* Attach a trained closure network to the context: every residual then evaluates the
 * features of its input state, the network (standardised input mu_x/sig_x [64], output
 * un-standardised with mu_t/sig_t [15]) and adds the resulting per-element flux. Wb, P and
 * the statistics are caller-owned device buffers (see sd_mlp_*). Enabling allocates the
 * context's closure buffers (features, activations, flux) once; Wb = NULL detaches. */
sd_status sd_closure_enable(sd_ctx* ctx, const void* Wb, const float* P, const float* mu_x,
                            const float* sig_x, const float* mu_t, const float* sig_t);

/* Allocation-free FP32 residual, for callers that cannot let a library allocate device
 * memory (an application whose own pool allocator owns the whole device, or a code path
 * that must not pay for an allocation or for the synchronisation cudaFree can imply).
 * The paper has no counterpart; it is the same FP32 residual as sd_residual, without a
 * context: mesh, p, scheme and physics as for sd_init; U, R device FP32 arrays as for
 * sd_residual (they must not overlap); work enqueued on `stream`.
 * Scratch: a static device array of 36 MiB (9 Mi FP32 values) inside the library, held by
 * every GPU that loads the library until the process exits. A grid needs about
 * nelem * (2 dim (F + G) + dim F) values, with F = nvar n^(dim-1) and G = ngrad n^(dim-1)
 * each rounded up to a multiple of 4 (ngrad = 9 for Navier-Stokes, 1 otherwise; 3375
 * elements at p = 4 for Navier-Stokes fit); larger grids return SD_EINVAL with a message
 * and nothing is launched. The first call on a device looks up the array's device address
 * and uploads the operator tables for that device; make that first call before any stream
 * capture. Every call shares the array: calls whose kernels overlap on the GPU race (give
 * them one stream, or order them). No memory is allocated by this call. */
sd_status sd_residual_f32_noalloc(const sd_mesh* mesh, int p, sd_scheme scheme,
                                  const sd_physics* phys, const float* U, float* R, void* stream);

/* FP32 FMA throughput of the current device in TFLOP/s (FMA = 2 flops), measured by a
 * fully occupied kernel of independent FMA chains; the denominator of the residual kernels'
 * ALU roofline. Not part of the method (the paper has no counterpart). packed = 0: scalar
 * fma.rn.f32; packed = 1: paired fma.rn.f32x2. Synchronous; allocates and frees 1 KB of
 * device memory and its own stream; takes about 20 ms. */
sd_status sd_measure_fp32_peak(int packed, double* tflops);

const char* sd_status_str(sd_status s);
/* Text of the last error raised on the calling thread ("" if none). */
const char* sd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SD_H */
