// Host-side launchers of the residual kernels, templated on the residual precision.
#pragma once

#include <algorithm>
#include <mutex>

#include "sd_internal.h"
#include "sd_kernels.cuh"
#include "sd_line.cuh"
#include "sd_closure.cuh"

namespace sdk {

template <typename real, int N>
static Ops<real, N> make_ops(const sd_ctx* c) {
    Ops<real, N> o;
    for (int k = 0; k < (N + 1) * N; ++k) o.L[k] = (real)c->L[k];
    for (int k = 0; k < N * (N + 1); ++k) o.M[k] = (real)c->M[k];
    for (int k = 0; k < N * N; ++k) o.D[k] = (real)c->D[k];
    for (int d = 0; d < 3; ++d) {
        const double th = d < c->dim ? 2.0 / c->h[d] : 0.0;
        o.two_h[d] = (real)th;
        o.corrL[d] = (real)(th * c->alpha);
        o.corrR[d] = (real)(th * c->beta);
    }
    return o;
}

template <typename real>
static Phys<real> make_phys(const sd_ctx* c) {
    const sd_physics& s = c->phys;
    Phys<real> P;
    P.kind = (int)s.kind;
    P.sutherland = s.sutherland ? 1 : 0;
    P.riemann = (int)s.riemann;
    P.vflux = (int)s.viscous_flux;
    P.pme_sol = (s.kind == SD_PME && s.pme_coef == SD_PME_COEF_SOLUTION) ? 1 : 0;
    P.nu = (real)s.nu;
    P.m_pme = (real)s.m_pme;
    const double gamma = s.gamma;
    const double mu0 = s.rho0 * s.u0 * s.L / (s.Re > 0 ? s.Re : 1.0);
    const double p0 = s.kind == SD_NS ? s.rho0 * (s.u0 / s.Ma) * (s.u0 / s.Ma) / gamma : 0.0;
    const double e0 = s.kind == SD_NS ? p0 / ((gamma - 1.0) * s.rho0) : 1.0;
    P.gamma = (real)gamma;
    P.gm1 = (real)(gamma - 1.0);
    P.gamma_Pr = (real)(gamma / (s.Pr > 0 ? s.Pr : 1.0));
    P.mu0 = (real)mu0;
    P.p0 = (real)p0;
    P.rhoE0 = (real)(p0 / (gamma - 1.0));
    P.inv_e0 = (real)(1.0 / e0);
    P.suth_s = (real)s.suth_s;
    P.suth_1ps = (real)(1.0 + s.suth_s);
    P.harten = (real)s.harten;
    P.rho0 = (real)(s.kind == SD_NS ? s.rho0 : 0.0);
    P.H0 = (real)(p0 / (gamma - 1.0) + p0);
    return P;
}

// reference offsets removed from variables 0 and 4 when the residual kernels stage a
// Navier-Stokes state (zero for scalar physics)
inline void stage_offsets(const sd_ctx* c, double& off0, double& off4) {
    off0 = off4 = 0.0;
    if (c->phys.kind == SD_NS) {
        const double p0 = c->phys.rho0 * (c->phys.u0 / c->phys.Ma) * (c->phys.u0 / c->phys.Ma) / c->phys.gamma;
        off0 = c->phys.rho0;
        off4 = p0 / (c->phys.gamma - 1.0);
    }
}

template <typename real>
static LineGeo<real> make_geo(const sd_ctx* c, int offset_in) {
    LineGeo<real> o;
    for (int d = 0; d < 3; ++d) {
        const double th = d < c->dim ? 2.0 / c->h[d] : 0.0;
        o.two_h[d] = (real)th;
        o.corrL[d] = (real)(th * c->alpha);
        o.corrR[d] = (real)(th * c->beta);
    }
    double off0, off4;
    stage_offsets(c, off0, off4);
    o.off0 = offset_in ? real(0) : (real)off0;
    o.off4 = offset_in ? real(0) : (real)off4;
    for (int d = 0; d < 3; ++d)
        o.tip[d] = (real)(d < c->dim ? c->phys.eta_ip * c->n * c->n / c->h[d] : 0.0);
    return o;
}

// upload the 1D operators of n = N to this translation unit's constant table on the
// current device (once per device and n)
template <typename real, int N>
static sd_status upload_ops(const sd_ctx* c) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lock(mu);
    if (c->device >= 0 && c->device < 64 && done[c->device]) return SD_OK;
    OpTab<real, N> t;
    for (int k = 0; k < (N + 1) * N; ++k) t.L[k] = (real)c->L[k];
    for (int k = 0; k < N * (N + 1); ++k) t.M[k] = (real)c->M[k];
    for (int k = 0; k < N * N; ++k) t.D[k] = (real)c->D[k];
    for (int k = 0; k < (N + 1) * N; ++k) t.LD[k] = (real)c->LD[k];
    for (int f = 0; f <= N; ++f) {
        t.LM0[f] = (real)c->LM0[f];
        t.LMN[f] = (real)c->LMN[f];
    }
    if (cudaMemcpyToSymbol(c_op<real, N>, &t, sizeof(t)) != cudaSuccess) {
        sdi_set_error("upload of the operator table failed");
        return SD_ECUDA;
    }
    if (c->device >= 0 && c->device < 64) done[c->device] = true;
    return SD_OK;
}

template <typename real>
static sd_status upload_dispatch(const sd_ctx* c) {
    switch (c->n) {
        case 2: return upload_ops<real, 2>(c);
        case 3: return upload_ops<real, 3>(c);
        case 4: return upload_ops<real, 4>(c);
        case 5: return upload_ops<real, 5>(c);
        case 6: return upload_ops<real, 6>(c);
        case 7: return upload_ops<real, 7>(c);
        case 8: return upload_ops<real, 8>(c);
        case 9: return upload_ops<real, 9>(c);
        default: return SD_EUNSUPPORTED;
    }
}

// flux-kernel operator rows with the metric folded in (FluxOps), from the context's FP64
// (80-bit host built) operators
template <typename real, int N>
static FluxOps<real, N> make_flux_ops(const sd_ctx* c) {
    FluxOps<real, N> o;
    for (int d = 0; d < 3; ++d) {
        const double th = d < c->dim ? 2.0 / c->h[d] : 0.0;
        for (int i = 0; i < N; ++i)
            for (int f = 0; f <= N; ++f) o.Mn[d][i][f] = (real)(-th * c->M[i * (N + 1) + f]);
        for (int f = 0; f <= N; ++f) {
            for (int i = 0; i < N; ++i) o.LDn[d][f][i] = (real)(th * c->LD[f * N + i]);
            o.LM0n[d][f] = (real)(th * c->LM0[f]);
            o.LMNn[d][f] = (real)(th * c->LMN[f]);
        }
    }
    return o;
}

inline Mesh make_mesh(const sd_ctx* c, int e_begin = 0, int e_end = -1) {
    Mesh g;
    for (int d = 0; d < 3; ++d) g.ne[d] = c->ne[d];
    g.nelem = c->nelem;
    g.e_begin = e_begin;
    g.e_end = e_end < 0 ? c->nelem : e_end;
    for (int d = 0; d < 3; ++d) {
        g.olo[d] = c->own_set ? c->own_lo[d] : 0;
        g.ohi[d] = c->own_set ? c->own_hi[d] : c->ne[d];
    }
    return g;
}

// elements per block for an element-staged kernel: ~256 threads, shared memory bounded
inline int pick_epb(int tpe, size_t bytes_per_elem) {
    int epb = std::max(1, 256 / tpe);
    while (epb > 1 && (size_t)epb * bytes_per_elem > 100 * 1024) --epb;
    return epb;
}

template <typename K>
static bool set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    if (bytes > 227 * 1024) return false;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes) == cudaSuccess;
}

// the status of a launch whose kernel cannot get the shared memory it needs, with a message
inline sd_status smem_fail(size_t bytes) {
    sdi_set_error("a residual kernel needs %zu bytes of shared memory per block, more than the device grants",
                  bytes);
    return SD_EUNSUPPORTED;
}

// number of SMs of a device (cached)
inline int sm_count(int device) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> lock(mu);
    const int d = device >= 0 && device < 64 ? device : 0;
    if (!cache[d]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n < 1) n = 1;
        cache[d] = n;
    }
    return cache[d];
}

// grid of a persistent kernel: as many blocks as can be resident on the device, at most
// one per element group
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, long long ngroups, int device) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1)
        occ = 1;
    const long long g = (long long)occ * sm_count(device);
    return (int)std::max<long long>(1, std::min<long long>(g, ngroups));
}

inline int trace_blocks(long long total) {
    long long b = (total + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), 148LL * 64);
}

// ------------------------------------------------------------------ closure data kernels
template <typename real, int N>
static sd_status features_impl(sd_ctx* c, const real* U, float* X, int offset_in) {
    using LL = LineLayout<N, 3, 5>;
    const LineGeo<real> geo = make_geo<real>(c, offset_in);
    const Mesh g = make_mesh(c);
    const Phys<real> P = make_phys<real>(c);
    const size_t sg = LL::NBR_BYTES + (size_t)LL::EB * LL::PER_GRAD * sizeof(real);
    if (!set_smem(k_line_features<real, N>, sg)) return smem_fail(sg);
    const int blocks = (g.nelem + LL::EB - 1) / LL::EB;
    const sd_physics& s = c->phys;
    sdi_prof_begin(c, SD_K_OTHER);
    k_line_features<real, N><<<blocks, LL::THREADS, sg, c->stream>>>(
        U, static_cast<const real*>(c->Tu), geo, g, P, c->dW, c->cl_tmode, c->h[0] / 2.0, s.rho0, s.u0,
        1.0 / s.Re, X);
    sdi_prof_end(c, SD_K_OTHER);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

template <typename real, int N>
static sd_status fluxmean_impl(sd_ctx* c, const real* U, double* out, int offset_in) {
    using LL = LineLayout<N, 3, 5>;
    const LineGeo<real> geo = make_geo<real>(c, offset_in);
    const Mesh g = make_mesh(c);
    const Phys<real> P = make_phys<real>(c);
    const size_t sg = LL::NBR_BYTES + (size_t)LL::EB * LL::PER_GRAD * sizeof(real);
    if (!set_smem(k_line_fluxmean<real, N>, sg)) return smem_fail(sg);
    const int blocks = (g.nelem + LL::EB - 1) / LL::EB;
    sdi_prof_begin(c, SD_K_OTHER);
    k_line_fluxmean<real, N><<<blocks, LL::THREADS, sg, c->stream>>>(
        U, static_cast<const real*>(c->Tu), geo, g, P, c->dW, out);
    sdi_prof_end(c, SD_K_OTHER);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

// per residual with the closure attached: features of the stage state -> standardised
// BF16 input -> MLP -> tau (the traces Tu of this state are already computed)
template <typename real, int N>
static sd_status closure_stage(sd_ctx* c, const real* U, int offset_in) {
    sd_status s = features_impl<real, N>(c, U, c->cl_X, offset_in);
    if (s != SD_OK) return s;
    return sdi_closure_network(c);
}

// One phase of the residual (SDI_PH_TRACE, _GRAD, _FACE, _FLUX) over the elements
// [e_begin, e_end) on `stream`. Each phase reads what the earlier phases wrote for the
// elements it touches (its own and their face neighbours).
template <typename real, int N, int DIM, int NV>
static sd_status residual_phase(sd_ctx* c, const real* U, real* R, int offset_in, int phase, int e_begin,
                                int e_end, cudaStream_t stream) {
    using LL = LineLayout<N, DIM, NV>;
    using FL = FluxLayout<N, DIM, NV>;
    const LineGeo<real> geo = make_geo<real>(c, offset_in);
    const Mesh g = make_mesh(c, e_begin, e_end);
    const Phys<real> P = make_phys<real>(c);
    const long long ne = e_end - e_begin;
    if (ne <= 0) return SD_OK;
    real* Tu = static_cast<real*>(c->Tu);
    real* Tg = static_cast<real*>(c->Tg);
    real* Fh = static_cast<real*>(c->Fh);
    if (phase == SDI_PH_TRACE) {
        const size_t st = TracePipe<real, LL>::BYTES;
        if (!set_smem(k_line_trace<real, N, DIM, NV>, st)) return smem_fail(st);
        const int bt = persistent_grid(k_line_trace<real, N, DIM, NV>, LL::THREADS, st, (ne + LL::EB - 1) / LL::EB,
                                       c->device);
        sdi_prof_begin(c, SD_K_TRACE);
        k_line_trace<real, N, DIM, NV><<<bt, LL::THREADS, st, stream>>>(U, Tu, geo, g, P);
        sdi_prof_end(c, SD_K_TRACE);
    } else if (phase == SDI_PH_GRAD) {
        const size_t sg = GradPipe<real, LL>::BYTES;
        if (!set_smem(k_line_grad<real, N, DIM, NV>, sg)) return smem_fail(sg);
        const int bg = persistent_grid(k_line_grad<real, N, DIM, NV>, LL::THREADS, sg, (ne + LL::EB - 1) / LL::EB,
                                       c->device);
        sdi_prof_begin(c, SD_K_GRAD);
        k_line_grad<real, N, DIM, NV><<<bg, LL::THREADS, sg, stream>>>(U, Tu, Tg, geo, g,
                                                                       c->scheme == SD_COMPACT ? 1 : 0);
        sdi_prof_end(c, SD_K_GRAD);
    } else if (phase == SDI_PH_FACE) {
        sdi_prof_begin(c, SD_K_FACE);
        k_face_flux<real, N, DIM, NV><<<trace_blocks(ne * DIM * LL::NQ), 256, 0, stream>>>(Tu, Tg, Fh, geo, g, P,
                                                                                          c->tau);
        sdi_prof_end(c, SD_K_FACE);
    } else {
        const size_t sf = FluxPipe<real, FL>::BYTES;
        if (!set_smem(k_line_flux<real, N, DIM, NV>, sf)) return smem_fail(sf);
        const int bf = persistent_grid(k_line_flux<real, N, DIM, NV>, FL::THREADS, sf, (ne + FL::EB - 1) / FL::EB,
                                       c->device);
        sdi_prof_begin(c, SD_K_FLUX);
        k_line_flux<real, N, DIM, NV><<<bf, FL::THREADS, sf, stream>>>(U, Tu, Fh, R, geo, g, P, c->tau,
                                                                       make_flux_ops<real, N>(c));
        sdi_prof_end(c, SD_K_FLUX);
    }
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        sdi_set_error("residual launch failed: %s", cudaGetErrorString(err));
        return SD_ECUDA;
    }
    return SD_OK;
}

template <typename real, int N, int DIM, int NV>
static sd_status residual_impl(sd_ctx* c, const real* U, real* R, int offset_in) {
    const int ne = c->nelem;
    sd_status s = residual_phase<real, N, DIM, NV>(c, U, R, offset_in, SDI_PH_TRACE, 0, ne, c->stream);
    if (s != SD_OK) return s;
    if (c->closure_on && NV == 5) {
        s = closure_stage<real, N>(c, U, offset_in);
        if (s != SD_OK) return s;
    }
    for (int ph : {SDI_PH_GRAD, SDI_PH_FACE, SDI_PH_FLUX})
        if ((s = residual_phase<real, N, DIM, NV>(c, U, R, offset_in, ph, 0, ne, c->stream)) != SD_OK) return s;
    return SD_OK;
}

template <typename real, int N>
static sd_status phase_n(sd_ctx* c, const real* U, real* R, int offset_in, int phase, int eb, int ee,
                         cudaStream_t st) {
    if (c->nvar == 5) return residual_phase<real, N, 3, 5>(c, U, R, offset_in, phase, eb, ee, st);
    if (c->dim == 1) return residual_phase<real, N, 1, 1>(c, U, R, offset_in, phase, eb, ee, st);
    return residual_phase<real, N, 3, 1>(c, U, R, offset_in, phase, eb, ee, st);
}

template <typename real>
static sd_status phase_dispatch(sd_ctx* c, const real* U, real* R, int offset_in, int phase, int eb, int ee,
                                cudaStream_t st) {
    switch (c->n) {
        case 2: return phase_n<real, 2>(c, U, R, offset_in, phase, eb, ee, st);
        case 3: return phase_n<real, 3>(c, U, R, offset_in, phase, eb, ee, st);
        case 4: return phase_n<real, 4>(c, U, R, offset_in, phase, eb, ee, st);
        case 5: return phase_n<real, 5>(c, U, R, offset_in, phase, eb, ee, st);
        case 6: return phase_n<real, 6>(c, U, R, offset_in, phase, eb, ee, st);
        case 7: return phase_n<real, 7>(c, U, R, offset_in, phase, eb, ee, st);
        case 8: return phase_n<real, 8>(c, U, R, offset_in, phase, eb, ee, st);
        case 9: return phase_n<real, 9>(c, U, R, offset_in, phase, eb, ee, st);
        default: return SD_EUNSUPPORTED;
    }
}

template <typename real, int N>
static sd_status residual_n(sd_ctx* c, const real* U, real* R, int offset_in) {
    if (c->nvar == 5) return residual_impl<real, N, 3, 5>(c, U, R, offset_in);
    if (c->dim == 1) return residual_impl<real, N, 1, 1>(c, U, R, offset_in);
    return residual_impl<real, N, 3, 1>(c, U, R, offset_in);
}

template <typename real>
static sd_status residual_dispatch(sd_ctx* c, const real* U, real* R, int offset_in) {
    switch (c->n) {
        case 2: return residual_n<real, 2>(c, U, R, offset_in);
        case 3: return residual_n<real, 3>(c, U, R, offset_in);
        case 4: return residual_n<real, 4>(c, U, R, offset_in);
        case 5: return residual_n<real, 5>(c, U, R, offset_in);
        case 6: return residual_n<real, 6>(c, U, R, offset_in);
        case 7: return residual_n<real, 7>(c, U, R, offset_in);
        case 8: return residual_n<real, 8>(c, U, R, offset_in);
        case 9: return residual_n<real, 9>(c, U, R, offset_in);
        default: return SD_EUNSUPPORTED;
    }
}

template <typename real>
static sd_status closure_data_dispatch(sd_ctx* c, const real* U, float* X, double* means, int offset_in) {
    if (c->nvar != 5) { sdi_set_error("closure data need Navier-Stokes"); return SD_EUNSUPPORTED; }
    // traces of this state first
    sd_status st = SD_OK;
    switch (c->n) {
#define SD_CASE(NN)                                                                              \
    case NN: {                                                                                   \
        using LL = LineLayout<NN, 3, 5>;                                                         \
        const LineGeo<real> geo = make_geo<real>(c, offset_in);                                  \
        const Mesh g = make_mesh(c);                                                             \
        const size_t stb = TracePipe<real, LL>::BYTES;                                           \
        if (!set_smem(k_line_trace<real, NN, 3, 5>, stb)) return smem_fail(stb);               \
        const int btr = persistent_grid(k_line_trace<real, NN, 3, 5>, LL::THREADS, stb,          \
                                        (g.nelem + LL::EB - 1) / LL::EB, c->device);            \
        k_line_trace<real, NN, 3, 5><<<btr, LL::THREADS, stb, c->stream>>>(                      \
            U, static_cast<real*>(c->Tu), geo, g, make_phys<real>(c));                           \
        if (X) st = features_impl<real, NN>(c, U, X, offset_in);                                 \
        if (st == SD_OK && means) st = fluxmean_impl<real, NN>(c, U, means, offset_in);          \
        return st;                                                                               \
    }
        SD_CASE(2) SD_CASE(3) SD_CASE(4) SD_CASE(5) SD_CASE(6) SD_CASE(7) SD_CASE(8) SD_CASE(9)
#undef SD_CASE
        default: return SD_EUNSUPPORTED;
    }
}

}  // namespace sdk
