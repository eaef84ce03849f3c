// Host-side launchers of the residual kernels, templated on the residual precision.
#pragma once

#include <algorithm>

#include "sd_internal.h"
#include "sd_kernels.cuh"

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
    return P;
}

inline Mesh make_mesh(const sd_ctx* c) {
    Mesh g;
    for (int d = 0; d < 3; ++d) g.ne[d] = c->ne[d];
    g.nelem = c->nelem;
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

inline int trace_blocks(long long total) {
    long long b = (total + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), 148LL * 64);
}

template <typename real, int N, int DIM, int NV>
static sd_status residual_impl(sd_ctx* c, const real* U, real* R) {
    using FP = Footprint<N, DIM, NV>;
    const Ops<real, N> ops = make_ops<real, N>(c);
    const Mesh g = make_mesh(c);
    const Phys<real> P = make_phys<real>(c);
    const int compact = c->scheme == SD_COMPACT ? 1 : 0;
    real* Tu = static_cast<real*>(c->Tu);
    real* Tg = static_cast<real*>(c->Tg);
    const long long ntr = (long long)g.nelem * FP::NF * NV * FP::NQ;
    sdi_prof_begin(c, SD_K_TRACE);
    k_trace<real, N, DIM, NV><<<trace_blocks(ntr), 256, 0, c->stream>>>(U, Tu, ops, g);
    sdi_prof_end(c, SD_K_TRACE);

    const size_t bg = FP::grad * sizeof(real);
    const int eg = pick_epb(FP::TPE, bg);
    if (!set_smem(k_grad<real, N, DIM, NV>, eg * bg)) return SD_EUNSUPPORTED;
    sdi_prof_begin(c, SD_K_GRAD);
    k_grad<real, N, DIM, NV><<<(g.nelem + eg - 1) / eg, eg * FP::TPE, eg * bg, c->stream>>>(
        U, Tu, Tg, ops, g, compact);
    sdi_prof_end(c, SD_K_GRAD);

    const size_t bf = FP::flux * sizeof(real);
    const int ef = pick_epb(FP::TPE, bf);
    if (!set_smem(k_flux_div<real, N, DIM, NV>, ef * bf)) return SD_EUNSUPPORTED;
    sdi_prof_begin(c, SD_K_FLUX);
    k_flux_div<real, N, DIM, NV><<<(g.nelem + ef - 1) / ef, ef * FP::TPE, ef * bf, c->stream>>>(
        U, Tu, Tg, R, ops, g, P, compact);
    sdi_prof_end(c, SD_K_FLUX);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        sdi_set_error("residual launch failed: %s", cudaGetErrorString(err));
        return SD_ECUDA;
    }
    return SD_OK;
}

template <typename real, int N>
static sd_status residual_n(sd_ctx* c, const real* U, real* R) {
    if (c->nvar == 5) return residual_impl<real, N, 3, 5>(c, U, R);
    if (c->dim == 1) return residual_impl<real, N, 1, 1>(c, U, R);
    return residual_impl<real, N, 3, 1>(c, U, R);
}

template <typename real>
static sd_status residual_dispatch(sd_ctx* c, const real* U, real* R) {
    switch (c->n) {
        case 2: return residual_n<real, 2>(c, U, R);
        case 3: return residual_n<real, 3>(c, U, R);
        case 4: return residual_n<real, 4>(c, U, R);
        case 5: return residual_n<real, 5>(c, U, R);
        case 6: return residual_n<real, 6>(c, U, R);
        case 7: return residual_n<real, 7>(c, U, R);
        case 8: return residual_n<real, 8>(c, U, R);
        case 9: return residual_n<real, 9>(c, U, R);
        default: return SD_EUNSUPPORTED;
    }
}

// shared-memory feasibility of every kernel of this configuration (checked at init)
template <typename real, int N, int DIM, int NV>
static bool smem_ok_impl() {
    using FP = Footprint<N, DIM, NV>;
    return FP::flux * sizeof(real) <= 227 * 1024 && FP::TPE <= 1024;
}

}  // namespace sdk
