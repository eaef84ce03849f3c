// Allocation-free FP32 residual entry point (see sd_residual_f32_noalloc in include/sd.h).
//
// Some callers cannot let a library call cudaMalloc: applications that hand the whole
// device memory to their own pool allocator and allow no allocation outside it, and code
// paths that must not pay for an allocation or for the device synchronisation that
// cudaFree can imply. For them this entry point evaluates the same FP32 residual as
// sd_residual without a context: the face-trace scratch lives in the file-scope device
// array below, whose size is fixed at build time and which every GPU that loads this
// library holds until the process exits.
#include <math.h>
#include <string.h>

#include <mutex>

#include "sd_internal.h"

// Scratch of the allocation-free path: the face traces of u, the interface gradient
// components and the interface fluxes of every element. Every call rewrites all the values it reads, so
// nothing has to be cleared between calls; calls that overlap on the GPU share it and race.
static __device__ __align__(256) float g_noalloc_scratch[SD_NOALLOC_SCRATCH_FLOATS];

// Host code cannot use g_noalloc_scratch as a device pointer (in host code the name is a
// host-side stand-in): its device address is taken once per device, with that device
// current, and cached.
static float* scratch_address(int device) {
    static std::mutex mu;
    static float* addr[64] = {nullptr};
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        addr[device] = static_cast<float*>(p);
    }
    return addr[device];
}

// Validate the problem and fill a stack context (operators, sizes); no CUDA call.
static sd_status prepare(const sd_mesh* mesh, int p, sd_scheme scheme, const sd_physics* phys,
                         void* stream, sd_ctx* c) {
    if (!mesh || !phys) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (mesh->dim != 1 && mesh->dim != 3) { sdi_set_error("dim must be 1 or 3"); return SD_EUNSUPPORTED; }
    if (p < 1 || p > SD_MAX_N - 1) { sdi_set_error("p must be in 1..%d", SD_MAX_N - 1); return SD_EUNSUPPORTED; }
    if (scheme != SD_BR1 && scheme != SD_COMPACT) { sdi_set_error("bad scheme"); return SD_EINVAL; }
    if (phys->kind != SD_HEAT && phys->kind != SD_PME && phys->kind != SD_NS) {
        sdi_set_error("bad physics kind");
        return SD_EINVAL;
    }
    if (phys->kind == SD_NS && mesh->dim != 3) { sdi_set_error("Navier-Stokes needs dim = 3"); return SD_EUNSUPPORTED; }
    if (phys->kind == SD_NS &&
        (!(phys->gamma > 1.0) || !(phys->Pr > 0.0) || !(phys->Re > 0.0) || !(phys->Ma > 0.0) ||
         !(phys->rho0 > 0.0) || !(phys->u0 > 0.0) || !(phys->L > 0.0) || phys->harten < 0.0 ||
         (phys->riemann != SD_ROE && phys->riemann != SD_RUSANOV))) {
        sdi_set_error("bad Navier-Stokes parameters");
        return SD_EINVAL;
    }
    if (phys->kind == SD_PME && !(phys->m_pme >= 1.0)) { sdi_set_error("m_pme must be >= 1"); return SD_EINVAL; }
    if (!(phys->eta_ip >= 0.0) ||
        (phys->viscous_flux != SD_VISC_STATE_AVG && phys->viscous_flux != SD_VISC_FLUX_AVG) ||
        (phys->pme_coef != SD_PME_COEF_FLUX && phys->pme_coef != SD_PME_COEF_SOLUTION)) {
        sdi_set_error("bad eta_ip, viscous_flux or pme_coef");
        return SD_EINVAL;
    }
    long long nelem = 1;
    for (int d = 0; d < mesh->dim; ++d) {
        if (mesh->ne[d] < 1) { sdi_set_error("ne[%d] must be >= 1", d); return SD_EINVAL; }
        if (!(mesh->hi[d] > mesh->lo[d])) { sdi_set_error("hi[%d] must exceed lo[%d]", d, d); return SD_EINVAL; }
        nelem *= mesh->ne[d];
    }
    if (nelem > (1LL << 30)) { sdi_set_error("too many elements"); return SD_EUNSUPPORTED; }
    memset(c, 0, sizeof(*c));
    c->dim = mesh->dim;
    for (int d = 0; d < 3; ++d) {
        c->ne[d] = d < mesh->dim ? mesh->ne[d] : 1;
        c->lo[d] = d < mesh->dim ? mesh->lo[d] : 0.0;
        c->hi[d] = d < mesh->dim ? mesh->hi[d] : 1.0;
        c->h[d] = (c->hi[d] - c->lo[d]) / c->ne[d];
    }
    c->nelem = (int)nelem;
    c->p = p;
    c->n = p + 1;
    c->nvar = phys->kind == SD_NS ? 5 : 1;
    c->ngrad = phys->kind == SD_NS ? 9 : 1;
    c->scheme = scheme;
    c->phys = *phys;
    c->prec = SD_F32;
    c->stream = (cudaStream_t)stream;
    c->J = 1.0;
    for (int d = 0; d < c->dim; ++d) c->J *= c->h[d] / 2.0;
    sdi_build_operators(c);
    int np = 1, nq = 1;
    for (int d = 0; d < c->dim; ++d) np *= c->n;
    for (int d = 0; d < c->dim - 1; ++d) nq *= c->n;
    c->npts = (size_t)c->nelem * np;
    c->nstate = c->npts * c->nvar;
    // face blocks padded to a multiple of 4 values (16-byte aligned, copied in 16-byte pieces)
    // (scalar trace blocks also hold the traces of the porous-medium diffusivity)
    const size_t fst = ((size_t)c->nvar * nq + (c->nvar == 1 ? nq : 0) + 3) / 4 * 4;
    const size_t gst = ((size_t)c->ngrad * nq + 3) / 4 * 4;
    c->ntu = (size_t)c->nelem * 2 * c->dim * fst;
    c->ntg = (size_t)c->nelem * 2 * c->dim * gst;
    c->nfh = (size_t)c->nelem * c->dim * fst;
    c->esize = sizeof(float);
    return SD_OK;
}

extern "C" sd_status sd_residual_f32_noalloc(const sd_mesh* mesh, int p, sd_scheme scheme,
                                             const sd_physics* phys, const float* U, float* R,
                                             void* stream) {
    if (!U || !R) { sdi_set_error("null argument"); return SD_EINVAL; }
    sd_ctx c;
    sd_status st = prepare(mesh, p, scheme, phys, stream, &c);
    if (st != SD_OK) return st;
    const size_t tu = ((c.ntu + 63) / 64) * 64;            // keeps Tg and Fh 256-byte aligned
    const size_t tg = ((c.ntg + 63) / 64) * 64;
    if (tu + tg + c.nfh > (size_t)SD_NOALLOC_SCRATCH_FLOATS) {
        sdi_set_error("sd_residual_f32_noalloc: this grid needs %zu scratch values; the static "
                      "scratch holds %d (use sd_init / sd_residual for larger grids)",
                      tu + tg + c.nfh, SD_NOALLOC_SCRATCH_FLOATS);
        return SD_EINVAL;
    }
    if ((const void*)U < (const void*)(R + c.nstate) && (const void*)R < (const void*)(U + c.nstate)) {
        sdi_set_error("U and R overlap");
        return SD_EINVAL;
    }
    if (cudaGetDevice(&c.device) != cudaSuccess) { sdi_set_error("no CUDA device"); return SD_ECUDA; }
    float* base = scratch_address(c.device);
    if (!base) { sdi_set_error("cudaGetSymbolAddress of the static scratch failed"); return SD_ECUDA; }
    if ((st = sdi_upload_f32(&c)) != SD_OK) return st;
    c.Tu = base;
    c.Tg = base + tu;
    c.Fh = base + tu + tg;
    return sdi_residual_f32(&c, U, R, 0);
}
