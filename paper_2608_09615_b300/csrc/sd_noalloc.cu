// Allocation-free FP32 residual entry point (see sd_residual_f32_noalloc in include/sd.h).
//
// Some callers cannot let a library call cudaMalloc: applications that hand the whole
// device memory to their own pool allocator and allow no allocation outside it, and code
// paths that must not pay for an allocation or for the device synchronisation that
// cudaFree can imply. For them this entry point evaluates the same FP32 residual as
// sd_residual without a context: the face-trace scratch lives in the file-scope device
// array below, whose size is fixed at build time and which every GPU that loads this
// library holds until the process exits.
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

extern "C" sd_status sd_residual_f32_noalloc(const sd_mesh* mesh, int p, sd_scheme scheme,
                                             const sd_physics* phys, const float* U, float* R,
                                             void* stream) {
    if (!U || !R) { sdi_set_error("null argument"); return SD_EINVAL; }
    sd_ctx c;
    sd_status st = sdi_setup(mesh, p, scheme, phys, SD_F32, stream, &c);
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
