// Domain decomposition support: the residual of a sub-domain of a periodic Cartesian grid.
//
// A sub-domain context is an ordinary context (sd_init) over the sub-domain's owned block
// extended by ghost layers along every split axis. Its residual is exact on the owned block
// once the ghost layers hold the neighbours' data, because the residual of an element reads
// only elements within its stencil (Secs. 2.1-2.3): for the compact scheme the element and
// those with max |d| <= 1, |d|_1 <= 2 (the interface gradients need only the own-face
// correction in the normal direction), for BR1 also the elements two away along each axis
// (the normal interface gradient uses both corrections of the neighbour). The kernels wrap
// periodically inside the extended box; whatever the wrap puts in the ghost elements'
// own results is never read by an owned element. Two exchange patterns:
//   compact: one exchange of one ghost layer of the state per residual;
//   BR1:     the state's ghost layer, then, between the gradient and interface-flux phases
//            (sd_residual_begin / sd_residual_end), the ghost elements' own interface
//            gradients on the faces they share with owned elements, from their owners.
// These kernels move whole element blocks of a state (pack / unpack by element index
// lists) and single face blocks of the interface-gradient buffer; the host decides the
// lists, the order of the exchanges and the transport.
#include <cuda_runtime.h>

#include "sd_internal.h"
#include "sd_launch.cuh"

namespace {

template <typename real>
__global__ void k_pack_elems(const real* __restrict__ U, const int* __restrict__ elems, int count, int nelem,
                             int nvar, int np, real* __restrict__ buf, int unpack) {
    const long long per_var = (long long)count * np;
    const long long total = per_var * nvar;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i / per_var);
        const long long r = i - v * per_var;
        const int k = (int)(r / np);
        const int pt = (int)(r - (long long)k * np);
        const int e = elems[k];
        if (e < 0 || e >= nelem) continue;          // lists are checked on the host; never touch outside
        const size_t at = ((size_t)v * nelem + e) * np + pt;
        // buf[v][k][pt]
        real* U_mut = const_cast<real*>(U);
        if (unpack) U_mut[at] = buf[i];
        else buf[i] = U[at];
    }
}

template <typename real>
__global__ void k_pack_faces(real* __restrict__ T, const int* __restrict__ elems, const int* __restrict__ faces,
                             int count, int nelem, int nface, int stride, real* __restrict__ buf, int unpack) {
    const long long total = (long long)count * stride;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / stride);
        const int w = (int)(i - (long long)k * stride);
        const int e = elems[k], f = faces[k];
        if (e < 0 || e >= nelem || f < 0 || f >= nface) continue;
        const size_t at = ((size_t)e * nface + f) * stride + w;
        if (unpack) T[at] = buf[i];
        else buf[i] = T[at];
    }
}

int blocks_for(long long total) {
    const long long b = (total + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), 148LL * 32);
}

sd_status pack_elements(sd_ctx* c, const void* U, int value_bytes, const int* elems, int count, void* buf,
                        int unpack) {
    if (!c || !U || !buf || (count > 0 && !elems) || count < 0 || (value_bytes != 4 && value_bytes != 8)) {
        sdi_set_error("bad argument");
        return SD_EINVAL;
    }
    if (count == 0) return SD_OK;
    const int np = (int)(c->npts / c->nelem);
    const long long total = (long long)count * np * c->nvar;
    sdi_prof_begin(c, SD_K_OTHER);
    // values are moved as raw 4- or 8-byte words
    if (value_bytes == 4)
        k_pack_elems<unsigned><<<blocks_for(total), 256, 0, c->stream>>>((const unsigned*)U, elems, count, c->nelem,
                                                                        c->nvar, np, (unsigned*)buf, unpack);
    else
        k_pack_elems<unsigned long long><<<blocks_for(total), 256, 0, c->stream>>>(
            (const unsigned long long*)U, elems, count, c->nelem, c->nvar, np, (unsigned long long*)buf, unpack);
    sdi_prof_end(c, SD_K_OTHER);
    if (cudaGetLastError() != cudaSuccess) { sdi_set_error("element pack launch failed"); return SD_ECUDA; }
    return SD_OK;
}

sd_status pack_faces(sd_ctx* c, const int* elems, const int* faces, int count, void* buf, int unpack) {
    if (!c || !buf || (count > 0 && (!elems || !faces)) || count < 0) { sdi_set_error("bad argument"); return SD_EINVAL; }
    if (c->curv) { sdi_set_error("sub-domains are available on Cartesian grids only"); return SD_EUNSUPPORTED; }
    if (count == 0) return SD_OK;
    const int nface = 2 * c->dim;
    const int stride = (int)(c->ntg / ((size_t)c->nelem * nface));
    const long long total = (long long)count * stride;
    sdi_prof_begin(c, SD_K_OTHER);
    if (c->prec == SD_F32)
        k_pack_faces<float><<<blocks_for(total), 256, 0, c->stream>>>((float*)c->Tg, elems, faces, count, c->nelem,
                                                                     nface, stride, (float*)buf, unpack);
    else
        k_pack_faces<double><<<blocks_for(total), 256, 0, c->stream>>>((double*)c->Tg, elems, faces, count,
                                                                       c->nelem, nface, stride, (double*)buf, unpack);
    sdi_prof_end(c, SD_K_OTHER);
    if (cudaGetLastError() != cudaSuccess) { sdi_set_error("face pack launch failed"); return SD_ECUDA; }
    return SD_OK;
}

}  // namespace

extern "C" sd_status sd_pack_elements(sd_ctx* c, const void* U, int value_bytes, const int* elems, int count,
                                      void* buf) {
    return pack_elements(c, U, value_bytes, elems, count, buf, 0);
}

extern "C" sd_status sd_unpack_elements(sd_ctx* c, const void* buf, int value_bytes, const int* elems, int count,
                                        void* U) {
    return pack_elements(c, U, value_bytes, elems, count, const_cast<void*>(buf), 1);
}

extern "C" size_t sd_face_gradient_size(const sd_ctx* c) {
    if (!c || c->curv) return 0;
    return c->ntg / ((size_t)c->nelem * 2 * c->dim);
}

extern "C" sd_status sd_pack_face_gradients(sd_ctx* c, const int* elems, const int* faces, int count, void* buf) {
    return pack_faces(c, elems, faces, count, buf, 0);
}

extern "C" sd_status sd_unpack_face_gradients(sd_ctx* c, const void* buf, const int* elems, const int* faces,
                                              int count) {
    return pack_faces(c, elems, faces, count, const_cast<void*>(buf), 1);
}

static sd_status phases(sd_ctx* c, const void* U, void* R, int first, int last) {
    for (int ph = first; ph <= last; ++ph) {
        sd_status s = c->prec == SD_F32
                          ? sdi_residual_phase_f32(c, (const float*)U, (float*)R, ph, 0, c->nelem, c->stream)
                          : sdi_residual_phase_f64(c, (const double*)U, (double*)R, ph, 0, c->nelem, c->stream);
        if (s != SD_OK) return s;
    }
    return SD_OK;
}

extern "C" sd_status sd_residual_begin(sd_ctx* c, const void* U) {
    if (!c || !U) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (c->curv) { sdi_set_error("the split residual is available on Cartesian grids only"); return SD_EUNSUPPORTED; }
    if (c->closure_on) { sdi_set_error("the split residual does not run the learned closure"); return SD_EUNSUPPORTED; }
    return phases(c, U, nullptr, SDI_PH_TRACE, SDI_PH_GRAD);
}

extern "C" sd_status sd_residual_end(sd_ctx* c, const void* U, void* R) {
    if (!c || !U || !R) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (c->curv) { sdi_set_error("the split residual is available on Cartesian grids only"); return SD_EUNSUPPORTED; }
    if (c->closure_on) { sdi_set_error("the split residual does not run the learned closure"); return SD_EUNSUPPORTED; }
    const char* a = (const char*)U;
    const char* b = (const char*)R;
    const size_t bytes = c->nstate * c->esize;
    if (a < b + bytes && b < a + bytes) { sdi_set_error("U and R overlap"); return SD_EINVAL; }
    return phases(c, U, R, SDI_PH_FACE, SDI_PH_FLUX);
}

extern "C" sd_status sd_set_owned_box(sd_ctx* c, const int* lo, const int* hi) {
    if (!c) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (!lo || !hi) {
        c->own_set = 0;
        return SD_OK;
    }
    for (int d = 0; d < 3; ++d) {
        const int l = d < c->dim ? lo[d] : 0, h = d < c->dim ? hi[d] : 1;
        if (l < 0 || h > c->ne[d] || l >= h) { sdi_set_error("owned box out of the grid along axis %d", d); return SD_EINVAL; }
        c->own_lo[d] = l;
        c->own_hi[d] = h;
    }
    c->own_set = 1;
    return SD_OK;
}
