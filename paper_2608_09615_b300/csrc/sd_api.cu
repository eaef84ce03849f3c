// C ABI of the SD residual library: context life cycle, the 1D operators, the residual
// entry points, Runge-Kutta steps and FP64 diagnostics. See include/sd.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "sd_internal.h"
#include "sd_launch.cuh"

// ------------------------------------------------------------------ error text
static thread_local char g_err[512] = "";

void sdi_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char* sd_last_error(void) { return g_err; }

extern "C" const char* sd_status_str(sd_status s) {
    switch (s) {
        case SD_OK: return "ok";
        case SD_EINVAL: return "invalid argument";
        case SD_ENOMEM: return "out of memory";
        case SD_ECUDA: return "CUDA error";
        case SD_EUNSUPPORTED: return "unsupported configuration";
        case SD_ENONFINITE: return "non-finite state";
        case SD_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            sdi_set_error("%s failed: %s", #call, cudaGetErrorString(e_));         \
            return SD_ECUDA;                                                       \
        }                                                                          \
    } while (0)

// ------------------------------------------------------------------ profiling
static void prof_fold(sd_ctx* c, int k) {
    if (c->prof_n[k] == 0) return;
    cudaEventSynchronize(c->prof_ev[k][2 * (c->prof_n[k] - 1) + 1]);
    for (int i = 0; i < c->prof_n[k]; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_ev[k][2 * i], c->prof_ev[k][2 * i + 1]) == cudaSuccess)
            c->prof_ms[k] += ms;
    }
    c->prof_count[k] += c->prof_n[k];
    c->prof_n[k] = 0;
}

void sdi_prof_begin(sd_ctx* c, int k) {
    c->launches++;
    if (!c->prof_on) return;
    if (c->prof_n[k] == SDI_PROF_CAP) prof_fold(c, k);
    cudaEventRecord(c->prof_ev[k][2 * c->prof_n[k]], c->stream);
}

void sdi_prof_end(sd_ctx* c, int k) {
    if (!c->prof_on) return;
    cudaEventRecord(c->prof_ev[k][2 * c->prof_n[k] + 1], c->stream);
    c->prof_n[k]++;
}

static void prof_destroy(sd_ctx* c) {
    for (int k = 0; k < SD_K_COUNT; ++k) {
        if (!c->prof_ev[k]) continue;
        for (int i = 0; i < 2 * SDI_PROF_CAP; ++i) cudaEventDestroy(c->prof_ev[k][i]);
        free(c->prof_ev[k]);
        c->prof_ev[k] = nullptr;
        c->prof_n[k] = 0;
    }
    c->prof_on = 0;
}

extern "C" sd_status sd_profile_enable(sd_ctx* c, int on) {
    if (!c) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (!on) { prof_destroy(c); return SD_OK; }
    if (c->prof_on) return SD_OK;
    for (int k = 0; k < SD_K_COUNT; ++k) {
        c->prof_ev[k] = (cudaEvent_t*)calloc(2 * SDI_PROF_CAP, sizeof(cudaEvent_t));
        if (!c->prof_ev[k]) { prof_destroy(c); return SD_ENOMEM; }
        for (int i = 0; i < 2 * SDI_PROF_CAP; ++i)
            if (cudaEventCreate(&c->prof_ev[k][i]) != cudaSuccess) {
                prof_destroy(c);
                sdi_set_error("cudaEventCreate failed");
                return SD_ECUDA;
            }
        c->prof_n[k] = 0;
        c->prof_ms[k] = 0.0;
        c->prof_count[k] = 0;
    }
    c->prof_on = 1;
    return SD_OK;
}

extern "C" sd_status sd_profile_read(sd_ctx* c, double* ms, long long* launches) {
    if (!c || !ms || !launches) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (!c->prof_on) { sdi_set_error("profiling is not enabled"); return SD_EINVAL; }
    for (int k = 0; k < SD_K_COUNT; ++k) {
        prof_fold(c, k);
        ms[k] = c->prof_ms[k];
        launches[k] = c->prof_count[k];
        c->prof_ms[k] = 0.0;
        c->prof_count[k] = 0;
    }
    return SD_OK;
}

extern "C" long long sd_launch_count(const sd_ctx* c) { return c ? c->launches : 0; }

// ------------------------------------------------------------------ 1D operators
// Gauss-Legendre nodes/weights by Newton iteration on the three-term recurrence of P_n.
// The operators are built in 80-bit long double and rounded once to double at the end.
typedef long double ldouble;

template <typename T>
static void gauss_legendre_t(int n, T* x, T* w) {
    const T pi = (T)3.14159265358979323846264338327950288L;
    for (int i = 0; i < n; ++i) {
        T z = cosl(pi * (i + (T)0.75) / (n + (T)0.5));
        for (int it = 0; it < 100; ++it) {
            T p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const T pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1; }
            const T dp = n * (z * p1 - p0) / (z * z - 1);
            const T dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < (T)1e-19) break;
        }
        T p0 = 1, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const T pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        if (n == 1) { p1 = z; p0 = 1; }
        const T dp = n * (z * p1 - p0) / (z * z - 1);
        x[n - 1 - i] = z;                       // ascending order
        w[n - 1 - i] = 2 / ((1 - z * z) * dp * dp);
    }
    if (n == 1) { x[0] = 0; w[0] = 2; }
}

static void gauss_legendre(int n, double* x, double* w) {
    ldouble xl[SD_MAX_N], wl[SD_MAX_N];
    gauss_legendre_t<ldouble>(n, xl, wl);
    for (int i = 0; i < n; ++i) {
        x[i] = (double)xl[i];
        w[i] = (double)wl[i];
    }
}

// l_j(x) on nodes t[0..m)
template <typename T>
static T lagrange_t(const T* t, int m, int j, T x) {
    T v = 1;
    for (int k = 0; k < m; ++k)
        if (k != j) v *= (x - t[k]) / (t[j] - t[k]);
    return v;
}

static double lagrange(const double* t, int m, int j, double x) { return lagrange_t<double>(t, m, j, x); }

// l_j'(x) = sum_{k != j} 1/(t_j - t_k) prod_{l != j,k} (x - t_l)/(t_j - t_l)
template <typename T>
static T lagrange_d_t(const T* t, int m, int j, T x) {
    T s = 0;
    for (int k = 0; k < m; ++k) {
        if (k == j) continue;
        T prod = 1 / (t[j] - t[k]);
        for (int l = 0; l < m; ++l)
            if (l != j && l != k) prod *= (x - t[l]) / (t[j] - t[l]);
        s += prod;
    }
    return s;
}

static void build_operators(sd_ctx* c) {
    const int n = c->n;
    ldouble xs[SD_MAX_N], ws[SD_MAX_N], xf[SD_MAX_N + 1], tmp[SD_MAX_N];
    ldouble L[(SD_MAX_N + 1) * SD_MAX_N], M[SD_MAX_N * (SD_MAX_N + 1)];
    gauss_legendre_t<ldouble>(n, xs, ws);
    xf[0] = -1;
    xf[n] = 1;
    if (n > 1) gauss_legendre_t<ldouble>(n - 1, xf + 1, tmp);
    for (int f = 0; f <= n; ++f)
        for (int i = 0; i < n; ++i) L[f * n + i] = lagrange_t<ldouble>(xs, n, i, xf[f]);
    for (int i = 0; i < n; ++i)
        for (int f = 0; f <= n; ++f) M[i * (n + 1) + f] = lagrange_d_t<ldouble>(xf, n + 1, f, xs[i]);
    ldouble D[SD_MAX_N * SD_MAX_N];
    for (int i = 0; i < n; ++i) {
        c->xs[i] = (double)xs[i];
        c->ws[i] = (double)ws[i];
        for (int j = 0; j < n; ++j) {
            ldouble s = 0;
            for (int f = 0; f <= n; ++f) s += M[i * (n + 1) + f] * L[f * n + j];
            D[i * n + j] = s;
            c->D[i * n + j] = (double)s;
        }
    }
    // products with L, used to evaluate the derivative along a line directly at the flux
    // points: L_f (D u + M[:,0] d_L + M[:,n] d_R) = (L D)_f u + (L M)_{f0} d_L + (L M)_{fn} d_R
    for (int f = 0; f <= n; ++f) {
        for (int i = 0; i < n; ++i) {
            ldouble s = 0;
            for (int j = 0; j < n; ++j) s += L[f * n + j] * D[j * n + i];
            c->LD[f * n + i] = (double)s;
        }
        ldouble s0 = 0, sn = 0;
        for (int j = 0; j < n; ++j) {
            s0 += L[f * n + j] * M[j * (n + 1) + 0];
            sn += L[f * n + j] * M[j * (n + 1) + n];
        }
        c->LM0[f] = (double)s0;
        c->LMN[f] = (double)sn;
    }
    for (int f = 0; f <= n; ++f) c->xf[f] = (double)xf[f];
    for (int k = 0; k < (n + 1) * n; ++k) c->L[k] = (double)L[k];
    for (int k = 0; k < n * (n + 1); ++k) c->M[k] = (double)M[k];
    ldouble a = 0, b = 0;
    for (int i = 0; i < n; ++i) {
        a += L[0 * n + i] * M[i * (n + 1) + n];
        b += L[n * n + i] * M[i * (n + 1) + 0];
    }
    c->alpha = (double)a;
    c->beta = (double)b;
}

void sdi_build_operators(sd_ctx* c) { build_operators(c); }

// ------------------------------------------------------------------ life cycle
static void free_closure(sd_ctx* c) {
    void* ptrs[] = {c->cl_X, c->cl_Xb, c->cl_Y, c->cl_H, c->cl_tau};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c->cl_X = nullptr;
    c->cl_Xb = nullptr;
    c->cl_Y = nullptr;
    c->cl_H = nullptr;
    c->cl_tau = nullptr;
    c->closure_on = 0;
    if (c->tau == c->cl_tau) c->tau = nullptr;
}

static void free_all(sd_ctx* c) {
    free_closure(c);
    if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
    if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    for (int k = 0; k < SDI_MAX_SLABS; ++k) {
        if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
        if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
    }
    if (c->cl_tmode) cudaFree(c->cl_tmode);
    void* ptrs[] = {c->Tu, c->Tg, c->Fh, c->S, c->K, c->rA, c->rB, c->rC, c->rX, c->rA64, c->rB64, c->rC64, c->dW,
                    c->partial, c->partial2, c->dsum, c->hU, c->hR, c->cih, c->cvs, c->cTg, c->cgeo64};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->cgeo && c->cgeo != (void*)c->cgeo64) cudaFree(c->cgeo);
    if (c->Tu64 && (void*)c->Tu64 != c->Tu) cudaFree(c->Tu64);
}

static int ipow_h(int b, int e) {
    int r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// Validate a problem description and fill the context's problem fields, operators and
// scratch sizes (no CUDA call, no allocation). Shared by sd_init and the allocation-free
// entry point, so both accept exactly the same problems.
sd_status sdi_setup(const sd_mesh* mesh, int p, sd_scheme scheme, const sd_physics* phys, sd_precision prec,
                    void* stream, sd_ctx* c) {
    if (!mesh || !phys) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (mesh->dim != 1 && mesh->dim != 3) { sdi_set_error("dim must be 1 or 3"); return SD_EUNSUPPORTED; }
    if (p < 1 || p > SD_MAX_N - 1) { sdi_set_error("p must be in 1..%d", SD_MAX_N - 1); return SD_EUNSUPPORTED; }
    if (scheme != SD_BR1 && scheme != SD_COMPACT) { sdi_set_error("bad scheme"); return SD_EINVAL; }
    if (prec != SD_F32 && prec != SD_F64) { sdi_set_error("bad precision"); return SD_EINVAL; }
    if (phys->kind != SD_HEAT && phys->kind != SD_PME && phys->kind != SD_NS) {
        sdi_set_error("bad physics kind");
        return SD_EINVAL;
    }
    if (phys->kind == SD_NS && mesh->dim != 3) { sdi_set_error("Navier-Stokes needs dim = 3"); return SD_EUNSUPPORTED; }
    if (phys->kind == SD_NS) {
        if (!(phys->gamma > 1.0) || !(phys->Pr > 0.0) || !(phys->Re > 0.0) || !(phys->Ma > 0.0) ||
            !(phys->rho0 > 0.0) || !(phys->u0 > 0.0) || !(phys->L > 0.0) || phys->harten < 0.0 ||
            (phys->riemann != SD_ROE && phys->riemann != SD_RUSANOV)) {
            sdi_set_error("bad Navier-Stokes parameters");
            return SD_EINVAL;
        }
    }
    if (phys->kind == SD_PME && !(phys->m_pme >= 1.0)) { sdi_set_error("m_pme must be >= 1"); return SD_EINVAL; }
    if (!(phys->eta_ip >= 0.0)) { sdi_set_error("eta_ip must be >= 0"); return SD_EINVAL; }
    if (phys->viscous_flux != SD_VISC_STATE_AVG && phys->viscous_flux != SD_VISC_FLUX_AVG) {
        sdi_set_error("bad viscous_flux");
        return SD_EINVAL;
    }
    if (phys->pme_coef != SD_PME_COEF_FLUX && phys->pme_coef != SD_PME_COEF_SOLUTION) {
        sdi_set_error("bad pme_coef");
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
    c->prec = prec;
    c->stream = (cudaStream_t)stream;
    c->J = 1.0;
    for (int d = 0; d < c->dim; ++d) c->J *= c->h[d] / 2.0;
    build_operators(c);
    const int np = ipow_h(c->n, c->dim), nq = ipow_h(c->n, c->dim - 1);
    c->npts = (size_t)c->nelem * np;
    c->nstate = c->npts * c->nvar;
    // face blocks padded to a multiple of 4 values (16-byte aligned, copied in 16-byte pieces)
    // (scalar trace blocks also hold the traces of the porous-medium diffusivity)
    const size_t fst = ((size_t)c->nvar * nq + (c->nvar == 1 ? nq : 0) + 3) / 4 * 4;
    const size_t gst = ((size_t)c->ngrad * nq + 3) / 4 * 4;
    c->ntu = (size_t)c->nelem * 2 * c->dim * fst;
    c->ntg = (size_t)c->nelem * 2 * c->dim * gst;
    c->nfh = (size_t)c->nelem * c->dim * fst;
    c->esize = prec == SD_F32 ? sizeof(float) : sizeof(double);

    // shared memory feasibility of the element-staged kernels (line layout of sd_line.cuh:
    // per element u, two trace sets, v^S and the neighbour interface gradients)
    {
        const int n = c->n, NV = c->nvar, DIM = c->dim;
        const size_t per = (size_t)(NV * np + 2 * 2 * DIM * NV * nq + NV * DIM * np + 2 * DIM * c->ngrad * nq);
        const int nqv = nq, epw = nqv <= 32 ? 32 / nqv : 1, wpd = nqv <= 32 ? 1 : (nqv + 31) / 32;
        const int unit = DIM * wpd * 32, upb = unit >= SD_LINE_THREADS ? 1 : SD_LINE_THREADS / unit;
        const size_t blk = per * (size_t)(upb * epw) * c->esize;
        const size_t diag = (size_t)(NV * np + 2 * 2 * DIM * NV * nq + NV * DIM * np) * sizeof(double);
        if (blk > 227 * 1024 || diag > 227 * 1024) {
            sdi_set_error("n = %d needs %zu bytes of shared memory per block", n, blk);
            return SD_EUNSUPPORTED;
        }
    }
    return SD_OK;
}

extern "C" sd_status sd_init(const sd_mesh* mesh, int p, sd_scheme scheme, const sd_physics* phys,
                             sd_precision prec, void* stream, sd_ctx** out) {
    g_err[0] = 0;
    if (!mesh || !phys || !out) { sdi_set_error("null argument"); return SD_EINVAL; }
    *out = nullptr;
    sd_ctx* c = (sd_ctx*)calloc(1, sizeof(sd_ctx));
    if (!c) return SD_ENOMEM;
    {
        const sd_status st = sdi_setup(mesh, p, scheme, phys, prec, stream, c);
        if (st != SD_OK) {
            free(c);
            return st;
        }
    }
    const int np = ipow_h(c->n, c->dim);
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        sdi_set_error("no CUDA device");
        free(c);
        return SD_ECUDA;
    }
    const size_t S = c->nstate;
    bool ok = true;
    auto alloc = [&](void** p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) ok = false;
    };
    alloc(&c->Tu, c->ntu * c->esize);
    alloc(&c->Tg, c->ntg * c->esize);
    alloc(&c->Fh, c->nfh * c->esize);
    if (prec == SD_F64) c->Tu64 = (double*)c->Tu;
    else alloc((void**)&c->Tu64, c->ntu * sizeof(double));
    alloc(&c->S, S * c->esize);
    alloc(&c->K, S * c->esize);
    alloc(&c->rA, S * c->esize);
    alloc(&c->rB, S * c->esize);
    if (prec == SD_F64) alloc(&c->rC, S * c->esize);           // FP32 increments need two registers
    if (prec == SD_F32) alloc(&c->rX, S * c->esize);
    alloc((void**)&c->dW, SD_MAX_N * sizeof(double));
    alloc((void**)&c->cl_tmode, (SD_MAX_N * SD_MAX_N + SD_MAX_N) * sizeof(double));
    const int tpe = ((np + 31) / 32) * 32;
    const int epb = std::max(1, 256 / tpe);
    c->diag_blocks = (c->nelem + epb - 1) / epb;
    alloc((void**)&c->partial, (size_t)c->diag_blocks * sdk::NDIAG * sizeof(double));
    alloc((void**)&c->dsum, sdk::NDIAG * sizeof(double));
    alloc((void**)&c->partial2, sdk::DIAG_L1 * sdk::NDIAG * sizeof(double));
    alloc(&c->hU, S * c->esize);
    alloc(&c->hR, S * c->esize);
    if (ok && c->dim == 3) {
        // streams and events of the slab-pipelined host-buffer residual
        ok = cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
             cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < SDI_MAX_SLABS; ++k)
            ok = cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        sdi_set_error("device allocation of the context scratch failed");
        free_all(c);
        free(c);
        return SD_ENOMEM;
    }
    if (sdi_upload_f32(c) != SD_OK || sdi_upload_f64(c) != SD_OK) {
        free_all(c);
        free(c);
        return SD_ECUDA;
    }
    {
        // Legendre modal transform T[m][i] = w_i P_m(x_i) (2m+1)/2 followed by the points x_i
        double tm[SD_MAX_N * SD_MAX_N + SD_MAX_N];
        const int n = c->n;
        for (int i = 0; i < n; ++i) {
            double p0 = 1.0, p1 = c->xs[i];
            for (int m = 0; m < n; ++m) {
                double pm;
                if (m == 0) pm = 1.0;
                else if (m == 1) pm = c->xs[i];
                else {
                    const double pk = ((2.0 * m - 1.0) * c->xs[i] * p1 - (m - 1.0) * p0) / m;
                    p0 = p1;
                    p1 = pk;
                    pm = pk;
                }
                tm[m * n + i] = c->ws[i] * pm * (2.0 * m + 1.0) / 2.0;
            }
            tm[n * n + i] = c->xs[i];
        }
        if (cudaMemcpy(c->cl_tmode, tm, (n * n + n) * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            sdi_set_error("cudaMemcpy of the modal transform failed");
            free_all(c);
            free(c);
            return SD_ECUDA;
        }
    }
    if (cudaMemcpy(c->dW, c->ws, c->n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        sdi_set_error("cudaMemcpy of the Gauss weights failed");
        free_all(c);
        free(c);
        return SD_ECUDA;
    }
    *out = c;
    return SD_OK;
}

extern "C" void sd_destroy(sd_ctx* c) {
    if (!c) return;
    prof_destroy(c);
    free_all(c);
    free(c);
}

extern "C" sd_status sd_init_curvilinear(const sd_mesh* mesh, const double* nodes, int p, sd_scheme scheme,
                                         const sd_physics* phys, sd_precision prec, void* stream, sd_ctx** out) {
    g_err[0] = 0;
    if (!mesh || !nodes || !phys || !out) { sdi_set_error("null argument"); return SD_EINVAL; }
    *out = nullptr;
    if (mesh->dim != 3) { sdi_set_error("curvilinear grids are 3D"); return SD_EUNSUPPORTED; }
    if (phys->kind == SD_PME && phys->pme_coef == SD_PME_COEF_SOLUTION) {
        sdi_set_error("the solution-point diffusivity variant is available on Cartesian grids only");
        return SD_EUNSUPPORTED;
    }
    for (int d = 0; d < 3; ++d)
        if (mesh->ne[d] < 1) { sdi_set_error("ne[%d] must be >= 1", d); return SD_EINVAL; }
    // the Cartesian box fields are not used on a curved grid: give the context a unit box
    sd_mesh m = *mesh;
    for (int d = 0; d < 3; ++d) {
        m.lo[d] = 0.0;
        m.hi[d] = 1.0;
    }
    sd_ctx* c = nullptr;
    sd_status s = sd_init(&m, p, scheme, phys, prec, stream, &c);
    if (s != SD_OK) return s;
    s = sdi_curv_setup(c, nodes);
    if (s != SD_OK) {
        sd_destroy(c);
        return s;
    }
    *out = c;
    return SD_OK;
}

extern "C" int sd_is_curvilinear(const sd_ctx* c) { return c ? c->curv : 0; }

extern "C" sd_status sd_set_stream(sd_ctx* c, void* stream) {
    if (!c) return SD_EINVAL;
    c->stream = (cudaStream_t)stream;
    return SD_OK;
}

extern "C" size_t sd_state_size(const sd_ctx* c) { return c ? c->nstate : 0; }
extern "C" int sd_nvar(const sd_ctx* c) { return c ? c->nvar : 0; }

extern "C" sd_status sd_points(const sd_ctx* c, double* xi, double* w) {
    if (!c || !xi || !w) return SD_EINVAL;
    for (int i = 0; i < c->n; ++i) {
        xi[i] = c->xs[i];
        w[i] = c->ws[i];
    }
    return SD_OK;
}

// ------------------------------------------------------------------ residual
static bool overlap(const void* a, const void* b, size_t bytes) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + bytes && y < x + bytes;
}

static sd_status residual_any(sd_ctx* c, const void* U, void* R, int offset_in = 0) {
    if (c->curv) {
        if (c->prec == SD_F32) return sdi_curv_residual_f32(c, (const float*)U, (float*)R, offset_in);
        return sdi_curv_residual_f64(c, (const double*)U, (double*)R, offset_in);
    }
    if (c->prec == SD_F32) return sdi_residual_f32(c, (const float*)U, (float*)R, offset_in);
    return sdi_residual_f64(c, (const double*)U, (double*)R, offset_in);
}

extern "C" sd_status sd_residual(sd_ctx* c, const void* U, void* R) {
    if (!c || !U || !R) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (overlap(U, R, c->nstate * c->esize)) { sdi_set_error("U and R overlap"); return SD_EINVAL; }
    return residual_any(c, U, R);
}

static sd_status residual_phase_any(sd_ctx* c, int phase, int e0, int e1) {
    if (c->prec == SD_F32)
        return sdi_residual_phase_f32(c, (const float*)c->hU, (float*)c->hR, phase, e0, e1, c->stream);
    return sdi_residual_phase_f64(c, (const double*)c->hU, (double*)c->hR, phase, e0, e1, c->stream);
}

// Host-buffer residual in z-slabs: the copies of U run on their own stream, slab by slab,
// and each residual phase of a slab starts as soon as the slabs it reads are in (its own
// and its z neighbours'); R goes back slab by slab on a third stream as each slab's flux
// phase ends. Phases of one slab: trace <- copy in; grad <- trace of slabs k-1, k, k+1;
// face <- grad of k, k+1 (+z faces); flux <- face of k-1, k. The slabs are copied in the
// order S-1, 0, 1, ..., S-2, so slab 0's periodic neighbour arrives first. The flux phases
// of slabs S-3, S-2, S-1 and 0 need the last slab copied in (through grad of S-2 and the
// periodic wrap), so their results are the ones still to go back when the copies in end:
// with at least two layers per slab to spare those four slabs are one element layer
// thick and the others share the rest.
static sd_status residual_host_slabs(sd_ctx* c, const void* U_host, void* R_host) {
    const int S = std::min(c->ne[2], SDI_MAX_SLABS);
    const int layer = c->ne[0] * c->ne[1];
    const size_t ppe = c->npts / c->nelem;
    int lay[SDI_MAX_SLABS + 1];                  // first element layer of each slab
    const bool thin = S >= 8 && c->ne[2] >= 2 * S;
    lay[0] = 0;
    for (int k = 0; k < S; ++k) {
        int n;
        if (!thin) n = (int)((long long)(k + 1) * c->ne[2] / S - (long long)k * c->ne[2] / S);
        else if (k == 0 || k >= S - 3) n = 1;
        else n = (c->ne[2] - 4) * k / (S - 4) - (c->ne[2] - 4) * (k - 1) / (S - 4);
        lay[k + 1] = lay[k] + n;
    }
    auto first = [&](int k) { return lay[k] * layer; };
    auto copy_slab = [&](int k, bool in) -> cudaError_t {
        const size_t e0 = first(k), e1 = first(k + 1);
        const size_t bytes = (e1 - e0) * ppe * c->esize;
        for (int v = 0; v < c->nvar; ++v) {
            const size_t off = ((size_t)v * c->nelem + e0) * ppe * c->esize;
            const cudaError_t e = in ? cudaMemcpyAsync((char*)c->hU + off, (const char*)U_host + off, bytes,
                                                       cudaMemcpyHostToDevice, c->s_h2d)
                                     : cudaMemcpyAsync((char*)R_host + off, (const char*)c->hR + off, bytes,
                                                       cudaMemcpyDeviceToHost, c->s_d2h);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    // the copies start after everything already queued on the context stream
    CK(cudaEventRecord(c->ev_start, c->stream));
    CK(cudaStreamWaitEvent(c->s_h2d, c->ev_start, 0));
    for (int a = 0; a < S; ++a) {
        const int k = (a + S - 1) % S;
        CK(copy_slab(k, true));
        CK(cudaEventRecord(c->ev_in[k], c->s_h2d));
    }
    bool tr[SDI_MAX_SLABS] = {false}, gr[SDI_MAX_SLABS] = {false}, fa[SDI_MAX_SLABS] = {false},
         fl[SDI_MAX_SLABS] = {false};
    auto m = [&](int k) { return (k + S) % S; };
    sd_status st;
    for (int a = 0; a < S; ++a) {
        const int k = (a + S - 1) % S;
        CK(cudaStreamWaitEvent(c->stream, c->ev_in[k], 0));
        if ((st = residual_phase_any(c, SDI_PH_TRACE, first(k), first(k + 1))) != SD_OK) return st;
        tr[k] = true;
        for (bool progress = true; progress;) {
            progress = false;
            for (int j = 0; j < S; ++j) {
                if (!gr[j] && tr[m(j - 1)] && tr[j] && tr[m(j + 1)]) {
                    if ((st = residual_phase_any(c, SDI_PH_GRAD, first(j), first(j + 1))) != SD_OK) return st;
                    gr[j] = progress = true;
                }
                if (!fa[j] && gr[j] && gr[m(j + 1)]) {
                    if ((st = residual_phase_any(c, SDI_PH_FACE, first(j), first(j + 1))) != SD_OK) return st;
                    fa[j] = progress = true;
                }
                if (!fl[j] && fa[j] && fa[m(j - 1)]) {
                    if ((st = residual_phase_any(c, SDI_PH_FLUX, first(j), first(j + 1))) != SD_OK) return st;
                    fl[j] = progress = true;
                    CK(cudaEventRecord(c->ev_out[j], c->stream));
                    CK(cudaStreamWaitEvent(c->s_d2h, c->ev_out[j], 0));
                    CK(copy_slab(j, false));
                }
            }
        }
    }
    for (int j = 0; j < S; ++j)
        if (!fl[j]) { sdi_set_error("slab schedule incomplete"); return SD_ECUDA; }
    CK(cudaStreamSynchronize(c->s_d2h));
    CK(cudaStreamSynchronize(c->stream));
    return SD_OK;
}

extern "C" sd_status sd_residual_host(sd_ctx* c, const void* U_host, void* R_host) {
    if (!c || !U_host || !R_host) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (c->s_h2d && !c->closure_on && !c->curv && c->ne[2] >= 4) return residual_host_slabs(c, U_host, R_host);
    const size_t bytes = c->nstate * c->esize;
    CK(cudaMemcpyAsync(c->hU, U_host, bytes, cudaMemcpyHostToDevice, c->stream));
    const sd_status st = residual_any(c, c->hU, c->hR);
    if (st != SD_OK) return st;
    CK(cudaMemcpyAsync(R_host, c->hR, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SD_OK;
}

// ------------------------------------------------------------------ Runge-Kutta
static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)std::min<size_t>(std::max<size_t>(b, 1), 148 * 16);
}

// ------------------------------------------------------------------ Runge-Kutta kernels, FP32 residual
// Each thread handles EWB values spaced one grid apart per iteration; all loads of an
// iteration are issued before any arithmetic, so every thread keeps several independent
// requests in flight (these kernels are bound by HBM bandwidth).
namespace sdk {
constexpr int EWB = 4;

__global__ void k_ssp_inc(int k, double* __restrict__ U, float* __restrict__ A, float* __restrict__ B,
                          const float* __restrict__ K, const float* __restrict__ X, float* __restrict__ S,
                          SSPInc c, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += EWB * stride) {
        float kk[EWB], x[EWB], a[EWB], b[EWB];
        double u[EWB];
#pragma unroll
        for (int w = 0; w < EWB; ++w) {
            const size_t i = base + w * stride;
            a[w] = b[w] = x[w] = 0.0f;
            u[w] = 0.0;
            if (i >= n) continue;
            kk[w] = K[i];
            if (k < 4) x[w] = X[i];
            if (k == 2 || k == 3) b[w] = B[i];          // stage 1 only writes B
            if (k == 1 || k >= 3) a[w] = A[i];
            if (k == 4) u[w] = U[i];
        }
#pragma unroll
        for (int w = 0; w < EWB; ++w) {
            const size_t i = base + w * stride;
            if (i >= n) continue;
            const float s = ssp_inc_point(c, k, kk[w], x[w], a[w], b[w], u[w]);
            if (k == 4) {
                U[i] = u[w];
                continue;
            }
            S[i] = s;
            if (k == 1) B[i] = b[w];
            else A[i] = a[w];
        }
    }
}

__global__ void k_rk4_inc(int k, double* __restrict__ U, float* __restrict__ A, const float* __restrict__ K,
                          const float* __restrict__ X, float* __restrict__ S, RK4Inc c, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += EWB * stride) {
        float kk[EWB], x[EWB], a[EWB];
        double u[EWB];
#pragma unroll
        for (int w = 0; w < EWB; ++w) {
            const size_t i = base + w * stride;
            if (i >= n) continue;
            kk[w] = K[i];
            if (k < 3) x[w] = X[i];
            if (k > 0) a[w] = A[i];
            if (k == 3) u[w] = U[i];
        }
#pragma unroll
        for (int w = 0; w < EWB; ++w) {
            const size_t i = base + w * stride;
            if (i >= n) continue;
            if (k == 0) {
                A[i] = c.h6 * kk[w];
                S[i] = fmaf(c.h2, kk[w], x[w]);
            } else if (k == 1) {
                A[i] = fmaf(c.h3, kk[w], a[w]);
                S[i] = fmaf(c.h2, kk[w], x[w]);
            } else if (k == 2) {
                A[i] = fmaf(c.h3, kk[w], a[w]);
                S[i] = fmaf(c.h1, kk[w], x[w]);
            } else {
                U[i] = u[w] + (double)fmaf(c.h6, kk[w], a[w]);
            }
        }
    }
}

__global__ void k_lsrk_inc(int k, int last, double* __restrict__ U, float* __restrict__ W,
                           float* __restrict__ D, const float* __restrict__ K, const float* __restrict__ X,
                           float* __restrict__ S, float a, float dt, float b, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += EWB * stride) {
        float kk[EWB], x[EWB], w0[EWB], d0[EWB];
        double u[EWB];
#pragma unroll
        for (int w = 0; w < EWB; ++w) {
            const size_t i = base + w * stride;
            if (i >= n) continue;
            kk[w] = K[i];
            w0[w] = k > 0 ? W[i] : 0.0f;
            d0[w] = k > 0 ? D[i] : 0.0f;
            if (last) u[w] = U[i];
            else x[w] = X[i];
        }
#pragma unroll
        for (int w = 0; w < EWB; ++w) {
            const size_t i = base + w * stride;
            if (i >= n) continue;
            const float wn = fmaf(a, w0[w], dt * kk[w]);
            const float dn = fmaf(b, wn, d0[w]);
            if (last) {
                U[i] = u[w] + (double)dn;
            } else {
                W[i] = wn;
                D[i] = dn;
                S[i] = x[w] + dn;
            }
        }
    }
}
}  // namespace sdk


// Shu-Osher coefficients of SSPRK(5,4) (Spiteri & Ruuth 2002)
static const sdk::SSPCoef kSSP = {0.391752226571890, 0.444370493651235, 0.555629506348765,
                                  0.368410593050371, 0.620101851488403, 0.379898148511597,
                                  0.251891774271694, 0.178079954393132, 0.821920045606868,
                                  0.544974750228521, 0.517231671970585, 0.096059710526147,
                                  0.063692468666290, 0.386708617503269, 0.226007483236906};
// Carpenter & Kennedy (1994) LSRK(5,4) coefficients
static const double kLSA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double kLSB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};

// Runge-Kutta steps, stage by stage. Three forms of the stage arithmetic:
//   FP64 contexts: full FP64 stage states (the parity build);
//   FP32 contexts, SD_RK_STAGES_F32: FP32 stage increments d_j, the state U updated in FP64
//     once per step; the stage input is X + d_j with X = U - offsets rounded once per step;
//   FP32 contexts, SD_RK_STAGES_F64: FP64 stage states and registers, FP32 residual of each
//     stage state (offsets removed in FP64, then rounded).
// rk_prepare writes the first stage input from U; rk_stage(k) evaluates the residual of
// stage k's input and applies the stage-k update, which writes the next stage input (or, at
// the last stage, U). stage_input(k) is the array the residual of stage k reads.
static bool inc_mode(const sd_ctx* c) { return c->prec == SD_F32 && c->rk_stages == SD_RK_STAGES_F32; }

static void* stage_input(sd_ctx* c, int k) { return inc_mode(c) && k == 0 ? c->rX : c->S; }

static int rk_stages_of(sd_rk rk) { return rk == SD_RK4 ? 4 : 5; }

static sd_status rk_prepare(sd_ctx* c, double* U) {
    const size_t n = c->nstate;
    sdk::StageOff so;
    so.npts = c->npts;
    sdk::stage_offsets(c, so.off0, so.off4);
    sdi_prof_begin(c, SD_K_OTHER);
    if (c->prec == SD_F64) sdk::k_to_real<double><<<grid_for(n), 256, 0, c->stream>>>(U, (double*)c->S, n, so);
    else sdk::k_to_real<float><<<grid_for(n), 256, 0, c->stream>>>(U, (float*)stage_input(c, 0), n, so);
    sdi_prof_end(c, SD_K_OTHER);
    CK(cudaGetLastError());
    return SD_OK;
}

static sd_status rk_stage(sd_ctx* c, double* U, int k, double dt, sd_rk rk) {
    const size_t n = c->nstate;
    cudaStream_t st = c->stream;
    sd_status s = residual_any(c, stage_input(c, k), c->K, 1);
    if (s != SD_OK) return s;
    sdk::StageOff so;
    so.npts = c->npts;
    sdk::stage_offsets(c, so.off0, so.off4);
    const int gb = grid_for(n);
    sdi_prof_begin(c, SD_K_OTHER);
    if (c->prec == SD_F64) {
        double* S = (double*)c->S;
        double* K = (double*)c->K;
        double *rA = (double*)c->rA, *rB = (double*)c->rB, *rC = (double*)c->rC;
        if (rk == SD_RK4) sdk::k_rk4<double><<<gb, 256, 0, st>>>(k, U, rA, K, S, dt, n, so);
        else if (rk == SD_SSPRK54) sdk::k_ssp<double><<<gb, 256, 0, st>>>(k, U, rA, rB, rC, K, S, dt, kSSP, n, so);
        else sdk::k_lsrk<double><<<gb, 256, 0, st>>>(U, rA, K, S, kLSA[k], kLSB[k], dt, n, so);
    } else if (!inc_mode(c)) {
        float* S = (float*)c->S;
        float* K = (float*)c->K;
        double *rA = c->rA64, *rB = c->rB64, *rC = c->rC64;
        if (rk == SD_RK4) sdk::k_rk4<float><<<gb, 256, 0, st>>>(k, U, rA, K, S, dt, n, so);
        else if (rk == SD_SSPRK54) sdk::k_ssp<float><<<gb, 256, 0, st>>>(k, U, rA, rB, rC, K, S, dt, kSSP, n, so);
        else sdk::k_lsrk<float><<<gb, 256, 0, st>>>(U, rA, K, S, kLSA[k], kLSB[k], dt, n, so);
    } else {
        float* S = (float*)c->S;
        float* K = (float*)c->K;
        float* X = (float*)c->rX;
        float *rA = (float*)c->rA, *rB = (float*)c->rB;
        const int gi = grid_for((n + sdk::EWB - 1) / sdk::EWB);
        const sdk::SSPCoef& a = kSSP;
        const sdk::SSPInc ci = {(float)(a.a10 * dt), (float)a.a21, (float)(a.b21 * dt), (float)a.a32,
                                (float)(a.b32 * dt), (float)a.a43, (float)(a.b43 * dt), (float)a.a52,
                                (float)a.a53, (float)(a.b53 * dt), (float)a.a54, (float)(a.b54 * dt)};
        const sdk::RK4Inc c4 = {(float)(0.5 * dt), (float)dt, (float)(dt / 6.0), (float)(dt / 3.0)};
        if (rk == SD_RK4)
            sdk::k_rk4_inc<<<gi, 256, 0, st>>>(k, U, rA, K, X, S, c4, n);
        else if (rk == SD_SSPRK54)
            sdk::k_ssp_inc<<<gi, 256, 0, st>>>(k, U, rA, rB, K, X, S, ci, n);
        else
            sdk::k_lsrk_inc<<<gi, 256, 0, st>>>(k, k == 4, U, rA, rB, K, X, S, (float)kLSA[k], (float)dt,
                                                (float)kLSB[k], n);
    }
    sdi_prof_end(c, SD_K_OTHER);
    CK(cudaGetLastError());
    return SD_OK;
}

static sd_status rk_check(sd_ctx* c, double* U64, double dt, sd_rk rk) {
    if (!c || !U64) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (!(dt > 0.0) || !isfinite(dt)) { sdi_set_error("dt must be positive and finite"); return SD_EINVAL; }
    if (rk != SD_RK4 && rk != SD_SSPRK54 && rk != SD_LSRK54) {
        sdi_set_error("bad Runge-Kutta scheme");
        return SD_EINVAL;
    }
    return SD_OK;
}

extern "C" sd_status sd_rk_step(sd_ctx* c, double* U64, double t, double dt, sd_rk rk) {
    (void)t;
    sd_status s = rk_check(c, U64, dt, rk);
    if (s != SD_OK) return s;
    if ((s = rk_prepare(c, U64)) != SD_OK) return s;
    for (int k = 0; k < rk_stages_of(rk); ++k)
        if ((s = rk_stage(c, U64, k, dt, rk)) != SD_OK) return s;
    return SD_OK;
}

extern "C" sd_status sd_rk_prepare(sd_ctx* c, double* U64, void** input) {
    if (!c || !U64 || !input) { sdi_set_error("null argument"); return SD_EINVAL; }
    const sd_status s = rk_prepare(c, U64);
    if (s == SD_OK) *input = stage_input(c, 0);
    return s;
}

extern "C" sd_status sd_rk_stage(sd_ctx* c, double* U64, int k, double dt, sd_rk rk, void** input) {
    sd_status s = rk_check(c, U64, dt, rk);
    if (s != SD_OK) return s;
    if (!input) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (k < 0 || k >= rk_stages_of(rk)) { sdi_set_error("stage %d out of range", k); return SD_EINVAL; }
    if ((s = rk_stage(c, U64, k, dt, rk)) != SD_OK) return s;
    *input = k + 1 < rk_stages_of(rk) ? stage_input(c, k + 1) : nullptr;
    return SD_OK;
}

extern "C" sd_status sd_set_rk_stages(sd_ctx* c, sd_rk_stages mode) {
    if (!c) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (mode != SD_RK_STAGES_F32 && mode != SD_RK_STAGES_F64) { sdi_set_error("bad stage mode"); return SD_EINVAL; }
    if (c->prec == SD_F64) {
        // FP64 contexts always keep FP64 stage states
        if (mode != SD_RK_STAGES_F64) {
            sdi_set_error("FP64 contexts keep FP64 stage states");
            return SD_EUNSUPPORTED;
        }
        return SD_OK;
    }
    if (mode == SD_RK_STAGES_F64 && !c->rA64) {
        // the three FP64 registers, allocated once on first use
        const size_t bytes = c->nstate * sizeof(double);
        if (cudaMalloc((void**)&c->rA64, bytes) != cudaSuccess || cudaMalloc((void**)&c->rB64, bytes) != cudaSuccess ||
            cudaMalloc((void**)&c->rC64, bytes) != cudaSuccess) {
            cudaGetLastError();
            if (c->rA64) cudaFree(c->rA64);
            if (c->rB64) cudaFree(c->rB64);
            c->rA64 = c->rB64 = c->rC64 = nullptr;
            sdi_set_error("device allocation of the FP64 stage registers failed");
            return SD_ENOMEM;
        }
    }
    c->rk_stages = mode;
    return SD_OK;
}

// ------------------------------------------------------------------ diagnostics
namespace sdk {
// two-level reduction of the block partials, in a fixed order (deterministic): block j of
// the first level sums partials [j chunk, (j + 1) chunk); one block then sums those

__global__ void k_diag_reduce(const double* __restrict__ partial, int nblocks, int chunk,
                              double* __restrict__ out) {
    __shared__ double red[NDIAG][256];
    const int b0 = blockIdx.x * chunk, b1 = min(nblocks, b0 + chunk);
    for (int k = 0; k < NDIAG; ++k) {
        double s = 0.0;
        for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) s += partial[(size_t)b * NDIAG + k];
        red[k][threadIdx.x] = s;
    }
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int k = 0; k < NDIAG; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NDIAG; ++k) out[(size_t)blockIdx.x * NDIAG + k] = red[k][0];
}

__global__ void k_diag_final(const double* __restrict__ partial, int nblocks,
                             double* __restrict__ out) {
    __shared__ double red[NDIAG][256];
    for (int k = 0; k < NDIAG; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)b * NDIAG + k];
        red[k][threadIdx.x] = s;
    }
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int k = 0; k < NDIAG; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NDIAG; ++k) out[k] = red[k][0];
}

// two-level deterministic reduction of the nb rows of diagnostics partial sums
static sd_status diag_reduce(sd_ctx* c, int nb) {
    const int chunk = (nb + DIAG_L1 - 1) / DIAG_L1;
    const int nb1 = (nb + chunk - 1) / chunk;
    sdi_prof_begin(c, SD_K_OTHER);
    k_diag_reduce<<<nb1, 256, 0, c->stream>>>(c->partial, nb, chunk, c->partial2);
    sdi_prof_end(c, SD_K_OTHER);
    sdi_prof_begin(c, SD_K_OTHER);
    k_diag_final<<<1, 256, 0, c->stream>>>(c->partial2, nb1, c->dsum);
    sdi_prof_end(c, SD_K_OTHER);
    CK(cudaGetLastError());
    return SD_OK;
}

// FP64 contexts stage the state in FP64; FP32 contexts stage (U - offsets) in FP32 and form the
// kinetic-energy and enstrophy integrands in FP32 (their sums, and the conserved totals taken
// from U itself, stay FP64)
template <typename real, int N, int DIM, int NV>
static sd_status diag_impl_r(sd_ctx* c, const double* U, real* Tu) {
    using FP = Footprint<N, DIM, NV>;
    const Ops<real, N> ops = make_ops<real, N>(c);
    const Mesh g = make_mesh(c);
    double off0 = 0.0, off4 = 0.0;
    if (sizeof(real) == 4) stage_offsets(c, off0, off4);
    const long long ntr = (long long)g.nelem * DIM * NV * FP::NQ;       // one thread per line
    sdi_prof_begin(c, SD_K_OTHER);
    k_trace_staged<real, N, DIM, NV><<<trace_blocks(ntr), 256, 0, c->stream>>>(U, Tu, ops, g, off0, off4);
    sdi_prof_end(c, SD_K_OTHER);
    const int epb = std::max(1, 256 / FP::TPE);
    const int threads = epb * FP::TPE;
    const size_t smem = std::max<size_t>(epb * FP::grad * sizeof(real), (size_t)NDIAG * threads * sizeof(double));
    if (!set_smem(k_diag<real, N, DIM, NV>, smem)) return smem_fail(smem);
    const int nb = (g.nelem + epb - 1) / epb;
    if (nb != c->diag_blocks) return SD_EINVAL;
    // persistent: as many blocks as are resident at once (fixed for a device, so the order
    // of the sums, and the result, are the same on every call)
    const int nbp = persistent_grid(k_diag<real, N, DIM, NV>, threads, smem, nb, c->device);
    sdi_prof_begin(c, SD_K_OTHER);
    k_diag<real, N, DIM, NV><<<nbp, threads, smem, c->stream>>>(U, Tu, ops, g, c->dW, c->J, c->partial, off0,
                                                                off4);
    sdi_prof_end(c, SD_K_OTHER);
    return diag_reduce(c, nbp);
}

template <int N, int DIM, int NV>
static sd_status diag_impl(sd_ctx* c, const double* U) {
    if (c->prec == SD_F32) return diag_impl_r<float, N, DIM, NV>(c, U, (float*)c->Tu64);
    return diag_impl_r<double, N, DIM, NV>(c, U, c->Tu64);
}

template <int N>
static sd_status diag_n(sd_ctx* c, const double* U) {
    if (c->nvar == 5) return diag_impl<N, 3, 5>(c, U);
    if (c->dim == 1) return diag_impl<N, 1, 1>(c, U);
    return diag_impl<N, 3, 1>(c, U);
}
}  // namespace sdk

extern "C" sd_status sd_diagnostics(sd_ctx* c, const double* U64, double t, sd_diag* out) {
    if (!c || !U64 || !out) { sdi_set_error("null argument"); return SD_EINVAL; }
    sd_status s;
    if (c->curv) {
        s = sdi_curv_diag_partials(c, U64);
        if (s == SD_OK) s = sdk::diag_reduce(c, c->diag_nb);
    } else switch (c->n) {
        case 2: s = sdk::diag_n<2>(c, U64); break;
        case 3: s = sdk::diag_n<3>(c, U64); break;
        case 4: s = sdk::diag_n<4>(c, U64); break;
        case 5: s = sdk::diag_n<5>(c, U64); break;
        case 6: s = sdk::diag_n<6>(c, U64); break;
        case 7: s = sdk::diag_n<7>(c, U64); break;
        case 8: s = sdk::diag_n<8>(c, U64); break;
        case 9: s = sdk::diag_n<9>(c, U64); break;
        default: s = SD_EUNSUPPORTED;
    }
    if (s != SD_OK) return s;
    double h[sdk::NDIAG];
    CK(cudaMemcpyAsync(h, c->dsum, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    memset(out, 0, sizeof(*out));
    out->t = t;
    out->ke = h[0];
    out->ke_rho = h[1];
    out->enstrophy = h[2];
    out->mass = h[3];
    out->mom[0] = h[4];
    out->mom[1] = h[5];
    out->mom[2] = h[6];
    out->energy = h[7];
    out->l2sq = h[8];
    double vol = 1.0;
    for (int d = 0; d < c->dim; ++d)
        vol *= c->own_set ? (c->own_hi[d] - c->own_lo[d]) * c->h[d] : c->hi[d] - c->lo[d];
    out->volume = c->curv ? c->curv_volume : vol;
    out->nonfinite = h[9] != 0.0 ? 1 : 0;
    if (out->nonfinite) {
        sdi_set_error("state holds %g non-finite points", h[9]);
        return SD_ENONFINITE;
    }
    return SD_OK;
}

// ------------------------------------------------------------------ closure
extern "C" sd_status sd_set_flux_tau(sd_ctx* c, const float* tau) {
    if (!c) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (c->nvar != 5 && tau) { sdi_set_error("a per-element flux needs Navier-Stokes"); return SD_EUNSUPPORTED; }
    if (c->curv && tau) { sdi_set_error("a per-element flux is available on Cartesian grids only"); return SD_EUNSUPPORTED; }
    c->tau = tau;
    return SD_OK;
}

extern "C" sd_status sd_closure_data(sd_ctx* c, const void* U, float* X, double* means) {
    if (!c || !U || (!X && !means)) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (c->curv) { sdi_set_error("closure data are available on Cartesian grids only"); return SD_EUNSUPPORTED; }
    if (c->prec == SD_F32) return sdi_closure_data_f32(c, (const float*)U, X, means);
    return sdi_closure_data_f64(c, (const double*)U, X, means);
}

extern "C" sd_status sd_filter_matrix(int pf, int pc, int r, double* P) {
    if (pf < 1 || pc < 1 || pf > SD_MAX_N - 1 || pc > SD_MAX_N - 1 || r < 1 || !P) {
        sdi_set_error("bad argument");
        return SD_EINVAL;
    }
    const int nf = pf + 1, nc = pc + 1;
    double xf[SD_MAX_N], wf[SD_MAX_N], xc[SD_MAX_N], wc[SD_MAX_N];
    gauss_legendre(nf, xf, wf);
    gauss_legendre(nc, xc, wc);
    for (int a = 0; a < nc; ++a)
        for (int s = 0; s < r; ++s)
            for (int k = 0; k < nf; ++k) {
                const double xi = -1.0 + (2.0 * s + 1.0 + xf[k]) / r;   // fine point, coarse coords
                P[a * r * nf + s * nf + k] = wf[k] * lagrange(xc, nc, a, xi) / (r * wc[a]);
            }
    return SD_OK;
}

sd_status sdi_closure_network(sd_ctx* c) {
    const int E = c->nelem;
    sd_status s = sd_standardise(c->cl_X, E, 64, c->cl_mux, c->cl_sgx, c->cl_Xb, nullptr, c->stream);
    if (s == SD_OK) s = sd_mlp_forward(c->cl_Xb, E, c->cl_Wb, c->cl_P, c->cl_Y, c->cl_H, c->stream);
    if (s == SD_OK) s = sd_unstandardise(c->cl_Y, E, 15, c->cl_mut, c->cl_sgt, c->cl_tau, c->stream);
    c->launches += 3;
    return s;
}

extern "C" sd_status sd_closure_enable(sd_ctx* c, const void* Wb, const float* P, const float* mu_x,
                                       const float* sig_x, const float* mu_t, const float* sig_t) {
    if (!c) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (!Wb) {                       // detach
        free_closure(c);
        return SD_OK;
    }
    if (!P || !mu_x || !sig_x || !mu_t || !sig_t) { sdi_set_error("null argument"); return SD_EINVAL; }
    if (c->nvar != 5) { sdi_set_error("the closure needs Navier-Stokes"); return SD_EUNSUPPORTED; }
    if (c->curv) { sdi_set_error("the closure is available on Cartesian grids only"); return SD_EUNSUPPORTED; }
    if (!c->cl_X) {
        const size_t E = (size_t)c->nelem;
        bool ok = cudaMalloc((void**)&c->cl_X, E * 64 * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&c->cl_Xb, E * 64 * 2) == cudaSuccess &&
                  cudaMalloc((void**)&c->cl_Y, E * 15 * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&c->cl_H, 2 * E * 128 * 2) == cudaSuccess &&
                  cudaMalloc((void**)&c->cl_tau, E * 15 * sizeof(float)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_closure(c);
            sdi_set_error("allocation of the closure buffers failed");
            return SD_ENOMEM;
        }
    }
    c->cl_Wb = Wb;
    c->cl_P = P;
    c->cl_mux = mu_x;
    c->cl_sgx = sig_x;
    c->cl_mut = mu_t;
    c->cl_sgt = sig_t;
    c->tau = c->cl_tau;
    c->closure_on = 1;
    return SD_OK;
}
