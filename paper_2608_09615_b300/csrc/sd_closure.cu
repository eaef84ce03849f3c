// Closure data path, precision-independent kernels: the box filter (L2 projection of a fine
// SD state onto the nested coarse SD space), the sub-grid flux targets, feature / target
// standardisation and the BF16 cast of the network input. The element-staged kernels
// (flux means, features) are in sd_closure.cuh.
#include <stdint.h>

#include <cuda_bf16.h>

#include "sd_internal.h"

namespace cls {

// One block per coarse element. Fine elements (r per axis) of the coarse element are read
// for one variable at a time; the 1D projection P[a][s nf + k] is applied along x, y, z.
// Uf: [nv][Ef_z][Ef_y][Ef_x][nf^3], Uc: [nv][Ec_z][Ec_y][Ec_x][nc^3] (FP64).
__global__ void k_project(const double* __restrict__ Uf, double* __restrict__ Uc,
                          const double* __restrict__ P, int nv, int ncx, int ncy, int ncz, int r, int nf,
                          int nc) {
    extern __shared__ __align__(16) double sh[];
    const int ec = blockIdx.x;
    const int cx = ec % ncx, cy = (ec / ncx) % ncy, cz = ec / (ncx * ncy);
    const int L = r * nf;                         // fine points per coarse line
    const int nfx = ncx * r, nfy = ncy * r;
    const size_t nef = (size_t)nfx * nfy * ncz * r;
    const size_t nec = (size_t)ncx * ncy * ncz;
    const int npf = nf * nf * nf, npc = nc * nc * nc;
    double* A = sh;                               // [L][L][L] (z, y, x)
    double* B = A + L * L * L;                    // [L][L][nc]  after x
    double* C = B + L * L * nc;                   // [L][nc][nc] after y
    for (int v = 0; v < nv; ++v) {
        for (int t = threadIdx.x; t < L * L * L; t += blockDim.x) {
            const int X = t % L, Y = (t / L) % L, Z = t / (L * L);
            const int sx = X / nf, i = X % nf, sy = Y / nf, j = Y % nf, sz = Z / nf, k = Z % nf;
            const size_t ef = ((size_t)(cz * r + sz) * nfy + (cy * r + sy)) * nfx + (cx * r + sx);
            A[t] = Uf[(size_t)v * nef * npf + ef * npf + (k * nf + j) * nf + i];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < L * L * nc; t += blockDim.x) {
            const int a = t % nc, Y = (t / nc) % L, Z = t / (nc * L);
            double s = 0.0;
            for (int X = 0; X < L; ++X) s += P[a * L + X] * A[(Z * L + Y) * L + X];
            B[t] = s;                             // B[Z][Y][a]
        }
        __syncthreads();
        for (int t = threadIdx.x; t < L * nc * nc; t += blockDim.x) {
            const int a = t % nc, b = (t / nc) % nc, Z = t / (nc * nc);
            double s = 0.0;
            for (int Y = 0; Y < L; ++Y) s += P[b * L + Y] * B[(Z * L + Y) * nc + a];
            C[t] = s;                             // C[Z][b][a]
        }
        __syncthreads();
        for (int t = threadIdx.x; t < npc; t += blockDim.x) {
            const int a = t % nc, b = (t / nc) % nc, c = t / (nc * nc);
            double s = 0.0;
            for (int Z = 0; Z < L; ++Z) s += P[c * L + Z] * C[(Z * nc + b) * nc + a];
            Uc[(size_t)v * nec * npc + (size_t)ec * npc + t] = s;
        }
        __syncthreads();
    }
}

// tau[ec][k] = mean over the r^3 children of fine[ef][k] - coarse[ec][k], k < 15 (FP32 out)
__global__ void k_targets(const double* __restrict__ fine, const double* __restrict__ coarse,
                          float* __restrict__ tau, int ncx, int ncy, int ncz, int r) {
    const int nec = ncx * ncy * ncz;
    const int nfx = ncx * r, nfy = ncy * r;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nec * 15; t += gridDim.x * blockDim.x) {
        const int ec = t / 15, k = t % 15;
        const int cx = ec % ncx, cy = (ec / ncx) % ncy, cz = ec / (ncx * ncy);
        double s = 0.0;
        for (int sz = 0; sz < r; ++sz)
            for (int sy = 0; sy < r; ++sy)
                for (int sx = 0; sx < r; ++sx) {
                    const size_t ef = ((size_t)(cz * r + sz) * nfy + (cy * r + sy)) * nfx + (cx * r + sx);
                    s += fine[ef * 15 + k];
                }
        tau[t] = (float)(s / (double)(r * r * r) - coarse[(size_t)ec * 15 + k]);
    }
}

// column means and standard deviations of A[rows][cols] (one block per column, fixed order)
__global__ void k_colstats(const float* __restrict__ A, int rows, int cols, float* __restrict__ mu,
                           float* __restrict__ sigma) {
    __shared__ double s1[256], s2[256];
    const int c = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double x = A[(size_t)r * cols + c];
        a += x;
        b += x * x;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            s1[threadIdx.x] += s1[threadIdx.x + st];
            s2[threadIdx.x] += s2[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = s1[0] / rows;
        const double var = s2[0] / rows - m * m;
        mu[c] = (float)m;
        sigma[c] = (float)(var > 1e-24 ? sqrt(var) : 1.0);
    }
}

// out = (A - mu) / sigma, as BF16 (network input) or FP32 (targets)
__global__ void k_standardise(const float* __restrict__ A, int rows, int cols, const float* __restrict__ mu,
                              const float* __restrict__ sigma, __nv_bfloat16* __restrict__ outb,
                              float* __restrict__ outf) {
    const size_t n = (size_t)rows * cols;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % cols);
        const float z = (A[t] - mu[c]) / sigma[c];
        if (outb) outb[t] = __float2bfloat16(z);
        if (outf) outf[t] = z;
    }
}

// tau = Y sigma + mu (network output back to physical sub-grid flux), FP32
__global__ void k_unstandardise(const float* __restrict__ Y, int rows, int cols, const float* __restrict__ mu,
                                const float* __restrict__ sigma, float* __restrict__ out) {
    const size_t n = (size_t)rows * cols;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % cols);
        out[t] = Y[t] * sigma[c] + mu[c];
    }
}

}  // namespace cls

using namespace cls;

extern "C" sd_status sd_filter_project(const double* Uf, double* Uc, const double* P, int nv,
                                       const int* ne_coarse, int r, int nf, int nc, void* stream) {
    if (!Uf || !Uc || !P || !ne_coarse || nv < 1 || r < 1 || nf < 1 || nc < 1) {
        sdi_set_error("bad argument");
        return SD_EINVAL;
    }
    const int L = r * nf;
    const size_t smem = sizeof(double) * ((size_t)L * L * L + (size_t)L * L * nc + (size_t)L * nc * nc);
    if (smem > 227 * 1024) { sdi_set_error("projection block too large"); return SD_EUNSUPPORTED; }
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SD_ECUDA;
    const int nec = ne_coarse[0] * ne_coarse[1] * ne_coarse[2];
    k_project<<<nec, 256, smem, (cudaStream_t)stream>>>(Uf, Uc, P, nv, ne_coarse[0], ne_coarse[1],
                                                        ne_coarse[2], r, nf, nc);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { sdi_set_error("projection launch: %s", cudaGetErrorString(e)); return SD_ECUDA; }
    return SD_OK;
}

extern "C" sd_status sd_closure_targets(const double* fine_means, const double* coarse_means, float* tau,
                                        const int* ne_coarse, int r, void* stream) {
    if (!fine_means || !coarse_means || !tau || !ne_coarse || r < 1) { sdi_set_error("bad argument"); return SD_EINVAL; }
    k_targets<<<128, 256, 0, (cudaStream_t)stream>>>(fine_means, coarse_means, tau, ne_coarse[0], ne_coarse[1],
                                                     ne_coarse[2], r);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

extern "C" sd_status sd_colstats(const float* A, int rows, int cols, float* mu, float* sigma, void* stream) {
    if (!A || !mu || !sigma || rows < 1 || cols < 1) { sdi_set_error("bad argument"); return SD_EINVAL; }
    k_colstats<<<cols, 256, 0, (cudaStream_t)stream>>>(A, rows, cols, mu, sigma);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

extern "C" sd_status sd_standardise(const float* A, int rows, int cols, const float* mu, const float* sigma,
                                    void* out_bf16, float* out_f32, void* stream) {
    if (!A || !mu || !sigma || rows < 0 || cols < 1 || (!out_bf16 && !out_f32)) {
        sdi_set_error("bad argument");
        return SD_EINVAL;
    }
    if (rows == 0) return SD_OK;
    k_standardise<<<256, 256, 0, (cudaStream_t)stream>>>(A, rows, cols, mu, sigma, (__nv_bfloat16*)out_bf16, out_f32);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

extern "C" sd_status sd_unstandardise(const float* Y, int rows, int cols, const float* mu, const float* sigma,
                                      float* out, void* stream) {
    if (!Y || !mu || !sigma || !out || rows < 0 || cols < 1) { sdi_set_error("bad argument"); return SD_EINVAL; }
    if (rows == 0) return SD_OK;
    k_unstandardise<<<256, 256, 0, (cudaStream_t)stream>>>(Y, rows, cols, mu, sigma, out);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}
