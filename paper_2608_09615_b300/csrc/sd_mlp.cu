// Per-element MLP closure 64 -> 128 -> 128 -> 15 (ReLU hidden layers): BF16 operands on
// the tensor cores (mma.sync m16n8k16, FP32 accumulation), FP32 biases, MSE loss and Adam
// on FP32 master parameters. All buffers are the caller's; nothing is allocated here.
//
// Parameter vector (FP32 masters and gradients), packed:
//   W1 [128][64] | b1 [128] | W2 [128][128] | b2 [128] | W3 [16][128] | b3 [16]
// (W3 and b3 carry a zero 16th output row so that layer 3 is one n = 16 tile). The BF16
// weight copy uses the same offsets for W1, W2, W3 (biases unused there).
#include <cuda_bf16.h>
#include <stdint.h>

#include "sd_internal.h"

namespace mlp {

constexpr int IN = 64, HID = 128, OUT = 15, OUTP = 16;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + OUTP * HID;
constexpr int NPARAM = OFF_B3 + OUTP;
constexpr int ROWS = 64;            // rows per block (4 warps x 16)

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t pack(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D(16 x 8) += A(16 x 16) B(16 x 8), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Warp tile: C[16 x 8 NB] += A[16 x K] B[K x 8 NB], A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn], BF16 in shared memory, K a multiple of 16. Fragment layout of
// m16n8k16 (g = lane / 4, t = lane % 4): A regs hold (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..),
// (g+8, 2t+8..); B regs hold (2t..2t+1, g), (2t+8..2t+9, g); C holds (g, 2t..2t+1) and
// (g+8, 2t..2t+1).
template <int NB>
__device__ __forceinline__ void warp_gemm(float (&acc)[NB][4], const bf16* A, int sam, int sak,
                                          const bf16* B, int sbk, int sbn, int K) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        const int ka = k0 + 2 * t;
        a[0] = pack(A[g * sam + ka * sak], A[g * sam + (ka + 1) * sak]);
        a[1] = pack(A[(g + 8) * sam + ka * sak], A[(g + 8) * sam + (ka + 1) * sak]);
        a[2] = pack(A[g * sam + (ka + 8) * sak], A[g * sam + (ka + 9) * sak]);
        a[3] = pack(A[(g + 8) * sam + (ka + 8) * sak], A[(g + 8) * sam + (ka + 9) * sak]);
#pragma unroll
        for (int nb = 0; nb < NB; ++nb) {
            const int n = nb * 8 + g;
            uint32_t b[2];
            b[0] = pack(B[ka * sbk + n * sbn], B[(ka + 1) * sbk + n * sbn]);
            b[1] = pack(B[(ka + 8) * sbk + n * sbn], B[(ka + 9) * sbk + n * sbn]);
            mma16816(acc[nb], a, b);
        }
    }
}

template <int NB>
__device__ __forceinline__ void zero(float (&acc)[NB][4]) {
#pragma unroll
    for (int nb = 0; nb < NB; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[nb][j] = 0.f;
}

__device__ __forceinline__ void copy_rows(bf16* dst, const bf16* src, int rows_valid, int cols, int row0,
                                          int nrows_total) {
    for (int k = threadIdx.x; k < ROWS * cols; k += blockDim.x) {
        const int r = k / cols, c = k - r * cols;
        dst[k] = (r < rows_valid) ? src[(size_t)(row0 + r) * cols + c] : __float2bfloat16(0.f);
    }
    (void)nrows_total;
}

// ---------------------------------------------------------------- forward
// Y[M][15] = W3 relu(W2 relu(W1 x + b1) + b2) + b3; H[0] = relu layer-1 output, H[1] =
// relu layer-2 output (BF16, kept for the backward pass).
__global__ void __launch_bounds__(128) k_forward(const bf16* __restrict__ X, int M,
                                                 const bf16* __restrict__ Wb,
                                                 const float* __restrict__ P,
                                                 float* __restrict__ Y, bf16* __restrict__ H) {
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* sW1 = reinterpret_cast<bf16*>(smem);
    bf16* sW2 = sW1 + HID * IN;
    bf16* sW3 = sW2 + HID * HID;
    bf16* sX = sW3 + OUTP * HID;
    bf16* sH1 = sX + ROWS * IN;
    bf16* sH2 = sH1 + ROWS * HID;
    const int row0 = blockIdx.x * ROWS;
    const int valid = min(ROWS, M - row0);
    for (int k = threadIdx.x; k < HID * IN; k += blockDim.x) sW1[k] = Wb[OFF_W1 + k];
    for (int k = threadIdx.x; k < HID * HID; k += blockDim.x) sW2[k] = Wb[OFF_W2 + k];
    for (int k = threadIdx.x; k < OUTP * HID; k += blockDim.x) sW3[k] = Wb[OFF_W3 + k];
    copy_rows(sX, X, valid, IN, row0, M);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = warp * 16;
    float acc[16][4];
    // layer 1
    zero(acc);
    warp_gemm<16>(acc, sX + r0 * IN, IN, 1, sW1, 1, IN, IN);
#pragma unroll
    for (int nb = 0; nb < 16; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
            sH1[r * HID + c] = __float2bfloat16(fmaxf(acc[nb][j] + P[OFF_B1 + c], 0.f));
        }
    __syncwarp();
    // layer 2
    zero(acc);
    warp_gemm<16>(acc, sH1 + r0 * HID, HID, 1, sW2, 1, HID, HID);
#pragma unroll
    for (int nb = 0; nb < 16; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
            sH2[r * HID + c] = __float2bfloat16(fmaxf(acc[nb][j] + P[OFF_B2 + c], 0.f));
        }
    __syncwarp();
    // layer 3
    float a3[2][4];
    zero(a3);
    warp_gemm<2>(a3, sH2 + r0 * HID, HID, 1, sW3, 1, HID, HID);
#pragma unroll
    for (int nb = 0; nb < 2; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
            if (c < OUT && r < valid) Y[(size_t)(row0 + r) * OUT + c] = a3[nb][j] + P[OFF_B3 + c];
        }
    __syncthreads();
    for (int k = threadIdx.x; k < valid * HID; k += blockDim.x) {
        H[(size_t)row0 * HID + k] = sH1[k];
        H[(size_t)M * HID + (size_t)row0 * HID + k] = sH2[k];
    }
}

// ---------------------------------------------------------------- loss
// loss = mean over rows and the 15 outputs of (Y - T)^2; dY = 2 (Y - T) / (15 M).
// Block partial sums of the squared error, added in a fixed order by k_loss_final.
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ T, int M,
                       float* __restrict__ dY, double* __restrict__ part) {
    __shared__ double red[256];
    const size_t n = (size_t)M * OUT;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d / (float)n;
        s += (double)d * (double)d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_final(const double* __restrict__ part, int nb, size_t n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *out = s / (double)n;
    }
}

// ---------------------------------------------------------------- backward
// Per block of 64 rows: back-propagate dY through layers 3, 2, 1 (ReLU masks from the cached
// activations) and write the block's partial parameter gradient (packed like the
// parameters) to part[blockIdx.x].
__global__ void __launch_bounds__(128) k_backward(const bf16* __restrict__ X, const bf16* __restrict__ H,
                                                  const float* __restrict__ dY, int M,
                                                  const bf16* __restrict__ Wb,
                                                  float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* sW2 = reinterpret_cast<bf16*>(smem);
    bf16* sW3 = sW2 + HID * HID;
    bf16* sX = sW3 + OUTP * HID;
    bf16* sH1 = sX + ROWS * IN;
    bf16* sH2 = sH1 + ROWS * HID;
    bf16* sdY = sH2 + ROWS * HID;
    bf16* sdZ2 = sdY + ROWS * OUTP;
    bf16* sdZ1 = sdZ2 + ROWS * HID;
    const int row0 = blockIdx.x * ROWS;
    const int valid = min(ROWS, M - row0);
    for (int k = threadIdx.x; k < HID * HID; k += blockDim.x) sW2[k] = Wb[OFF_W2 + k];
    for (int k = threadIdx.x; k < OUTP * HID; k += blockDim.x) sW3[k] = Wb[OFF_W3 + k];
    copy_rows(sX, X, valid, IN, row0, M);
    copy_rows(sH1, H, valid, HID, row0, M);
    copy_rows(sH2, H + (size_t)M * HID, valid, HID, row0, M);
    for (int k = threadIdx.x; k < ROWS * OUTP; k += blockDim.x) {
        const int r = k / OUTP, c = k - r * OUTP;
        sdY[k] = __float2bfloat16((r < valid && c < OUT) ? dY[(size_t)(row0 + r) * OUT + c] : 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = warp * 16;
    float acc[16][4];
    // dH2 = dY W3, dZ2 = dH2 * (H2 > 0)
    zero(acc);
    warp_gemm<16>(acc, sdY + r0 * OUTP, OUTP, 1, sW3, HID, 1, OUTP);
#pragma unroll
    for (int nb = 0; nb < 16; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
            const float m = __bfloat162float(sH2[r * HID + c]) > 0.f ? 1.f : 0.f;
            sdZ2[r * HID + c] = __float2bfloat16(acc[nb][j] * m);
        }
    __syncwarp();
    // dH1 = dZ2 W2, dZ1 = dH1 * (H1 > 0)
    zero(acc);
    warp_gemm<16>(acc, sdZ2 + r0 * HID, HID, 1, sW2, HID, 1, HID);
#pragma unroll
    for (int nb = 0; nb < 16; ++nb)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
            const float m = __bfloat162float(sH1[r * HID + c]) > 0.f ? 1.f : 0.f;
            sdZ1[r * HID + c] = __float2bfloat16(acc[nb][j] * m);
        }
    __syncthreads();
    float* out = part + (size_t)blockIdx.x * NPARAM;
    // dW2[o][i] = sum_r dZ2[r][o] H1[r][i]: warp handles outputs o in [32 w, 32 w + 32)
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int o0 = warp * 32 + mt * 16;
        zero(acc);
        warp_gemm<16>(acc, sdZ2 + o0, 1, HID, sH1, HID, 1, ROWS);
#pragma unroll
        for (int nb = 0; nb < 16; ++nb)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = o0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
                out[OFF_W2 + o * HID + c] = acc[nb][j];
            }
    }
    // dW1[o][i] = sum_r dZ1[r][o] X[r][i]
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int o0 = warp * 32 + mt * 16;
        float a1[8][4];
        zero(a1);
        warp_gemm<8>(a1, sdZ1 + o0, 1, HID, sX, IN, 1, ROWS);
#pragma unroll
        for (int nb = 0; nb < 8; ++nb)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = o0 + g + (j >> 1) * 8, c = nb * 8 + 2 * t + (j & 1);
                out[OFF_W1 + o * IN + c] = a1[nb][j];
            }
    }
    // dW3[o][i] = sum_r dY[r][o] H2[r][i]: warp handles columns i in [32 w, 32 w + 32)
    {
        float a3[4][4];
        zero(a3);
        warp_gemm<4>(a3, sdY, 1, OUTP, sH2 + warp * 32, HID, 1, ROWS);
#pragma unroll
        for (int nb = 0; nb < 4; ++nb)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = g + (j >> 1) * 8, c = warp * 32 + nb * 8 + 2 * t + (j & 1);
                out[OFF_W3 + o * HID + c] = a3[nb][j];
            }
    }
    // bias gradients: column sums over the block's rows (FP32, fixed order)
    for (int c = threadIdx.x; c < HID; c += blockDim.x) {
        float s1 = 0.f, s2 = 0.f;
        for (int r = 0; r < ROWS; ++r) {
            s1 += __bfloat162float(sdZ1[r * HID + c]);
            s2 += __bfloat162float(sdZ2[r * HID + c]);
        }
        out[OFF_B1 + c] = s1;
        out[OFF_B2 + c] = s2;
    }
    for (int c = threadIdx.x; c < OUTP; c += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += __bfloat162float(sdY[r * OUTP + c]);
        out[OFF_B3 + c] = s;
    }
}

// grad[k] = sum over blocks of part[b][k] (fixed order)
__global__ void k_reduce(const float* __restrict__ part, int nblocks, float* __restrict__ grad) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * NPARAM + k];
        grad[k] = s;
    }
}

// Adam on the FP32 masters; refreshes the BF16 weight copy
__global__ void k_adam(float* __restrict__ P, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ grad, bf16* __restrict__ Wb, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
        const float gk = grad[k];
        const float a = b1 * m1[k] + (1.f - b1) * gk;
        const float v = b2 * m2[k] + (1.f - b2) * gk * gk;
        m1[k] = a;
        m2[k] = v;
        const float p = P[k] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        P[k] = p;
        Wb[k] = __float2bfloat16(p);
    }
}

__global__ void k_cast(const float* __restrict__ P, bf16* __restrict__ Wb) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x)
        Wb[k] = __float2bfloat16(P[k]);
}

constexpr size_t FWD_SMEM = sizeof(bf16) * (HID * IN + HID * HID + OUTP * HID + ROWS * IN + 2 * ROWS * HID);
constexpr size_t BWD_SMEM = sizeof(bf16) * (HID * HID + OUTP * HID + ROWS * IN + 2 * ROWS * HID +
                                            ROWS * OUTP + 2 * ROWS * HID);

}  // namespace mlp

using namespace mlp;

static bool mlp_smem_ready() {
    static bool ok = false;
    static int dev_done = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (ok && dev == dev_done) return true;
    ok = cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM) == cudaSuccess &&
         cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BWD_SMEM) == cudaSuccess;
    dev_done = dev;
    return ok;
}

extern "C" int sd_mlp_param_count(void) { return NPARAM; }

extern "C" sd_status sd_mlp_cast(const float* P, void* Wb, void* stream) {
    if (!P || !Wb) { sdi_set_error("null argument"); return SD_EINVAL; }
    k_cast<<<32, 256, 0, (cudaStream_t)stream>>>(P, (bf16*)Wb);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

extern "C" sd_status sd_mlp_forward(const void* X, int M, const void* Wb, const float* P, float* Y,
                                    void* H, void* stream) {
    if (!X || !Wb || !P || !Y || !H || M < 0) { sdi_set_error("bad argument"); return SD_EINVAL; }
    if (M == 0) return SD_OK;
    if (!mlp_smem_ready()) { sdi_set_error("MLP shared-memory configuration failed"); return SD_ECUDA; }
    k_forward<<<(M + ROWS - 1) / ROWS, 128, FWD_SMEM, (cudaStream_t)stream>>>(
        (const bf16*)X, M, (const bf16*)Wb, P, Y, (bf16*)H);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { sdi_set_error("MLP forward launch: %s", cudaGetErrorString(e)); return SD_ECUDA; }
    return SD_OK;
}

extern "C" sd_status sd_mlp_loss(const float* Y, const float* T, int M, float* dY, double* part,
                                 double* loss, void* stream) {
    if (!Y || !T || !dY || !part || !loss || M <= 0) { sdi_set_error("bad argument"); return SD_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    k_loss<<<64, 256, 0, s>>>(Y, T, M, dY, part);
    k_loss_final<<<1, 32, 0, s>>>(part, 64, (size_t)M * OUT, loss);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}

extern "C" sd_status sd_mlp_backward(const void* X, const void* H, const float* dY, int M, const void* Wb,
                                     float* part, float* grad, void* stream) {
    if (!X || !H || !dY || !Wb || !part || !grad || M <= 0) { sdi_set_error("bad argument"); return SD_EINVAL; }
    if (!mlp_smem_ready()) { sdi_set_error("MLP shared-memory configuration failed"); return SD_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (M + ROWS - 1) / ROWS;
    k_backward<<<nb, 128, BWD_SMEM, s>>>((const bf16*)X, (const bf16*)H, dY, M, (const bf16*)Wb, part);
    k_reduce<<<(NPARAM + 255) / 256, 256, 0, s>>>(part, nb, grad);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { sdi_set_error("MLP backward launch: %s", cudaGetErrorString(e)); return SD_ECUDA; }
    return SD_OK;
}

extern "C" sd_status sd_mlp_adam(float* P, float* m1, float* m2, const float* grad, void* Wb, int step,
                                 float lr, float b1, float b2, float eps, void* stream) {
    if (!P || !m1 || !m2 || !grad || !Wb || step < 1) { sdi_set_error("bad argument"); return SD_EINVAL; }
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, m1, m2, grad, (bf16*)Wb, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? SD_OK : SD_ECUDA;
}
