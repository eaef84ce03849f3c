// Closure data kernels on the line-staged element layout (Navier-Stokes, 3D):
//   k_line_fluxmean  Gauss-weighted element means of the physical flux F = F_c - F_v at the
//                    solution points, with the SD gradient v^S      -> out[e][3 v + d] (FP64)
//   k_line_features  the 64 element features of the learned closure -> X[e][64] (FP32)
// Both stage the element exactly like the residual kernels (offset state, own and
// neighbour traces, v^S), so v^S is the same auxiliary gradient the residual uses.
// Feature list (per element; V = (rho - rho0, rho u, rho v, rho w, rho E - rhoE0) scaled by
// (rho0, rho0 u0, rho0 u0, rho0 u0, rho0 u0^2), means by Gauss quadrature over the element):
//    0-4   mean V_v              5-19  3 mean(V_v xi_d)          20-34 (h/2) mean dU_v/dx_d / scale_v
//   35-43  (h/2) mean du_i/dx_k / u0                             44-46 (h/2) mean de/dx_k / u0^2
//   47-51  fraction of the modal energy of V_v (mean excluded) in modes of degree p, with 1e-14
//          added to the denominator
//   52-56  variance of V_v       57-62 covariances of u_i/u0, u_j/u0 (i <= j)   63  1000/Re
#pragma once

#include "sd_line.cuh"

namespace sdk {

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// velocity gradient, de/dx and the flux pieces at one solution point from the staged data
template <typename real, int N>
__device__ __forceinline__ void point_state(const real* su, const real* vS, int pt, const Phys<real>& P,
                                            real* U, real (*g)[5]) {
    constexpr int NP = N * N * N;
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = su[v * NP + pt];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int v = 0; v < 5; ++v) g[k][v] = vS[(v * 3 + k) * NP + pt];   // g[k][v] = dU_v/dx_k
}

template <typename real, int N>
__global__ void __launch_bounds__(LineLayout<N, 3, 5>::THREADS)
k_line_fluxmean(const real* __restrict__ U, const real* __restrict__ Tu, LineGeo<real> geo, Mesh g,
                Phys<real> P, const double* __restrict__ wq, double* __restrict__ out) {
    using LL = LineLayout<N, 3, 5>;
    constexpr int NP = LL::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* nbr = reinterpret_cast<int*>(smem_raw);
    real* sm = reinterpret_cast<real*>(smem_raw + LL::NBR_BYTES);
    const int e0 = blockIdx.x * LL::EB;
    stage_load<real, LL, 5>(U, Tu, g, e0, sm, LL::PER_GRAD, geo.off0, geo.off4, nbr);
    __syncthreads();
    const LineId id = line_id<LL>(threadIdx.x);
    const bool live = id.ok && e0 + id.eb < g.nelem;
    {
        real* su = sm + id.eb * LL::PER_GRAD;
        real* tro = su + LL::S_U;
        real* trn = tro + LL::S_TR;
        real* vS = trn + LL::S_TR;
        prologue<real, N, 3, 5, ElemStrides<LL>>(geo, id, live, su, tro, trn, vS);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= LL::EB || e0 + warp >= g.nelem) return;
    const real* su = sm + warp * LL::PER_GRAD;
    const real* vS = su + LL::S_U + 2 * LL::S_TR;
    double acc[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) acc[k] = 0.0;
    for (int pt = lane; pt < NP; pt += 32) {
        const double w = wq[pt % N] * wq[(pt / N) % N] * wq[pt / (N * N)] * 0.125;
        real Up[5], gp[3][5];
        point_state<real, N>(su, vS, pt, P, Up, gp);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            real gd[9];
            for (int c = 0; c < 9; ++c) {
                int v, m;
                comp_map<5>(d, c, v, m);
                gd[c] = gp[m][v];
            }
            real Fc[5], Fv[5];
            ns_convective(Up, d, P, Fc);
            ns_viscous(Up, gd, d, P, Fv);
            // ns_convective carries p - p0 in the momentum rows; the physical flux has p
            Fc[1 + d] += P.p0;
#pragma unroll
            for (int v = 0; v < 5; ++v) acc[3 * v + d] += w * (double)(Fc[v] - Fv[v]);
        }
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        const double s = warp_sum(acc[k]);
        if (lane == 0) out[(size_t)(e0 + warp) * 15 + k] = s;
    }
}

template <typename real, int N>
__global__ void __launch_bounds__(LineLayout<N, 3, 5>::THREADS)
k_line_features(const real* __restrict__ U, const real* __restrict__ Tu, LineGeo<real> geo, Mesh g,
                Phys<real> P, const double* __restrict__ wq, const double* __restrict__ tmode,
                double half_h, double rho0, double u0, double inv_re, float* __restrict__ X) {
    using LL = LineLayout<N, 3, 5>;
    constexpr int NP = LL::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* nbr = reinterpret_cast<int*>(smem_raw);
    real* sm = reinterpret_cast<real*>(smem_raw + LL::NBR_BYTES);
    const int e0 = blockIdx.x * LL::EB;
    stage_load<real, LL, 5>(U, Tu, g, e0, sm, LL::PER_GRAD, geo.off0, geo.off4, nbr);
    __syncthreads();
    const LineId id = line_id<LL>(threadIdx.x);
    const bool live = id.ok && e0 + id.eb < g.nelem;
    {
        real* su = sm + id.eb * LL::PER_GRAD;
        real* tro = su + LL::S_U;
        real* trn = tro + LL::S_TR;
        real* vS = trn + LL::S_TR;
        prologue<real, N, 3, 5, ElemStrides<LL>>(geo, id, live, su, tro, trn, vS);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= LL::EB || e0 + warp >= g.nelem) return;
    const real* su = sm + warp * LL::PER_GRAD;
    const real* vS = su + LL::S_U + 2 * LL::S_TR;
    float* xo = X + (size_t)(e0 + warp) * 64;
    const double sc[5] = {rho0, rho0 * u0, rho0 * u0, rho0 * u0, rho0 * u0 * u0};
    // pass 1: means, linear moments, second moments
    {
        double a[5 + 15 + 5 + 9];
#pragma unroll
        for (int k = 0; k < 34; ++k) a[k] = 0.0;
        for (int pt = lane; pt < NP; pt += 32) {
            const int i = pt % N, j = (pt / N) % N, kk = pt / (N * N);
            const double w = wq[i] * wq[j] * wq[kk] * 0.125;
            const double xi[3] = {tmode[N * N + i], tmode[N * N + j], tmode[N * N + kk]};
            double V[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) V[v] = (double)su[v * NP + pt] / sc[v];
            const double rho = (double)su[pt] + (double)P.rho0;
            const double vel[3] = {(double)su[NP + pt] / rho / u0, (double)su[2 * NP + pt] / rho / u0,
                                   (double)su[3 * NP + pt] / rho / u0};
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                a[v] += w * V[v];
#pragma unroll
                for (int d = 0; d < 3; ++d) a[5 + 3 * v + d] += w * V[v] * xi[d];
                a[20 + v] += w * V[v] * V[v];
            }
            int q = 0;
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int jj = ii; jj < 3; ++jj) a[25 + q++] += w * vel[ii] * vel[jj];
#pragma unroll
            for (int ii = 0; ii < 3; ++ii) a[31 + ii] += w * vel[ii];
        }
#pragma unroll
        for (int k = 0; k < 34; ++k) a[k] = warp_sum(a[k]);
        if (lane == 0) {
            for (int v = 0; v < 5; ++v) {
                xo[v] = (float)a[v];
                for (int d = 0; d < 3; ++d) xo[5 + 3 * v + d] = (float)(3.0 * a[5 + 3 * v + d]);
                xo[52 + v] = (float)(a[20 + v] - a[v] * a[v]);
            }
            int q = 0;
            for (int ii = 0; ii < 3; ++ii)
                for (int jj = ii; jj < 3; ++jj) {
                    xo[57 + q] = (float)(a[25 + q] - a[31 + ii] * a[31 + jj]);
                    ++q;
                }
            xo[63] = (float)(1000.0 * inv_re);
        }
    }
    // pass 2: gradient means
    {
        double a[15 + 9 + 3];
#pragma unroll
        for (int k = 0; k < 27; ++k) a[k] = 0.0;
        for (int pt = lane; pt < NP; pt += 32) {
            const double w = wq[pt % N] * wq[(pt / N) % N] * wq[pt / (N * N)] * 0.125;
            double gk[3][5];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int v = 0; v < 5; ++v) gk[k][v] = (double)vS[(v * 3 + k) * NP + pt];
            const double rho = (double)su[pt] + (double)P.rho0;
            const double vel[3] = {(double)su[NP + pt] / rho, (double)su[2 * NP + pt] / rho,
                                   (double)su[3 * NP + pt] / rho};
            const double Et = ((double)su[4 * NP + pt] + (double)P.rhoE0) / rho;
#pragma unroll
            for (int v = 0; v < 5; ++v)
#pragma unroll
                for (int d = 0; d < 3; ++d) a[3 * v + d] += w * gk[d][v];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double de = (gk[k][4] - Et * gk[k][0]) / rho;
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) {
                    const double du = (gk[k][1 + ii] - vel[ii] * gk[k][0]) / rho;
                    a[15 + 3 * ii + k] += w * du;
                    de -= vel[ii] * du;
                }
                a[24 + k] += w * de;
            }
        }
#pragma unroll
        for (int k = 0; k < 27; ++k) a[k] = warp_sum(a[k]);
        if (lane == 0) {
            for (int v = 0; v < 5; ++v)
                for (int d = 0; d < 3; ++d) xo[20 + 3 * v + d] = (float)(half_h * a[3 * v + d] / sc[v]);
            for (int k = 0; k < 9; ++k) xo[35 + k] = (float)(half_h * a[15 + k] / u0);
            for (int k = 0; k < 3; ++k) xo[44 + k] = (float)(half_h * a[24 + k] / (u0 * u0));
        }
    }
    // pass 3: modal energy fractions; c_abc = sum T[c][k] T[b][j] T[a][i] V[k][j][i] with
    // T[m][i] = w_i P_m(x_i) (2m+1)/2 (tmode[m N + i]); energy c^2 prod 2/(2m+1)
    for (int v = 0; v < 5; ++v) {
        double top = 0.0, tot = 0.0;
        for (int md = lane; md < NP; md += 32) {
            const int a = md % N, b = (md / N) % N, c = md / (N * N);
            double s = 0.0;
            for (int pt = 0; pt < NP; ++pt) {
                const int i = pt % N, j = (pt / N) % N, kk = pt / (N * N);
                s += tmode[c * N + kk] * tmode[b * N + j] * tmode[a * N + i] * ((double)su[v * NP + pt] / sc[v]);
            }
            const double e = s * s * (2.0 / (2 * a + 1)) * (2.0 / (2 * b + 1)) * (2.0 / (2 * c + 1));
            if (md != 0) tot += e;
            if (a == N - 1 || b == N - 1 || c == N - 1) top += e;
        }
        top = warp_sum(top);
        tot = warp_sum(tot);
        if (lane == 0) xo[47 + v] = (float)(top / (tot + 1e-14));
    }
}

}  // namespace sdk
