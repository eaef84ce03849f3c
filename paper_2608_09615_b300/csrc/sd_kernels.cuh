// Device code of the SD residual (Lodato & Tonicello, Secs. 2.1-2.3, 4.3, 4.4).
//
// This header holds the physics device functions, the element staging used by the FP64
// diagnostics, and the Runge-Kutta stage kernels. The residual kernels themselves are
// in sd_line.cuh. Values exchanged between elements go through two face-trace buffers:
// Tu[e][face][var][q] (traces of u) and Tg[e][face][comp][q] (own interface gradients).
//
// Bitwise consistency: a value computed by both elements sharing an interface (the
// trace, the correction delta, the own-side interface gradient) is produced by the same
// device function with an explicit fma sequence, so both sides see identical bits and
// the interface flux is single-valued; conservation then holds to round-off.
//
// Compact closed form (Cartesian grids). With delta_L = (u_{e-}(1) - u_e(-1))/2 and
// delta_R = (u_{e+}(-1) - u_e(1))/2 along direction d, Eqs. v:s:l / v:s:r remove from
// v^S the derivative of the opposite-face correction; extrapolated to the own face this
// leaves, for the d-component of the gradient only,
//   left  face: c_L^T L v^S - (2/h_d) alpha delta_R,  alpha = c_L^T L M c_R = (-1)^p / 2
//   right face: c_R^T L v^S - (2/h_d) beta  delta_L,  beta  = c_R^T L M c_L = -alpha
// The transverse components equal the BR1 values (Sec. 2.3: transverse fluxes stay
// continuous). The CPU oracle forms the one-sided arrays literally instead.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdk {

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <typename real, int N>
struct Ops {
    real L[(N + 1) * N];     // L[f*N + i]     = l_i(xi_{f-1/2})          (Eq. Lmat)
    real M[N * (N + 1)];     // M[i*(N+1) + f] = l'_{f-1/2}(xi_i)         (Eq. Mmat)
    real D[N * N];           // D = M L: derivative at solution points
    real two_h[3];           // 2/h_d  (J^-1 S_dd of the affine map)
    real corrL[3];           // (2/h_d) alpha
    real corrR[3];           // (2/h_d) beta
};

template <typename real>
struct Phys {
    int kind;                // 0 heat, 1 porous medium, 2 Navier-Stokes
    int sutherland;
    int riemann;             // 0 Roe, 1 Rusanov
    int vflux;               // interface viscous flux: 0 option (a), 1 option (b) (Sec. 2.1)
    int pme_sol;             // porous medium diffusivity at the solution points (Sec. 4.3 variant)
    real nu, m_pme;
    real gamma, gm1, gamma_Pr, mu0, p0, rhoE0, inv_e0, suth_s, suth_1ps, harten;
    real rho0, H0;           // reference offsets: rho0, rhoE0 + p0
};

struct Mesh {
    int ne[3];
    int nelem;
    int e_begin, e_end;      // elements [e_begin, e_end) processed by a residual launch
    int olo[3], ohi[3];      // owned box of a sub-domain (the diagnostics sum over it only)
};

// element e lies in the owned box [olo, ohi) of the grid
__device__ __forceinline__ bool owned(const Mesh& g, int e) {
    const int c0 = e % g.ne[0];
    const int r = e / g.ne[0];
    const int c1 = r % g.ne[1];
    const int c2 = r / g.ne[1];
    return c0 >= g.olo[0] && c0 < g.ohi[0] && c1 >= g.olo[1] && c1 < g.ohi[1] && c2 >= g.olo[2] && c2 < g.ohi[2];
}

// ------------------------------------------------------------------ index helpers
template <int N>
__device__ __forceinline__ int npow(int d) {
    return d == 0 ? 1 : (d == 1 ? N : N * N);
}

// point index of the point at position i along direction d on the line whose
// face index (point index with direction d removed) is q
template <int N>
__device__ __forceinline__ int pt_of(int d, int i, int q) {
    const int lo = npow<N>(d);
    return (q % lo) + lo * i + lo * N * (q / lo);
}

// (periodic wrap; the direction picks its coordinate by branches, not by indexing a local
// array, which would live in local memory)
__device__ __forceinline__ int neighbour(const Mesh& g, int e, int d, int side) {
    const int nx = g.ne[0], ny = g.ne[1], nz = g.ne[2];
    int c0 = e % nx;
    const int r = e / nx;
    int c1 = r % ny;
    int c2 = r / ny;
    const int s = side ? 1 : -1;
    if (d == 0) {
        c0 += s;
        c0 = c0 < 0 ? c0 + nx : (c0 >= nx ? c0 - nx : c0);
    } else if (d == 1) {
        c1 += s;
        c1 = c1 < 0 ? c1 + ny : (c1 >= ny ? c1 - ny : c1);
    } else {
        c2 += s;
        c2 = c2 < 0 ? c2 + nz : (c2 >= nz ? c2 - nz : c2);
    }
    return c0 + nx * (c1 + ny * c2);
}

// sum_i row[i] * base[i*stride], one fixed fma sequence
template <typename real, int N>
__device__ __forceinline__ real line_dot(const real* row, const real* base, int stride) {
    real s = row[0] * base[0];
#pragma unroll
    for (int i = 1; i < N; ++i) s = fma(row[i], base[i * stride], s);
    return s;
}

// gradient components exchanged at a face normal to d: the d-derivative of every
// variable, and for NS the two transverse derivatives of rho and rho u_d (all the
// viscous flux in direction d needs when lambda = 0).
template <int NV>
__device__ __forceinline__ void comp_map(int d, int c, int& v, int& m) {
    if (NV == 1 || c < NV) {
        v = (NV == 1) ? 0 : c;
        m = d;
        return;
    }
    const int t = (c - NV) >> 1;            // 0 -> first transverse, 1 -> second
    m = (d + 1 + t) % 3;
    v = ((c - NV) & 1) ? 1 + d : 0;
}

template <int NV>
struct NumGrad {
    static constexpr int value = (NV == 1) ? 1 : 9;
};

// ------------------------------------------------------------------ physics
template <typename real>
__device__ __forceinline__ real sutherland_mu(const Phys<real>& P, real e) {
    if (!P.sutherland) return P.mu0;
    const real th = e * P.inv_e0;
    return P.mu0 * th * sqrt(th) * P.suth_1ps / (th + P.suth_s);
}

// Navier-Stokes fluxes on reference-offset states. The residual kernels stage
// U' = (rho - rho0, rho u, rho v, rho w, rho E - rhoE0) with rhoE0 = p0/(gamma - 1): the
// 1D operators commute with constant offsets (rows of L sum to 1, rows of D and M to 0),
// so this is the same scheme, but the sweeps no longer carry the O(p0/(gamma-1)) constant
// part of rho E (at Ma = 0.1 it is ~180 against O(1) variations, and its round-off in the
// extrapolated traces was the dominant residual error). p' = p - p0 = (gamma-1)(U'_4 - rho
// |u|^2/2) and the momentum rows carry p' (the constant p0 has zero discrete divergence).

// Sec. 4.4 inviscid flux along d (F_c), offset state
template <typename real>
__device__ __forceinline__ void ns_convective(const real* U, int d, const Phys<real>& P,
                                              real* F) {
    const real ir = real(1) / (U[0] + P.rho0);
    const real v0 = U[1] * ir, v1 = U[2] * ir, v2 = U[3] * ir;
    const real ke2 = U[1] * v0 + U[2] * v1 + U[3] * v2;        // rho |u|^2
    const real pp = P.gm1 * (U[4] - real(0.5) * ke2);          // p - p0
    const real ud = (d == 0) ? v0 : (d == 1 ? v1 : v2);
    F[0] = U[1 + d];
    F[1] = U[1] * ud;
    F[2] = U[2] * ud;
    F[3] = U[3] * ud;
    F[1 + d] += pp;
    F[4] = ((U[4] + pp) + P.H0) * ud;                          // (rho E + p) u_d
}

// Sec. 4.4 viscous flux along d from the 9 exchanged conservative-gradient components g
// (comp_map order): tau = mu (grad u + grad u^T) (lambda = 0), heat flux
// kappa grad T = (mu gamma / Pr) grad e, primitive gradients from conservative ones.
template <typename real>
__device__ __forceinline__ void ns_viscous(const real* U, const real* g, int d,
                                           const Phys<real>& P, real* Fv) {
    const real ir = real(1) / (U[0] + P.rho0);
    const real vel[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const real E = (U[4] + P.rhoE0) * ir;
    const real e = E - real(0.5) * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    const real mu = sutherland_mu(P, e);
    real dud[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dud[i] = (g[1 + i] - vel[i] * g[0]) * ir;   // d u_i / d x_d
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const real ud = vel[d];
    const real dt1 = (g[6] - ud * g[5]) * ir;                               // d u_d / d x_t1
    const real dt2 = (g[8] - ud * g[7]) * ir;                               // d u_d / d x_t2
    const real dE = (g[4] - E * g[0]) * ir;
    const real de = dE - (vel[0] * dud[0] + vel[1] * dud[1] + vel[2] * dud[2]);
    real tau[3];
    tau[d] = real(2) * mu * dud[d];
    tau[t1] = mu * (dud[t1] + dt1);
    tau[t2] = mu * (dud[t2] + dt2);
    Fv[0] = real(0);
    Fv[1] = tau[0];
    Fv[2] = tau[1];
    Fv[3] = tau[2];
    Fv[4] = vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + mu * P.gamma_Pr * de;
}

// F_c - F_v along d at an interior flux point (Sec. 4.4), offset state U and the 9 exchanged
// gradient components g (comp_map order): ns_convective minus ns_viscous with the
// reciprocal of rho, the velocity and the pressure shared by both parts
template <typename real>
__device__ __forceinline__ void ns_flux_point(const real* U, const real* g, int d, const Phys<real>& P,
                                              real* F) {
    const real ir = real(1) / (U[0] + P.rho0);
    const real vel[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const real ke2 = U[1] * vel[0] + U[2] * vel[1] + U[3] * vel[2];     // rho |u|^2
    const real pp = P.gm1 * (U[4] - real(0.5) * ke2);                   // p - p0
    const real ud = vel[d];
    const real E = (U[4] + P.rhoE0) * ir;
    const real e = E - real(0.5) * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    const real mu = sutherland_mu(P, e);
    real dud[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dud[i] = (g[1 + i] - vel[i] * g[0]) * ir;   // d u_i / d x_d
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const real dt1 = (g[6] - ud * g[5]) * ir;                               // d u_d / d x_t1
    const real dt2 = (g[8] - ud * g[7]) * ir;                               // d u_d / d x_t2
    const real dE = (g[4] - E * g[0]) * ir;
    const real de = dE - (vel[0] * dud[0] + vel[1] * dud[1] + vel[2] * dud[2]);
    real tau[3];
    tau[d] = real(2) * mu * dud[d];
    tau[t1] = mu * (dud[t1] + dt1);
    tau[t2] = mu * (dud[t2] + dt2);
    F[0] = U[1 + d];
#pragma unroll
    for (int i = 0; i < 3; ++i) F[1 + i] = U[1 + i] * ud - tau[i];
    F[1 + d] += pp;
    F[4] = ((U[4] + pp) + P.H0) * ud - (vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + mu * P.gamma_Pr * de);
}

// Roe flux with Harten's fix on the acoustic eigenvalues (Sec. 4.4), or Rusanov; offset
// states (jumps and p' differences are offset-free)
template <typename real>
__device__ __forceinline__ void ns_riemann(const real* UL, const real* UR, int d,
                                           const Phys<real>& P, real* F) {
    // central part first: F = (F_c(U_L) + F_c(U_R)) / 2
    ns_convective(UL, d, P, F);
    {
        real FR[5];
        ns_convective(UR, d, P, FR);
#pragma unroll
        for (int k = 0; k < 5; ++k) F[k] = real(0.5) * (F[k] + FR[k]);
    }
    const real rl = UL[0] + P.rho0, rr = UR[0] + P.rho0;
    const real irl = real(1) / rl, irr = real(1) / rr;
    const real vl[3] = {UL[1] * irl, UL[2] * irl, UL[3] * irl};
    const real vr[3] = {UR[1] * irr, UR[2] * irr, UR[3] * irr};
    const real ppl = P.gm1 * (UL[4] - real(0.5) * (UL[1] * vl[0] + UL[2] * vl[1] + UL[3] * vl[2]));
    const real ppr = P.gm1 * (UR[4] - real(0.5) * (UR[1] * vr[0] + UR[2] * vr[1] + UR[3] * vr[2]));
    if (P.riemann == 1) {
        const real cl = sqrt(P.gamma * (ppl + P.p0) * irl), cr = sqrt(P.gamma * (ppr + P.p0) * irr);
        const real sl = fabs(vl[d]) + cl, sr = fabs(vr[d]) + cr;
        const real smax = sl > sr ? sl : sr;
#pragma unroll
        for (int k = 0; k < 5; ++k) F[k] -= real(0.5) * smax * (UR[k] - UL[k]);
        return;
    }
    const real sl = sqrt(rl), sr = sqrt(rr);
    const real iw = real(1) / (sl + sr);
    const real Ht = (sl * (((UL[4] + ppl) + P.H0) * irl) + sr * (((UR[4] + ppr) + P.H0) * irr)) * iw;
    real ut[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ut[i] = (sl * vl[i] + sr * vr[i]) * iw;
    const real rt = sl * sr;
    const real q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
    const real c2 = P.gm1 * (Ht - real(0.5) * q2);
    const real c = sqrt(c2);
    const real qn = ut[d];
    const real drho = UR[0] - UL[0];
    const real dp = ppr - ppl;
    real dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dv[i] = vr[i] - vl[i];
    const real dvn = dv[d];
    real l1 = fabs(qn - c), l2 = fabs(qn), l5 = fabs(qn + c);
    if (P.harten > real(0)) {
        const real del = P.harten * c;
        if (l1 < del) l1 = (l1 * l1 + del * del) / (real(2) * del);
        if (l5 < del) l5 = (l5 * l5 + del * del) / (real(2) * del);
    }
    const real ic2 = real(1) / c2;
    const real a1 = (dp - rt * c * dvn) * real(0.5) * ic2;
    const real a2 = drho - dp * ic2;
    const real a5 = (dp + rt * c * dvn) * real(0.5) * ic2;
    // half of the dissipation sum_k |lambda_k| alpha_k r_k, subtracted component by component
    const real w1 = real(0.5) * l1 * a1, w2 = real(0.5) * l2 * a2, w5 = real(0.5) * l5 * a5;
    const real ws = real(0.5) * l2 * rt;
    F[0] -= w1 + w2 + w5;
    real utdvt = real(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const real dvt = dv[i] - (i == d ? dvn : real(0));
        const real en = (i == d) ? c : real(0);
        F[1 + i] -= w1 * (ut[i] - en) + w2 * ut[i] + w5 * (ut[i] + en) + ws * dvt;
        utdvt += ut[i] * dvt;
    }
    F[4] -= w1 * (Ht - qn * c) + w2 * real(0.5) * q2 + w5 * (Ht + qn * c) + ws * utdvt;
}

// scalar diffusivity (heat: nu; PME: m |u|^(m-1), Eq. pme) and flux -coef v_d
template <typename real>
__device__ __forceinline__ real scalar_coef(const Phys<real>& P, real u) {
    if (P.kind == 1) return P.m_pme * pow(fabs(u), P.m_pme - real(1));
    return P.nu;
}

template <typename real>
__device__ __forceinline__ real scalar_flux(const Phys<real>& P, real u, real g) {
    return -scalar_coef(P, u) * g;
}

// ------------------------------------------------------------------ element staging
// Shared-memory footprint per element (in reals) for the gradient / flux kernels.
template <int N, int DIM, int NV>
struct Footprint {
    static constexpr int NP = ipow(N, DIM);
    static constexpr int NQ = ipow(N, DIM - 1);
    static constexpr int NF = 2 * DIM;
    static constexpr int U = NV * NP;
    static constexpr int TR = NF * NV * NQ;
    static constexpr int VS = NV * DIM * NP;
    static constexpr int G = NV * (N + 1) * NQ;
    static constexpr int grad = U + 2 * TR + VS;
    static constexpr int flux = U + 2 * TR + VS + G;
    static constexpr int TPE = ((NP + 31) / 32) * 32;   // threads per element
    // largest block the host launches: ~256 threads, or one element when TPE > 256
    static constexpr int MAXT = TPE > 256 ? TPE : 256;
};

// Stage u, the own traces, the neighbour traces and v^S of element e in shared memory.
// All TPE threads of the element call this; ends with the element's v^S ready.
template <typename real, int N, int DIM, int NV>
__device__ __forceinline__ void stage_element(const real* __restrict__ U,
                                              const real* __restrict__ Tu,
                                              const Ops<real, N>& ops, const Mesh& g,
                                              int e, bool valid, int tid, real* su,
                                              real* tro, real* trn, real* vS) {
    using FP = Footprint<N, DIM, NV>;
    constexpr int NP = FP::NP, NQ = FP::NQ, NF = FP::NF, TPE = FP::TPE;
    // (the diagnostics need no gradient of a scalar, and for Navier-Stokes only the
    // derivatives of rho and of the momentum components across the derivative direction:
    // the vorticity)
    if (valid) {
        // (U = nullptr: the caller has staged u already)
        for (int k = tid; U && k < NV * NP; k += TPE) {
            const int v = k / NP, pt = k - v * NP;
            su[k] = U[(size_t)v * g.nelem * NP + (size_t)e * NP + pt];
        }
        if constexpr (NV == 5) {
            for (int k = tid; k < NF * NV * NQ; k += TPE) {
                const int f = k / (NV * NQ);
                const int rem = k - f * NV * NQ;
                if (rem >= 4 * NQ) continue;
                const int d = f >> 1, s = f & 1;
                const int en = neighbour(g, e, d, s);
                // the neighbour's trace on the shared face is its face of opposite side
                trn[k] = Tu[((size_t)en * NF + (f ^ 1)) * NV * NQ + rem];
            }
        }
    }
    __syncthreads();
    if constexpr (NV != 5) return;
    if (valid) {
        for (int k = tid; k < NF * NV * NQ; k += TPE) {
            const int f = k / (NV * NQ);
            const int rem = k - f * NV * NQ;
            const int v = rem / NQ, q = rem - v * NQ;
            if (v >= 4) continue;
            const int d = f >> 1, s = f & 1;
            tro[k] = line_dot<real, N>(ops.L + (s ? N * N : 0), su + v * NP + pt_of<N>(d, 0, q),
                                       npow<N>(d));
        }
    }
    __syncthreads();
    if (valid) {
        // Eq. w:e in Cartesian form: v_m = (2/h_m) M_m u^{Fm,C}
        //   = (2/h_m) (D u + M[:,0] delta_L + M[:,N] delta_R) along m.
        for (int k = tid; k < NV * DIM * NP; k += TPE) {
            const int vm = k / NP, pt = k - vm * NP;
            const int v = vm / DIM, m = vm - v * DIM;
            if (v >= 4 || (v >= 1 && v - 1 == m)) continue;
            const int lo = npow<N>(m);
            const int i = (pt / lo) % N;
            const int q = (pt % lo) + lo * (pt / (lo * N));
            real acc = line_dot<real, N>(ops.D + i * N, su + v * NP + pt_of<N>(m, 0, q), lo);
            const int fl = 2 * m, fr = 2 * m + 1;
            const real dl = real(0.5) * (trn[(fl * NV + v) * NQ + q] - tro[(fl * NV + v) * NQ + q]);
            const real dr = real(0.5) * (trn[(fr * NV + v) * NQ + q] - tro[(fr * NV + v) * NQ + q]);
            acc = fma(ops.M[i * (N + 1)], dl, acc);
            acc = fma(ops.M[i * (N + 1) + N], dr, acc);
            vS[k] = ops.two_h[m] * acc;
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ kernels
// ------------------------------------------------------------------ diagnostics (FP64)
// Sums, per block, of the Gauss-weighted integrands of Sec. 4.4 plus conserved totals;
// k_diag_final adds the block partials in a fixed order (deterministic).
constexpr int NDIAG = 10;   // ke, ke_rho, enstrophy, mass, mom0..2, energy, l2sq, nonfinite
constexpr int DIAG_L1 = 256;   // blocks of the first level of the partials' reduction

// The diagnostics of a state whose values are staged in `real`: FP64 contexts stage U as it
// is; FP32 contexts stage (U - offsets) rounded to FP32 (the offsets of rho and rho E, as the
// residual kernels do) and evaluate the kinetic-energy and enstrophy integrands in FP32. Every
// sum is FP64 and the conserved totals are taken from the FP64 state itself.
// The face traces for the diagnostics: one thread per line (element, direction d, variable,
// line q) extrapolates the staged values to both faces of direction d.
template <typename real, int N, int DIM, int NV>
__global__ void k_trace_staged(const double* __restrict__ U, real* __restrict__ Tu, Ops<real, N> ops, Mesh g,
                               double off0, double off4) {
    constexpr int NP = ipow(N, DIM), NQ = ipow(N, DIM - 1), NF = 2 * DIM;
    const long long total = (long long)g.nelem * DIM * NV * NQ;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(idx % NQ);
        long long r = idx / NQ;
        const int v = (int)(r % NV);
        r /= NV;
        if (NV == 5 && v == 4) continue;      // the diagnostics use no trace of rho E
        const int d = (int)(r % DIM);
        const int e = (int)(r / DIM);
        const double off = (NV == 5 && v == 0) ? off0 : 0.0;
        const double* src = U + (size_t)v * g.nelem * NP + (size_t)e * NP + pt_of<N>(d, 0, q);
        real x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = (real)(src[i * npow<N>(d)] - off);
        real* out = Tu + (((size_t)e * NF + 2 * d) * NV + v) * NQ + q;
        out[0] = line_dot<real, N>(ops.L, x, 1);
        out[NV * NQ] = line_dot<real, N>(ops.L + N * N, x, 1);
    }
}

template <typename real, int N, int DIM, int NV>
__global__ void __launch_bounds__(Footprint<N, DIM, NV>::MAXT) k_diag(const double* __restrict__ U, const real* __restrict__ Tu,
                       Ops<real, N> ops, Mesh g, const double* __restrict__ wq, double J,
                       double* __restrict__ partial, double off0, double off4) {
    using FP = Footprint<N, DIM, NV>;
    constexpr int NP = FP::NP, TPE = FP::TPE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sm = reinterpret_cast<real*>(smem_raw);
    const int le = threadIdx.x / TPE, tid = threadIdx.x - le * TPE;
    const int epb = blockDim.x / TPE;
    real* base = sm + le * FP::grad;
    real* su = base;
    real* tro = su + FP::U;
    real* trn = tro + FP::TR;
    real* vS = trn + FP::TR;
    // persistent: block b handles the element groups b, b + grid, ...; each thread adds its
    // points' integrands over all of them in FP64, and the block's threads are summed once
    double acc[NDIAG];
#pragma unroll
    for (int k = 0; k < NDIAG; ++k) acc[k] = 0.0;
    const int ngroups = (g.nelem + epb - 1) / epb;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int e = grp * epb + le;
        const bool valid = e < g.nelem;
        // stage_element reads the state in `real`: give it the staged values through shared memory
        if (valid) {
            for (int k = tid; k < NV * NP; k += TPE) {
                const int v = k / NP, pt = k - v * NP;
                const double off = (NV == 5 && v == 0) ? off0 : ((NV == 5 && v == 4) ? off4 : 0.0);
                su[k] = (real)(U[(size_t)v * g.nelem * NP + (size_t)e * NP + pt] - off);
            }
        }
        stage_element<real, N, DIM, NV>(nullptr, Tu, ops, g, e, valid, tid, su, tro, trn, vS);
        if (valid && owned(g, e)) {
            for (int pt = tid; pt < NP; pt += TPE) {
                double w = J;
                int r = pt;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    w *= wq[r % N];
                    r /= N;
                }
                const double* Ue = U + (size_t)e * NP + pt;
                bool bad = false;
#pragma unroll
                for (int v = 0; v < NV; ++v) bad |= !isfinite(Ue[(size_t)v * g.nelem * NP]);
                acc[9] += bad ? 1.0 : 0.0;
                if constexpr (NV == 5) {
                    const real rho = su[pt] + (real)off0;
                    const real vel[3] = {su[NP + pt] / rho, su[2 * NP + pt] / rho, su[3 * NP + pt] / rho};
                    const real q2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
                    real du[3][3] = {};   // du[k][i] = d u_i / d x_k, off-diagonal (the vorticity)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int i = 0; i < 3; ++i)
                            if (i != k)
                                du[k][i] = (vS[((1 + i) * DIM + k) * NP + pt] - vel[i] * vS[(0 * DIM + k) * NP + pt]) / rho;
                    const real o0 = du[1][2] - du[2][1], o1 = du[2][0] - du[0][2], o2 = du[0][1] - du[1][0];
                    acc[0] += w * (0.5 * (double)q2);
                    acc[1] += w * (0.5 * (double)rho * (double)q2);
                    acc[2] += w * (double)(o0 * o0 + o1 * o1 + o2 * o2);
                    const size_t S = (size_t)g.nelem * NP;
                    acc[3] += w * Ue[0];
                    acc[4] += w * Ue[S];
                    acc[5] += w * Ue[2 * S];
                    acc[6] += w * Ue[3 * S];
                    acc[7] += w * Ue[4 * S];
                } else {
                    const double u = Ue[0];
                    acc[3] += w * u;
                    acc[8] += w * u * u;
                }
            }
        }
        __syncthreads();   // the group's staged values are read before the next group
    }
    // deterministic block reduction (fixed tree over the threads), in FP64
    double* red = reinterpret_cast<double*>(smem_raw);   // NDIAG * blockDim doubles fit (host sizes it)
    for (int k = 0; k < NDIAG; ++k) red[k * blockDim.x + threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = 1; s < (int)blockDim.x; s <<= 1) {
        if ((threadIdx.x % (2 * s)) == 0 && threadIdx.x + s < blockDim.x)
            for (int k = 0; k < NDIAG; ++k)
                red[k * blockDim.x + threadIdx.x] += red[k * blockDim.x + threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NDIAG; ++k) partial[(size_t)blockIdx.x * NDIAG + k] = red[k * blockDim.x];
}

__global__ void k_diag_final(const double* __restrict__ partial, int nblocks,
                             double* __restrict__ out);

// ------------------------------------------------------------------ Runge-Kutta (FP64)
// Stage inputs of the residual are written in the residual precision and with the
// reference offsets of the first and last variable removed (rho - rho0, rho E - rhoE0 for
// Navier-Stokes; zero offsets otherwise), in FP64 before rounding.
struct StageOff {
    size_t npts;      // values per variable
    double off0, off4;
};

__device__ __forceinline__ double stage_offset(const StageOff& o, size_t i) {
    return i < o.npts ? o.off0 : (i >= 4 * o.npts ? o.off4 : 0.0);
}

// y = x - offsets, rounded to real. Each thread handles 8 values spaced one grid apart per
// iteration and issues their loads together (one load in flight per thread reached only
// half the copy bandwidth). FP64 subtraction only in the first and last variable (FP64
// issue is scarce; the test is on the index, not on the offset's value).
template <typename real>
__global__ void k_to_real(const double* __restrict__ x, real* __restrict__ y, size_t n, StageOff o) {
    constexpr int W = 8;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += W * stride) {
        double v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const size_t i = base + w * stride;
            v[w] = i < n ? x[i] : 0.0;
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const size_t i = base + w * stride;
            if (i >= n) continue;
            if (i < o.npts) y[i] = (real)(v[w] - o.off0);
            else if (i >= 4 * o.npts) y[i] = (real)(v[w] - o.off4);
            else y[i] = (real)v[w];
        }
    }
}

// RK4 stage k (0..3): K holds R(stage input). Uacc accumulates the weighted stages; S is
// the next stage input (residual precision); the last stage writes U.
template <typename real>
__global__ void k_rk4(int k, double* __restrict__ U, double* __restrict__ Uacc,
                      const real* __restrict__ K, real* __restrict__ S, double dt, size_t n,
                      StageOff o) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double u = U[i];
        const double kk = (double)K[i];
        const double off = stage_offset(o, i);
        if (k == 0) {
            Uacc[i] = u + dt / 6.0 * kk;
            S[i] = (real)(u + 0.5 * dt * kk - off);
        } else if (k == 1) {
            Uacc[i] += dt / 3.0 * kk;
            S[i] = (real)(u + 0.5 * dt * kk - off);
        } else if (k == 2) {
            Uacc[i] += dt / 3.0 * kk;
            S[i] = (real)(u + dt * kk - off);
        } else {
            U[i] = Uacc[i] + dt / 6.0 * kk;
        }
    }
}

// SSPRK(5,4) in Shu-Osher form (Spiteri & Ruuth 2002). Registers: U = u0, A = u1/u3/u4,
// B = u2, C = a52 u2 + a53 u3 + b53 dt L(u3).
struct SSPCoef {
    double a10, a20, a21, b21, a30, a32, b32, a40, a43, b43, a52, a53, b53, a54, b54;
};

template <typename real>
__global__ void k_ssp(int k, double* __restrict__ U, double* __restrict__ A,
                      double* __restrict__ B, double* __restrict__ C, const real* __restrict__ K,
                      real* __restrict__ S, double dt, SSPCoef c, size_t n, StageOff o) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double kk = dt * (double)K[i];
        const double off = stage_offset(o, i);
        if (k == 0) {
            const double u1 = U[i] + c.a10 * kk;
            A[i] = u1;
            S[i] = (real)(u1 - off);
        } else if (k == 1) {
            const double u2 = c.a20 * U[i] + c.a21 * A[i] + c.b21 * kk;
            B[i] = u2;
            S[i] = (real)(u2 - off);
        } else if (k == 2) {
            const double u3 = c.a30 * U[i] + c.a32 * B[i] + c.b32 * kk;
            A[i] = u3;
            S[i] = (real)(u3 - off);
        } else if (k == 3) {
            const double u3 = A[i];
            C[i] = c.a52 * B[i] + c.a53 * u3 + c.b53 * kk;
            const double u4 = c.a40 * U[i] + c.a43 * u3 + c.b43 * kk;
            A[i] = u4;
            S[i] = (real)(u4 - off);
        } else {
            U[i] = C[i] + c.a54 * A[i] + c.b54 * kk;
        }
    }
}

// LSRK(5,4) of Carpenter & Kennedy: dU <- a dU + dt K; U <- U + b dU.
template <typename real>
__global__ void k_lsrk(double* __restrict__ U, double* __restrict__ dU, const real* __restrict__ K,
                       real* __restrict__ S, double a, double b, double dt, size_t n, StageOff o) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double du = a * dU[i] + dt * (double)K[i];
        dU[i] = du;
        const double u = U[i] + b * du;
        U[i] = u;
        S[i] = (real)(u - stage_offset(o, i));
    }
}

// ------------------------------------------------------------------ Runge-Kutta, FP32 residual
// Increment form used by FP32 contexts. Within one step every stage state is u_j = U + d_j,
// with U the FP64 state at the start of the step and d_0 = 0. The Shu-Osher weights of each
// stage sum to one, so the stage combination only involves the increments d_j = O(dt). The
// increments live in FP32: their rounding (6e-8 of an O(dt) quantity) is far below the FP32
// residual's own error. The conserved state accumulates in FP64 once per step: U <- U + d_s.
// The stage input is X + d_j in FP32, where X = U - offsets is rounded once per step.
// Coefficients arrive premultiplied by dt (FP64 products rounded once).
struct SSPInc {
    float b10, a21, b21, a32, b32, a43, b43, a52, a53, b53, a54, b54;
};

// One point of stage k of that form: kk is the stage residual, x the step-start value minus
// the offsets, a / b the increment registers A, B at the point (updated in place). Stages
// 0-3 return the next stage input x + d; stage 4 updates the FP64 state u. Stage 3 leaves in
// A not its increment d_4 but a54 d_4 + (a52 d_2 + a53 d_3 + b53 K_3), the only form in
// which stage 4 uses d_4, so no third register is needed. Every operation is explicitly
// rounded (no contraction into other operations).
__device__ __forceinline__ float ssp_inc_point(const SSPInc& c, int k, float kk, float x, float& a, float& b,
                                               double& u) {
    if (k == 0) {
        const float d = __fmul_rn(c.b10, kk);
        a = d;
        return __fadd_rn(x, d);
    }
    if (k == 1) {
        const float d = __fmaf_rn(c.a21, a, __fmul_rn(c.b21, kk));
        b = d;
        return __fadd_rn(x, d);
    }
    if (k == 2) {
        const float d = __fmaf_rn(c.a32, b, __fmul_rn(c.b32, kk));
        a = d;
        return __fadd_rn(x, d);
    }
    if (k == 3) {
        const float cc = __fmaf_rn(c.a52, b, __fmaf_rn(c.a53, a, __fmul_rn(c.b53, kk)));
        const float d = __fmaf_rn(c.a43, a, __fmul_rn(c.b43, kk));
        a = __fmaf_rn(c.a54, d, cc);
        return __fadd_rn(x, d);
    }
    u = __dadd_rn(u, (double)__fmaf_rn(c.b54, kk, a));
    return 0.0f;
}


__global__ void k_ssp_inc(int k, double* __restrict__ U, float* __restrict__ A, float* __restrict__ B,
                          const float* __restrict__ K, const float* __restrict__ X, float* __restrict__ S,
                          SSPInc c, size_t n);

struct RK4Inc {
    float h2, h1, h6, h3;     // dt/2, dt, dt/6, dt/3
};

__global__ void k_rk4_inc(int k, double* __restrict__ U, float* __restrict__ A, const float* __restrict__ K,
                          const float* __restrict__ X, float* __restrict__ S, RK4Inc c, size_t n);

// Low-storage form: W <- a W + dt K, D <- D + b W (D = the running increment of U).
__global__ void k_lsrk_inc(int k, int last, double* __restrict__ U, float* __restrict__ W,
                           float* __restrict__ D, const float* __restrict__ K, const float* __restrict__ X,
                           float* __restrict__ S, float a, float dt, float b, size_t n);

}  // namespace sdk
