// SD residual on periodic grids of curved hexahedra: the mapping of Sec. 2 with K = 8
// corner nodes (trilinear elements), Eqs. ns:mapped and adj:f (q = J u, G = S . F,
// H = S^T u with S = adj(dx/dxi)) and the steps of Sec. 2.3 with the metric terms taken
// point by point: row d of S at the flux points of family d, J^-1 at the solution points.
//
// Metric terms are computed in the kernels from seven coefficient vectors per element:
//   x(xi, eta, zeta) = c0 + c1 xi + c2 eta + c3 zeta + c4 xi eta + c5 eta zeta + c6 xi zeta
//                      + c7 xi eta zeta,
// so the tangents a_t = dx/dxi_t are bilinear, S row d = a_{d+1} x a_{d+2} (cyclic) and
// J = a_0 . (a_1 x a_2). This costs ~40 flops per point and replaces ~1.5 k stored metric
// values per element at n = 5 with 21 coefficients. Row d of S along xi_d is a polynomial of
// degree 2, which the n + 1 >= 3 flux points resolve exactly, so the discrete metric
// identity sum_d M_d S_dm = 0 holds and a uniform flow stays uniform.
//
// Kernels (one residual = 4 launches; the element kernels stage one element at a time in
// shared memory; k_cflux is persistent and copies the next element in while it computes):
//   k_ctrace  face traces of u                         Tc[e][face][v][q]
//   k_cgrad   v^S = J^-1 sum_d M_d (u^{Fd,C} S_dm), one thread per (line, variable) with the
//             line in registers, kept in VS[e][v][m][pt], and the own interface gradient of
//             every face (BR1: L v^S; compact: the one-sided form of Eqs. aux:v:cmp:l-t,
//             i.e. L v^S minus the extrapolated derivative of the opposite face's correction,
//             a per-line coefficient here since J varies)  Tg[e][face][v][m][q]
//   k_cface   one common flux per interface point: |S| F_riemann(n) - S . F_v  Fh[d][e][v][q]
//   k_cflux   S . F at the interior flux points, the stored interface fluxes at the ends,
//             R = -J^-1 sum_d M_d G^{Fd}
// Navier-Stokes states are staged with the reference offsets removed, as in the Cartesian
// kernels (the constant p0 part of the momentum flux is dropped: its discrete divergence is
// p0 times the metric identity, zero).
#include <algorithm>
#include <cmath>
#include <vector>

#include "sd_internal.h"
#include "sd_launch.cuh"

namespace sdc {

using sdk::Mesh;
using sdk::Phys;

constexpr int NGEO = 24;       // map coefficients per element: c1..c7 (x, y, z each), padded
constexpr int CURV_THREADS = 256;

template <typename real, int N>
struct COps {
    real L[(N + 1) * N];       // L[f*N + i] = l_i(xf_f)
    real M[N * (N + 1)];       // M[i*(N+1) + f] = l'_f(xs_i)
    real xs[N];
    real xf[N + 1];
};


// Direction-specialised index helpers: D is a template argument wherever a loop runs over
// one family, so strides are constants and no small array is indexed at run time.
template <int N, int D>
__device__ __forceinline__ int cpt(int i, int q) {
    constexpr int lo = D == 0 ? 1 : (D == 1 ? N : N * N);
    return (q % lo) + lo * i + lo * N * (q / lo);
}

// position along D and line index q of solution point pt
template <int N, int D>
__device__ __forceinline__ void line_of(int pt, int& i, int& q) {
    constexpr int lo = D == 0 ? 1 : (D == 1 ? N : N * N);
    i = (pt / lo) % N;
    q = (pt % lo) + lo * (pt / (lo * N));
}

// reference coordinates (xi, eta, zeta) of flux point f of family D on line q (transverse
// coordinates at the solution points; the lower transverse axis runs fastest in q)
template <typename real, int N, int D>
__device__ __forceinline__ void flux_point_coords(const COps<real, N>& o, int f, int q, real r[3]) {
    constexpr int t1 = D == 0 ? 1 : 0, t2 = D == 2 ? 1 : 2;
    r[D] = o.xf[f];
    r[t1] = o.xs[q % N];
    r[t2] = o.xs[q / N];
}

template <typename real, int N>
__device__ __forceinline__ void solution_point_coords(const COps<real, N>& o, int pt, real r[3]) {
    r[0] = o.xs[pt % N];
    r[1] = o.xs[(pt / N) % N];
    r[2] = o.xs[pt / (N * N)];
}

// tangent a_t[k] = d x_k / d xi_t of the trilinear map with coefficients c (c1..c7)
template <typename real, int T>
__device__ __forceinline__ void tangent(const real* c, const real r[3], real a[3]) {
    const real x = r[0], y = r[1], z = r[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (T == 0) a[k] = c[k] + c[9 + k] * y + c[15 + k] * z + c[18 + k] * (y * z);
        if (T == 1) a[k] = c[3 + k] + c[9 + k] * x + c[12 + k] * z + c[18 + k] * (x * z);
        if (T == 2) a[k] = c[6 + k] + c[12 + k] * y + c[15 + k] * x + c[18 + k] * (x * y);
    }
}

template <typename real>
__device__ __forceinline__ void cross3(const real* u, const real* v, real* w) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}

// row D of S = adj(dx/dxi) at reference point r: a_{D+1} x a_{D+2}
template <typename real, int D>
__device__ __forceinline__ void metric_row(const real* c, const real r[3], real S[3]) {
    real a1[3], a2[3];
    tangent<real, (D + 1) % 3>(c, r, a1);
    tangent<real, (D + 2) % 3>(c, r, a2);
    cross3(a1, a2, S);
}

template <typename real>
__device__ __forceinline__ real jacobian(const real* c, const real r[3]) {
    real a0[3], a1[3], a2[3], s[3];
    tangent<real, 0>(c, r, a0);
    tangent<real, 1>(c, r, a1);
    tangent<real, 2>(c, r, a2);
    cross3(a1, a2, s);
    return a0[0] * s[0] + a0[1] * s[1] + a0[2] * s[2];
}

// ------------------------------------------------------------------ physics on a general area vector
// sum_m S_m F_c,m(U) on an offset state (Sec. 4.4 inviscid flux; p' = p - p0)
template <typename real>
__device__ __forceinline__ void cv_convective(const real* U, const real* S, const Phys<real>& P, real* G) {
    const real ir = real(1) / (U[0] + P.rho0);
    const real v0 = U[1] * ir, v1 = U[2] * ir, v2 = U[3] * ir;
    const real pp = P.gm1 * (U[4] - real(0.5) * (U[1] * v0 + U[2] * v1 + U[3] * v2));
    const real us = v0 * S[0] + v1 * S[1] + v2 * S[2];
    G[0] = U[1] * S[0] + U[2] * S[1] + U[3] * S[2];
    G[1] = U[1] * us + pp * S[0];
    G[2] = U[2] * us + pp * S[1];
    G[3] = U[3] * us + pp * S[2];
    G[4] = ((U[4] + pp) + P.H0) * us;
}

// sum_m S_m F_v,m(U, g) with the full conservative gradient g[v*3 + k] = d U_v / d x_k:
// tau = mu (grad u + grad u^T) (lambda = 0), heat flux (mu gamma / Pr) grad e
template <typename real>
__device__ __forceinline__ void cv_viscous(const real* U, const real* g, const real* S, const Phys<real>& P,
                                           real* G) {
    const real ir = real(1) / (U[0] + P.rho0);
    const real vel[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
    const real E = (U[4] + P.rhoE0) * ir;
    const real e = E - real(0.5) * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
    const real mu = sdk::sutherland_mu(P, e);
    real du[3][3];             // du[i][k] = d u_i / d x_k
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) du[i][k] = (g[(1 + i) * 3 + k] - vel[i] * g[k]) * ir;
    real q[3];                 // heat flux direction: grad e
#pragma unroll
    for (int k = 0; k < 3; ++k)
        q[k] = (g[12 + k] - E * g[k]) * ir - (vel[0] * du[0][k] + vel[1] * du[1][k] + vel[2] * du[2][k]);
    G[0] = real(0);
    real en = real(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        real ti = real(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) ti += mu * (du[i][k] + du[k][i]) * S[k];
        G[1 + i] = ti;
        en += vel[i] * ti;
    }
    G[4] = en + mu * P.gamma_Pr * (q[0] * S[0] + q[1] * S[1] + q[2] * S[2]);
}

// Roe flux with Harten's fix (or Rusanov) along the unit normal n, offset states
template <typename real>
__device__ __forceinline__ void cv_riemann(const real* UL, const real* UR, const real* n, const Phys<real>& P,
                                           real* F) {
    cv_convective(UL, n, P, F);
    {
        real FR[5];
        cv_convective(UR, n, P, FR);
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
        const real sl = fabs(vl[0] * n[0] + vl[1] * n[1] + vl[2] * n[2]) + cl;
        const real sr = fabs(vr[0] * n[0] + vr[1] * n[1] + vr[2] * n[2]) + cr;
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
    const real qn = ut[0] * n[0] + ut[1] * n[1] + ut[2] * n[2];
    const real drho = UR[0] - UL[0];
    const real dp = ppr - ppl;
    real dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dv[i] = vr[i] - vl[i];
    const real dvn = dv[0] * n[0] + dv[1] * n[1] + dv[2] * n[2];
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
    const real w1 = real(0.5) * l1 * a1, w2 = real(0.5) * l2 * a2, w5 = real(0.5) * l5 * a5;
    const real ws = real(0.5) * l2 * rt;
    F[0] -= w1 + w2 + w5;
    real utdvt = real(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const real dvt = dv[i] - dvn * n[i];
        const real en = c * n[i];
        F[1 + i] -= w1 * (ut[i] - en) + w2 * ut[i] + w5 * (ut[i] + en) + ws * dvt;
        utdvt += ut[i] * dvt;
    }
    F[4] -= w1 * (Ht - qn * c) + w2 * real(0.5) * q2 + w5 * (Ht + qn * c) + ws * utdvt;
}

// ------------------------------------------------------------------ kernels
template <typename real, int N, int NV>
struct CSizes {
    static constexpr int NP = N * N * N;
    static constexpr int NQ = N * N;
    static constexpr int NFP = (N + 1) * NQ;          // flux points of one family
    static constexpr int OPS = (N + 1) * N + N * (N + 1) + N + (N + 1);   // L, M, xs, xf
    static constexpr int OPS_PAD = (OPS + 3) / 4 * 4;
    // gradient staging: operators, u, face corrections, J^-1, v^S, row D of S at the flux
    // points of family D for the three families, the compact corrections of the face
    // gradients, the map
    static constexpr int G_U = OPS_PAD;
    static constexpr int G_DL = G_U + NV * NP;
    static constexpr int G_JI = G_DL + 6 * NV * NQ;
    static constexpr int G_VS = G_JI + NP;
    static constexpr int G_W = G_VS + 3 * NV * NP;
    static constexpr int G_CR = G_W + 9 * NFP;
    static constexpr int G_C = G_CR + 18 * NQ;
    static constexpr int GRAD = G_C + NGEO;
};

// periodic face neighbour of element e across its face (d, side) (no run-time indexed array)
__device__ __forceinline__ int cneighbour(const Mesh& g, int e, int d, int side) {
    int cx = e % g.ne[0];
    const int r = e / g.ne[0];
    int cy = r % g.ne[1], cz = r / g.ne[1];
    const int s = side ? 1 : -1;
    if (d == 0) {
        cx += s;
        cx = cx < 0 ? cx + g.ne[0] : (cx >= g.ne[0] ? cx - g.ne[0] : cx);
    } else if (d == 1) {
        cy += s;
        cy = cy < 0 ? cy + g.ne[1] : (cy >= g.ne[1] ? cy - g.ne[1] : cy);
    } else {
        cz += s;
        cz = cz < 0 ? cz + g.ne[2] : (cz >= g.ne[2] ? cz - g.ne[2] : cz);
    }
    return cx + g.ne[0] * (cy + g.ne[1] * cz);
}

template <typename real, int NV>
__device__ __forceinline__ real var_offset(int v, real off0, real off4) {
    if (NV != 5) return real(0);
    return v == 0 ? off0 : (v == 4 ? off4 : real(0));
}

// copy the 1D operators to shared memory (their indices vary across a warp in the loops)
template <typename real, int N>
__device__ __forceinline__ void stage_ops(const COps<real, N>& o, real* s) {
    for (int k = threadIdx.x; k < (N + 1) * N; k += blockDim.x) {
        s[k] = o.L[k];
        s[(N + 1) * N + k] = o.M[k];
    }
    for (int k = threadIdx.x; k < N; k += blockDim.x) s[2 * N * (N + 1) + k] = o.xs[k];
    for (int k = threadIdx.x; k <= N; k += blockDim.x) s[2 * N * (N + 1) + N + k] = o.xf[k];
}

template <typename real, int N>
struct SOps {
    const real *L, *M, *xs, *xf;
    __device__ __forceinline__ explicit SOps(const real* s)
        : L(s), M(s + (N + 1) * N), xs(s + 2 * N * (N + 1)), xf(s + 2 * N * (N + 1) + N) {}
};

template <typename real, int N, int D>
__device__ __forceinline__ void flux_point_coords(const real* xs, const real* xf, int f, int q, real r[3]) {
    constexpr int t1 = D == 0 ? 1 : 0, t2 = D == 2 ? 1 : 2;
    r[D] = xf[f];
    r[t1] = xs[q % N];
    r[t2] = xs[q / N];
}

// values at the two faces of direction D on line q: (l(-1) . v, l(+1) . v); L0, LN are the
// first and last rows of L
template <typename real, int N, int D>
__device__ __forceinline__ void face_pair(const real* vs, const real* L0, const real* LN, int q, real& lo,
                                          real& hi) {
    real x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = vs[cpt<N, D>(i, q)];
    lo = L0[0] * x[0];
    hi = LN[0] * x[0];
#pragma unroll
    for (int i = 1; i < N; ++i) {
        lo = fma(L0[i], x[i], lo);
        hi = fma(LN[i], x[i], hi);
    }
}

// face traces of u, one element per block at a time (coalesced loads of the element's u):
// Tc[((e*6 + f)*NV + v)*NQ + q] = l(+-1) . u along d on line q, faces f = 2d (-d), 2d + 1 (+d)
template <typename real, int N, int NV>
__global__ void __launch_bounds__(128) k_ctrace(const real* __restrict__ U, real* __restrict__ Tc,
                                                const __grid_constant__ COps<real, N> o, Mesh g, real off0,
                                                real off4) {
    using CS = CSizes<real, N, NV>;
    constexpr int NP = CS::NP, NQ = CS::NQ;
    __shared__ real su[NV * NP];
    __shared__ real sL[2 * N];
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid < N) {
        sL[tid] = o.L[tid];
        sL[N + tid] = o.L[N * N + tid];
    }
    constexpr int LPT = (NV * NP + 127) / 128;   // loads per thread (blockDim.x = 128)
    for (int e = blockIdx.x; e < g.nelem; e += gridDim.x) {
        // all of a thread's loads are issued before the first store (one load in flight per
        // thread left the kernel at a third of the copy bandwidth)
        real x[LPT];
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int k = tid + j * T;
            if (k < NV * NP) {
                const int v = k / NP, pt = k - v * NP;
                x[j] = U[(size_t)v * g.nelem * NP + (size_t)e * NP + pt];
            }
        }
#pragma unroll
        for (int j = 0; j < LPT; ++j) {
            const int k = tid + j * T;
            if (k < NV * NP) su[k] = x[j] - var_offset<real, NV>(k / NP, off0, off4);
        }
        __syncthreads();
        for (int k = tid; k < 3 * NV * NQ; k += T) {
            const int d = k / (NV * NQ), rem = k - d * NV * NQ;
            const int v = rem / NQ, q = rem - v * NQ;
            real lo, hi;
            switch (d) {
                case 0: face_pair<real, N, 0>(su + v * NP, sL, sL + N, q, lo, hi); break;
                case 1: face_pair<real, N, 1>(su + v * NP, sL, sL + N, q, lo, hi); break;
                default: face_pair<real, N, 2>(su + v * NP, sL, sL + N, q, lo, hi); break;
            }
            Tc[((size_t)e * 6 + 2 * d) * NV * NQ + rem] = lo;
            Tc[((size_t)e * 6 + 2 * d + 1) * NV * NQ + rem] = hi;
        }
        __syncthreads();
    }
}

// row D of S at the n + 1 flux points of family D, point k = f * NQ + q: sf[m * NFP + k]
template <typename real, int N, int D>
__device__ __forceinline__ void metric_rows(const SOps<real, N>& op, const real* sc, int k, real* sf) {
    constexpr int NQ = N * N, NFP = (N + 1) * NQ;
    const int f = k / NQ, q = k - f * NQ;
    real r[3], S[3];
    flux_point_coords<real, N, D>(op.xs, op.xf, f, q, r);
    metric_row<real, D>(sc, r, S);
#pragma unroll
    for (int m = 0; m < 3; ++m) sf[m * NFP + k] = S[m];
}

// compact scheme, face point q of face 2D + s: the one-sided gradient removes the derivative
// of the opposite face's correction, extrapolated to this face (Eqs. aux:v:cmp:l-t):
//   L_s (J^-1 M[:, opp]) delta_opp S_Dm(opp);  cr[m] = (L_s J^-1 M[:, opp]) S_Dm(opp)
template <typename real, int N, int NV, int D>
__device__ __forceinline__ void face_correction(const real* sm, int s, int q, real* cr) {
    using CS = CSizes<real, N, NV>;
    const SOps<real, N> op(sm);
    const real* sji = sm + CS::G_JI;
    const real* sc = sm + CS::G_C;
    const int fo = s ? 0 : N;
    const real* Lr = op.L + (s ? N * N : 0);
    real kap = real(0);
#pragma unroll
    for (int i = 0; i < N; ++i) kap = fma(Lr[i] * sji[cpt<N, D>(i, q)], op.M[i * (N + 1) + fo], kap);
    real r[3], S[3];
    flux_point_coords<real, N, D>(op.xs, op.xf, fo, q, r);
    metric_row<real, D>(sc, r, S);
#pragma unroll
    for (int m = 0; m < 3; ++m) cr[m] = kap * S[m];
}

// One family of Sec. 2.3 step 3: one thread per (line q, variable v) forms u^{FD,C} at the
// line's n + 1 flux points in registers, the flux vectors H_m = u^{FD,C} S_Dm (rows of S
// from shared memory), and adds M_D H_m to v^S_m at the line's n solution points. Family 0
// starts the sums (0 + its term), family 2 applies J^-1 and, with VSe, writes v^S out. With
// `compact`, family 0 also forms the compact face coefficients (G_CR). Ends with
// __syncthreads.
template <typename real, int N, int NV, int D>
__device__ __forceinline__ void family_gradient(real* sm, real* __restrict__ VSe, int compact) {
    using CS = CSizes<real, N, NV>;
    constexpr int NP = CS::NP, NQ = CS::NQ, NFP = CS::NFP;
    const SOps<real, N> op(sm);
    const real* su = sm + CS::G_U;
    const real* sdl = sm + CS::G_DL;
    const real* sji = sm + CS::G_JI;
    real* svs = sm + CS::G_VS;
    const real* ssf = sm + CS::G_W + D * 3 * NFP;
    real* scr = sm + CS::G_CR;
    const int tid = threadIdx.x, T = blockDim.x;
    const int nitem = NV * NQ + (D == 0 && compact ? 6 * NQ : 0);
    for (int k = tid; k < nitem; k += T) {
        if (D == 0 && k >= NV * NQ) {
            const int kf = k - NV * NQ, f = kf / NQ, q = kf - f * NQ;
            switch (f >> 1) {
                case 0: face_correction<real, N, NV, 0>(sm, f & 1, q, scr + 3 * kf); break;
                case 1: face_correction<real, N, NV, 1>(sm, f & 1, q, scr + 3 * kf); break;
                default: face_correction<real, N, NV, 2>(sm, f & 1, q, scr + 3 * kf); break;
            }
            continue;
        }
        const int v = k / NQ, q = k - v * NQ;
        real ul[N];
#pragma unroll
        for (int i = 0; i < N; ++i) ul[i] = su[v * NP + cpt<N, D>(i, q)];
        real uf[N + 1];
#pragma unroll
        for (int f = 0; f <= N; ++f) {
            real acc = op.L[f * N] * ul[0];
#pragma unroll
            for (int i = 1; i < N; ++i) acc = fma(op.L[f * N + i], ul[i], acc);
            uf[f] = acc;
        }
        uf[0] += sdl[(2 * D) * NV * NQ + v * NQ + q];
        uf[N] += sdl[(2 * D + 1) * NV * NQ + v * NQ + q];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            real h[N + 1];
#pragma unroll
            for (int f = 0; f <= N; ++f) h[f] = uf[f] * ssf[m * NFP + f * NQ + q];
            real* vs = svs + (v * 3 + m) * NP;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                real acc = op.M[i * (N + 1)] * h[0];
#pragma unroll
                for (int f = 1; f <= N; ++f) acc = fma(op.M[i * (N + 1) + f], h[f], acc);
                const int pt = cpt<N, D>(i, q);
                if (D == 0) {
                    vs[pt] = real(0) + acc;
                } else if (D == 1) {
                    vs[pt] += acc;
                } else {
                    const real x = (vs[pt] + acc) * sji[pt];
                    vs[pt] = x;
                    if (VSe) VSe[(v * 3 + m) * NP + pt] = x;
                }
            }
        }
    }
    __syncthreads();
}

// Stage element e and form v^S (Sec. 2.3 step 3): on return sm + G_VS holds v^S[v][m][pt]
// (J^-1 applied; also written to VSe unless it is null), sm + G_DL the face corrections
// delta = (u_nb - u_own)/2 [face][v][q], sm + G_JI the values of J^-1, and with `compact`
// sm + G_CR the compact face coefficients. The operators must already be staged. Ends with
// __syncthreads.
template <typename real, int N, int NV>
__device__ void element_gradient(const real* __restrict__ U, const real* __restrict__ Tc,
                                 const real* __restrict__ geo, const Mesh& g, int e, real off0, real off4,
                                 real* sm, real* __restrict__ VSe, int compact) {
    using CS = CSizes<real, N, NV>;
    constexpr int NP = CS::NP, NQ = CS::NQ;
    const SOps<real, N> op(sm);
    const int tid = threadIdx.x, T = blockDim.x;
    real* su = sm + CS::G_U;
    real* sdl = sm + CS::G_DL;
    real* sji = sm + CS::G_JI;
    real* sc = sm + CS::G_C;
    for (int k = tid; k < NGEO; k += T) sc[k] = geo[(size_t)e * NGEO + k];
    // W values per thread per pass, all loads issued before the stores (more loads in flight)
    constexpr int W = 4;
    for (int k0 = tid; k0 < NV * NP; k0 += W * T) {
        real x[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int k = k0 + j * T;
            if (k < NV * NP) {
                const int v = k / NP, pt = k - v * NP;
                x[j] = U[(size_t)v * g.nelem * NP + (size_t)e * NP + pt];
            }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int k = k0 + j * T;
            if (k < NV * NP) su[k] = x[j] - var_offset<real, NV>(k / NP, off0, off4);
        }
    }
    for (int k0 = tid; k0 < 6 * NV * NQ; k0 += W * T) {
        real own[W], nb[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int k = k0 + j * T;
            if (k < 6 * NV * NQ) {
                const int f = k / (NV * NQ), rem = k - f * NV * NQ;
                const int en = cneighbour(g, e, f >> 1, f & 1);
                own[j] = Tc[((size_t)e * 6 + f) * NV * NQ + rem];
                nb[j] = Tc[((size_t)en * 6 + (f ^ 1)) * NV * NQ + rem];
            }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const int k = k0 + j * T;
            if (k < 6 * NV * NQ) sdl[k] = real(0.5) * (nb[j] - own[j]);
        }
    }
    __syncthreads();
    // J^-1 at the solution points and the S rows of all three families at their flux points
    for (int pt = tid; pt < NP; pt += T) {
        const real r[3] = {op.xs[pt % N], op.xs[(pt / N) % N], op.xs[pt / (N * N)]};
        sji[pt] = real(1) / jacobian(sc, r);
    }
    real* ssf = sm + CS::G_W;
    for (int k = tid; k < 3 * CS::NFP; k += T) {
        const int D = k / CS::NFP, kk = k - D * CS::NFP;
        if (D == 0) metric_rows<real, N, 0>(op, sc, kk, ssf);
        else if (D == 1) metric_rows<real, N, 1>(op, sc, kk, ssf + 3 * CS::NFP);
        else metric_rows<real, N, 2>(op, sc, kk, ssf + 6 * CS::NFP);
    }
    __syncthreads();
    family_gradient<real, N, NV, 0>(sm, VSe, compact);
    family_gradient<real, N, NV, 1>(sm, VSe, compact);
    family_gradient<real, N, NV, 2>(sm, VSe, compact);
}

template <typename real, int N, int NV>
__global__ void __launch_bounds__(CURV_THREADS) k_cgrad(const real* __restrict__ U, const real* __restrict__ Tc,
                                                        const real* __restrict__ geo, real* __restrict__ VS,
                                                        real* __restrict__ Tg, const __grid_constant__ COps<real, N> o,
                                                        Mesh g, real off0, real off4, int compact) {
    using CS = CSizes<real, N, NV>;
    constexpr int NP = CS::NP, NQ = CS::NQ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sm = reinterpret_cast<real*>(smem_raw);
    const int tid = threadIdx.x, T = blockDim.x;
    stage_ops(o, sm);
    __syncthreads();
    const SOps<real, N> op(sm);
    for (int e = blockIdx.x; e < g.nelem; e += gridDim.x) {
        element_gradient<real, N, NV>(U, Tc, geo, g, e, off0, off4, sm, VS + (size_t)e * 3 * NV * NP, compact);
        const real* svs = sm + CS::G_VS;
        const real* sdl = sm + CS::G_DL;
        const real* scr = sm + CS::G_CR;
        // both faces of each line of direction d: the -d face (2d) and the +d face (2d+1)
        for (int k = tid; k < 3 * 3 * NV * NQ; k += T) {
            const int d = k / (3 * NV * NQ), rem = k - d * 3 * NV * NQ;
            const int vm = rem / NQ, q = rem - vm * NQ;
            const real* vs = svs + vm * NP;
            real lo, hi;
            switch (d) {
                case 0: face_pair<real, N, 0>(vs, op.L, op.L + N * N, q, lo, hi); break;
                case 1: face_pair<real, N, 1>(vs, op.L, op.L + N * N, q, lo, hi); break;
                default: face_pair<real, N, 2>(vs, op.L, op.L + N * N, q, lo, hi); break;
            }
            if (compact) {
                // the -d face removes the +d face's correction and vice versa
                const int v = vm / 3, m = vm - 3 * v;
                lo -= scr[3 * ((2 * d) * NQ + q) + m] * sdl[(2 * d + 1) * NV * NQ + v * NQ + q];
                hi -= scr[3 * ((2 * d + 1) * NQ + q) + m] * sdl[(2 * d) * NV * NQ + v * NQ + q];
            }
            Tg[((size_t)e * 6 + 2 * d) * 3 * NV * NQ + rem] = lo;
            Tg[((size_t)e * 6 + 2 * d + 1) * 3 * NV * NQ + rem] = hi;
        }
        __syncthreads();
    }
}

// one common flux per interface point (the -D face of element e): Fh[((D*nelem + e)*NV + v)*NQ + q]
template <typename real, int N, int NV, int D>
__device__ __forceinline__ void face_point(const real* __restrict__ Tc, const real* __restrict__ Tg,
                                           const real* __restrict__ geo, const real* __restrict__ ih,
                                           real* __restrict__ Fh, const COps<real, N>& o, const Mesh& g,
                                           const Phys<real>& P, real eta_n2, int e, int q) {
    using CS = CSizes<real, N, NV>;
    constexpr int NQ = CS::NQ;
    const int el = cneighbour(g, e, D, 0);
    const real* tl = Tc + ((size_t)el * 6 + 2 * D + 1) * NV * NQ + q;
    const real* tr = Tc + ((size_t)e * 6 + 2 * D) * NV * NQ + q;
    const real* gl = Tg + ((size_t)el * 6 + 2 * D + 1) * 3 * NV * NQ + q;
    const real* gr = Tg + ((size_t)e * 6 + 2 * D) * 3 * NV * NQ + q;
    real uL[NV], uR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        uL[v] = tl[v * NQ];
        uR[v] = tr[v * NQ];
    }
    real c[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) c[k] = geo[(size_t)e * NGEO + k];
    real rr[3], S[3];
    flux_point_coords<real, N, D>(o.xs, o.xf, 0, q, rr);
    metric_row<real, D>(c, rr, S);
    const real area = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    const real ia = real(1) / area;
    const real nv[3] = {S[0] * ia, S[1] * ia, S[2] * ia};
    const real tau = eta_n2 > real(0) ? eta_n2 * ih[(size_t)e * 3 + D] : real(0);
    // own-side gradients with the penalty tau (u_R - u_L) n added (Sec. 3, IP)
    real vl[NV * 3], vr[NV * 3];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const real pen = tau * (uR[v] - uL[v]) * nv[m];
            vl[v * 3 + m] = gl[(v * 3 + m) * NQ] + pen;
            vr[v * 3 + m] = gr[(v * 3 + m) * NQ] + pen;
        }
    real G[NV];
    if constexpr (NV == 5) {
        cv_riemann(uL, uR, nv, P, G);
#pragma unroll
        for (int k = 0; k < 5; ++k) G[k] *= area;
        if (P.vflux == 0) {
            real uh[5], vh[15], Gv[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) uh[k] = real(0.5) * (uL[k] + uR[k]);
#pragma unroll
            for (int k = 0; k < 15; ++k) vh[k] = real(0.5) * (vl[k] + vr[k]);
            cv_viscous(uh, vh, S, P, Gv);
#pragma unroll
            for (int k = 0; k < 5; ++k) G[k] -= Gv[k];
        } else {
            real Ga[5], Gb[5];
            cv_viscous(uL, vl, S, P, Ga);
            cv_viscous(uR, vr, S, P, Gb);
#pragma unroll
            for (int k = 0; k < 5; ++k) G[k] -= real(0.5) * (Ga[k] + Gb[k]);
        }
    } else {
        if (P.vflux == 0) {
            const real uh = real(0.5) * (uL[0] + uR[0]);
            real s = real(0);
#pragma unroll
            for (int m = 0; m < 3; ++m) s += S[m] * (real(0.5) * (vl[m] + vr[m]));
            G[0] = -sdk::scalar_coef(P, uh) * s;
        } else {
            real sa = real(0), sb = real(0);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                sa += S[m] * vl[m];
                sb += S[m] * vr[m];
            }
            G[0] = real(0.5) * (-sdk::scalar_coef(P, uL[0]) * sa - sdk::scalar_coef(P, uR[0]) * sb);
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) Fh[(((size_t)D * g.nelem + e) * NV + v) * NQ + q] = G[v];
}

template <typename real, int N, int NV>
__global__ void __launch_bounds__(256) k_cface(const real* __restrict__ Tc, const real* __restrict__ Tg,
                                               const real* __restrict__ geo, const real* __restrict__ ih,
                                               real* __restrict__ Fh, const __grid_constant__ COps<real, N> o,
                                               Mesh g, Phys<real> P, real eta_n2) {
    constexpr int NQ = N * N;
    const long long total = 3LL * g.nelem * NQ;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(idx % NQ);
        const long long r = idx / NQ;
        const int e = (int)(r % g.nelem);
        switch ((int)(r / g.nelem)) {
            case 0: face_point<real, N, NV, 0>(Tc, Tg, geo, ih, Fh, o, g, P, eta_n2, e, q); break;
            case 1: face_point<real, N, NV, 1>(Tc, Tg, geo, ih, Fh, o, g, P, eta_n2, e, q); break;
            default: face_point<real, N, NV, 2>(Tc, Tg, geo, ih, Fh, o, g, P, eta_n2, e, q); break;
        }
    }
}

// Flux-kernel staging of one element: u as stored (the offsets are removed where u is
// read), v^S, the interface fluxes of the six faces (face 2D holds block (D, e), the -D face;
// face 2D + 1 block (D, +D neighbour)) and the map coefficients. Two copies when they fit in
// shared memory (the next element's copies in flight while this one is computed), else one.
// After the copies: G at the interior flux points of the three families [D][v][f - 1][q]
// and J^-1 at the solution points.
template <typename real, int N, int NV>
struct CFluxPipe {
    using CS = CSizes<real, N, NV>;
    static constexpr int NP = CS::NP, NQ = CS::NQ;
    static constexpr int NI = (N - 1) * NQ;               // interior flux points of one family
    static constexpr int S_U = 0;
    static constexpr int S_VS = S_U + NV * NP;
    static constexpr int S_FH = S_VS + 3 * NV * NP;
    static constexpr int S_C = S_FH + 6 * NV * NQ;
    static constexpr int LOAD = (S_C + NGEO + 3) / 4 * 4;
    static constexpr int NG_INT = 3 * NV * NI;
    static constexpr size_t bytes_n(int nbuf) {
        return sizeof(real) * ((size_t)CS::OPS_PAD + (size_t)nbuf * LOAD + NG_INT + NP);
    }
    static constexpr int NBUF = bytes_n(2) <= 227 * 1024 ? 2 : 1;
    static constexpr size_t BYTES = bytes_n(NBUF);
};

// issue (do not wait for) the copies of element e into buf
template <typename real, int N, int NV>
__device__ __forceinline__ void cflux_issue(const real* __restrict__ U, const real* __restrict__ VS,
                                            const real* __restrict__ Fh, const real* __restrict__ geo,
                                            const Mesh& g, int e, real* buf) {
    using PL = CFluxPipe<real, N, NV>;
    constexpr int NP = PL::NP, NQ = PL::NQ;
    for (int k = threadIdx.x; k < NV * NP; k += blockDim.x) {
        const int v = k / NP, pt = k - v * NP;
        sdk::cp_async(buf + PL::S_U + k, U + (size_t)v * g.nelem * NP + (size_t)e * NP + pt);
    }
    const real* vs = VS + (size_t)e * 3 * NV * NP;
    for (int k = threadIdx.x; k < 3 * NV * NP; k += blockDim.x) sdk::cp_async(buf + PL::S_VS + k, vs + k);
    const int nb[3] = {cneighbour(g, e, 0, 1), cneighbour(g, e, 1, 1), cneighbour(g, e, 2, 1)};
    for (int k = threadIdx.x; k < 6 * NV * NQ; k += blockDim.x) {
        const int f = k / (NV * NQ), r = k - f * (NV * NQ);
        const int D = f >> 1;
        const int ee = (f & 1) ? (D == 0 ? nb[0] : (D == 1 ? nb[1] : nb[2])) : e;
        sdk::cp_async(buf + PL::S_FH + k, Fh + ((size_t)D * g.nelem + ee) * NV * NQ + r);
    }
    for (int k = threadIdx.x; k < NGEO; k += blockDim.x) sdk::cp_async(buf + PL::S_C + k, geo + (size_t)e * NGEO + k);
}

// Sec. 2.3 step 4 at interior flux point f (1..N-1) of family D on line q: G = S_D . (F_c - F_v)
// of the extrapolated state and full gradient; writes G[v] at out[v * NI]
template <typename real, int N, int NV, int D>
__device__ __forceinline__ void cflux_point(const SOps<real, N>& op, const real* buf, int f, int q,
                                            const Phys<real>& P, real off0, real off4, real* out) {
    using PL = CFluxPipe<real, N, NV>;
    constexpr int NP = PL::NP, NI = PL::NI;
    const real* su = buf + PL::S_U;
    const real* svs = buf + PL::S_VS;
    const real* Lr = op.L + f * N;
    real uF[NV], vF[3 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        real acc = Lr[0] * sdk::unoffset<real, NV>(su[v * NP + cpt<N, D>(0, q)], v, off0, off4);
#pragma unroll
        for (int i = 1; i < N; ++i)
            acc = fma(Lr[i], sdk::unoffset<real, NV>(su[v * NP + cpt<N, D>(i, q)], v, off0, off4), acc);
        uF[v] = acc;
    }
#pragma unroll
    for (int vm = 0; vm < 3 * NV; ++vm) {
        real acc = Lr[0] * svs[vm * NP + cpt<N, D>(0, q)];
#pragma unroll
        for (int i = 1; i < N; ++i) acc = fma(Lr[i], svs[vm * NP + cpt<N, D>(i, q)], acc);
        vF[vm] = acc;
    }
    real r[3], S[3];
    flux_point_coords<real, N, D>(op.xs, op.xf, f, q, r);
    metric_row<real, D>(buf + PL::S_C, r, S);
    if constexpr (NV == 5) {
        real Gc[5], Gv[5];
        cv_convective(uF, S, P, Gc);
        cv_viscous(uF, vF, S, P, Gv);
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v * NI] = Gc[v] - Gv[v];
    } else {
        out[0] = -sdk::scalar_coef(P, uF[0]) * (S[0] * vF[0] + S[1] * vF[1] + S[2] * vF[2]);
    }
}

// Sec. 2.3 step 5 for family D at solution point pt of variable v: (M_D G)[pt], the
// interface fluxes at f = 0 and f = N from the staged face blocks
template <typename real, int N, int NV, int D>
__device__ __forceinline__ real cflux_div(const SOps<real, N>& op, const real* buf, const real* sG, int v,
                                          int pt) {
    using PL = CFluxPipe<real, N, NV>;
    constexpr int NQ = PL::NQ, NI = PL::NI;
    int i, q;
    line_of<N, D>(pt, i, q);
    const real* Mr = op.M + i * (N + 1);
    const real* gi = sG + (D * NV + v) * NI + q;
    real acc = Mr[0] * buf[PL::S_FH + ((2 * D) * NV + v) * NQ + q];
#pragma unroll
    for (int f = 1; f < N; ++f) acc = fma(Mr[f], gi[(f - 1) * NQ], acc);
    return fma(Mr[N], buf[PL::S_FH + ((2 * D + 1) * NV + v) * NQ + q], acc);
}

// Persistent: block b handles elements b, b + grid, ... Per element: J^-1 at the solution
// points and G at the interior flux points of all three families (one pass, so the threads
// are busy across families), one barrier, then R = -J^-1 sum_d M_d G with the families
// subtracted in the order x, y, z. Two barriers per element (the copies' wait and the one
// after G).
template <typename real, int N, int NV>
__global__ void __launch_bounds__(CURV_THREADS, sizeof(real) == 4 ? 3 : 1) k_cflux(const real* __restrict__ U, const real* __restrict__ VS,
                                                        const real* __restrict__ Fh, const real* __restrict__ geo,
                                                        real* __restrict__ R, const __grid_constant__ COps<real, N> o,
                                                        Mesh g, Phys<real> P, real off0, real off4) {
    using CS = CSizes<real, N, NV>;
    using PL = CFluxPipe<real, N, NV>;
    constexpr int NP = CS::NP, NI = PL::NI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sm = reinterpret_cast<real*>(smem_raw);
    real* buf0 = sm + CS::OPS_PAD;
    real* buf1 = buf0 + (PL::NBUF - 1) * PL::LOAD;
    real* sG = buf0 + PL::NBUF * PL::LOAD;
    real* sji = sG + PL::NG_INT;
    const int tid = threadIdx.x, T = blockDim.x;
    int e = blockIdx.x;
    if (e >= g.nelem) return;
    stage_ops(o, sm);
    if constexpr (PL::NBUF == 2) {
        cflux_issue<real, N, NV>(U, VS, Fh, geo, g, e, buf0);
        sdk::cp_async_commit();
    }
    const SOps<real, N> op(sm);
    for (int b = 0; e < g.nelem; e += gridDim.x, b ^= 1) {
        real* buf = b ? buf1 : buf0;
        if constexpr (PL::NBUF == 1) {
            if (e != (int)blockIdx.x) __syncthreads();      // the previous element's reads are done
            cflux_issue<real, N, NV>(U, VS, Fh, geo, g, e, buf);
            sdk::cp_async_commit();
        }
        sdk::cp_async_wait_group<0>();
        __syncthreads();
        if constexpr (PL::NBUF == 2) {
            const int en = e + gridDim.x;
            if (en < g.nelem) {
                cflux_issue<real, N, NV>(U, VS, Fh, geo, g, en, b ? buf0 : buf1);
                sdk::cp_async_commit();
            }
        }
        const real* sc = buf + PL::S_C;
        for (int pt = tid; pt < NP; pt += T) {
            const real r[3] = {op.xs[pt % N], op.xs[(pt / N) % N], op.xs[pt / (N * N)]};
            sji[pt] = real(1) / jacobian(sc, r);
        }
        for (int k = tid; k < 3 * NI; k += T) {
            const int D = k / NI, rr = k - D * NI;
            const int f = 1 + rr / CS::NQ, q = rr - (f - 1) * CS::NQ;
            real* out = sG + D * NV * NI + rr;
            if (D == 0) cflux_point<real, N, NV, 0>(op, buf, f, q, P, off0, off4, out);
            else if (D == 1) cflux_point<real, N, NV, 1>(op, buf, f, q, P, off0, off4, out);
            else cflux_point<real, N, NV, 2>(op, buf, f, q, P, off0, off4, out);
        }
        __syncthreads();
        for (int k = tid; k < NV * NP; k += T) {
            const int v = k / NP, pt = k - v * NP;
            real r = real(0);
            r -= cflux_div<real, N, NV, 0>(op, buf, sG, v, pt);
            r -= cflux_div<real, N, NV, 1>(op, buf, sG, v, pt);
            r -= cflux_div<real, N, NV, 2>(op, buf, sG, v, pt);
            R[(size_t)v * g.nelem * NP + (size_t)e * NP + pt] = r * sji[pt];
        }
    }
}

// FP64 volume diagnostics on the curved grid: block b handles elements b*epb .. b*epb+epb-1
// and writes one row of NDIAG partial sums (same quantities and order as the Cartesian
// diagnostics, with the quadrature weights J w_i w_j w_k)
template <int N, int NV>
__global__ void __launch_bounds__(CURV_THREADS) k_cdiag(const double* __restrict__ U, const double* __restrict__ Tc,
                                                        const double* __restrict__ geo,
                                                        const __grid_constant__ COps<double, N> o, Mesh g,
                                                        const double* __restrict__ wq, int epb,
                                                        double* __restrict__ partial) {
    using CS = CSizes<double, N, NV>;
    constexpr int NP = CS::NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* sm = reinterpret_cast<double*>(smem_raw);
    stage_ops(o, sm);
    __syncthreads();
    double acc[sdk::NDIAG];
#pragma unroll
    for (int k = 0; k < sdk::NDIAG; ++k) acc[k] = 0.0;
    for (int le = 0; le < epb; ++le) {
        const int e = blockIdx.x * epb + le;
        if (e >= g.nelem) break;
        element_gradient<double, N, NV>(U, Tc, geo, g, e, 0.0, 0.0, sm, nullptr, 0);
        const double* su = sm + CS::G_U;
        const double* vS = sm + CS::G_VS;
        const double* sji = sm + CS::G_JI;
        for (int pt = threadIdx.x; pt < NP; pt += blockDim.x) {
            const double w = wq[pt % N] * wq[(pt / N) % N] * wq[pt / (N * N)] / sji[pt];
            bool bad = false;
#pragma unroll
            for (int v = 0; v < NV; ++v) bad |= !isfinite(su[v * NP + pt]);
            acc[9] += bad ? 1.0 : 0.0;
            if constexpr (NV == 5) {
                const double rho = su[pt];
                const double vel[3] = {su[NP + pt] / rho, su[2 * NP + pt] / rho, su[3 * NP + pt] / rho};
                const double q2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2];
                double du[3][3];   // du[i][k] = d u_i / d x_k
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        du[i][k] = (vS[((1 + i) * 3 + k) * NP + pt] - vel[i] * vS[k * NP + pt]) / rho;
                const double o0 = du[2][1] - du[1][2], o1 = du[0][2] - du[2][0], o2 = du[1][0] - du[0][1];
                acc[0] += w * 0.5 * q2;
                acc[1] += w * 0.5 * rho * q2;
                acc[2] += w * (o0 * o0 + o1 * o1 + o2 * o2);
                acc[3] += w * rho;
                acc[4] += w * su[NP + pt];
                acc[5] += w * su[2 * NP + pt];
                acc[6] += w * su[3 * NP + pt];
                acc[7] += w * su[4 * NP + pt];
            } else {
                const double u = su[pt];
                acc[3] += w * u;
                acc[8] += w * u * u;
            }
        }
        __syncthreads();
    }
    // deterministic block reduction (fixed tree over the threads); the operators staged at
    // the front of shared memory are no longer needed
    double* red = sm;
    for (int k = 0; k < sdk::NDIAG; ++k) red[k * blockDim.x + threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = 1; s < (int)blockDim.x; s <<= 1) {
        if ((threadIdx.x % (2 * s)) == 0 && threadIdx.x + s < blockDim.x)
            for (int k = 0; k < sdk::NDIAG; ++k) red[k * blockDim.x + threadIdx.x] += red[k * blockDim.x + threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < sdk::NDIAG; ++k) partial[(size_t)blockIdx.x * sdk::NDIAG + k] = red[k * blockDim.x];
}

// ------------------------------------------------------------------ host side
template <typename real, int N>
static COps<real, N> make_cops(const sd_ctx* c) {
    COps<real, N> o;
    for (int k = 0; k < (N + 1) * N; ++k) o.L[k] = (real)c->L[k];
    for (int k = 0; k < N * (N + 1); ++k) o.M[k] = (real)c->M[k];
    for (int i = 0; i < N; ++i) o.xs[i] = (real)c->xs[i];
    for (int f = 0; f <= N; ++f) o.xf[f] = (real)c->xf[f];
    return o;
}

inline Mesh cmesh(const sd_ctx* c) {
    Mesh g;
    for (int d = 0; d < 3; ++d) g.ne[d] = c->ne[d];
    g.nelem = c->nelem;
    g.e_begin = 0;
    g.e_end = c->nelem;
    for (int d = 0; d < 3; ++d) {
        g.olo[d] = 0;
        g.ohi[d] = c->ne[d];
    }
    return g;
}

inline int flat_blocks(long long total) {
    const long long b = (total + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(b, 1), 148LL * 64);
}

inline int elem_threads(int n) {
    const int nfp = (n + 1) * n * n;
    return std::min(CURV_THREADS, std::max(64, (nfp + 31) / 32 * 32));
}

template <typename real, int N, int NV>
static sd_status residual_impl(sd_ctx* c, const real* U, real* R, int offset_in) {
    using CS = CSizes<real, N, NV>;
    const COps<real, N> o = make_cops<real, N>(c);
    const Mesh g = cmesh(c);
    const Phys<real> P = sdk::make_phys<real>(c);
    double d0 = 0.0, d4 = 0.0;
    if (c->nvar == 5 && !offset_in) {
        const double p0 = c->phys.rho0 * (c->phys.u0 / c->phys.Ma) * (c->phys.u0 / c->phys.Ma) / c->phys.gamma;
        d0 = c->phys.rho0;
        d4 = p0 / (c->phys.gamma - 1.0);
    }
    const real off0 = (real)d0, off4 = (real)d4;
    real* Tc = static_cast<real*>(c->Tu);
    real* Tg = static_cast<real*>(c->cTg);
    real* Fh = static_cast<real*>(c->Fh);
    real* VS = static_cast<real*>(c->cvs);
    const real* geo = static_cast<const real*>(c->cgeo);
    const real* ih = static_cast<const real*>(c->cih);
    const size_t sg = (size_t)CS::GRAD * sizeof(real);
    const size_t sf = CFluxPipe<real, N, NV>::BYTES;
    if (!sdk::set_smem(k_cgrad<real, N, NV>, sg) || !sdk::set_smem(k_cflux<real, N, NV>, sf)) {
        sdi_set_error("curvilinear kernels need %zu / %zu bytes of shared memory", sg, sf);
        return SD_EUNSUPPORTED;
    }
    const int th = elem_threads(N);
    const int eb = std::min(c->nelem, 1 << 30);
    sdi_prof_begin(c, SD_K_TRACE);
    k_ctrace<real, N, NV><<<std::min(c->nelem, 148 * 32), 128, 0, c->stream>>>(U, Tc, o, g, off0, off4);
    sdi_prof_end(c, SD_K_TRACE);
    sdi_prof_begin(c, SD_K_GRAD);
    k_cgrad<real, N, NV><<<eb, th, sg, c->stream>>>(U, Tc, geo, VS, Tg, o, g, off0, off4,
                                                    c->scheme == SD_COMPACT ? 1 : 0);
    sdi_prof_end(c, SD_K_GRAD);
    const real eta_n2 = (real)(c->phys.eta_ip * c->n * c->n);
    sdi_prof_begin(c, SD_K_FACE);
    k_cface<real, N, NV><<<flat_blocks(3LL * c->nelem * CS::NQ), 256, 0, c->stream>>>(Tc, Tg, geo, ih, Fh, o, g, P,
                                                                                     eta_n2);
    sdi_prof_end(c, SD_K_FACE);
    sdi_prof_begin(c, SD_K_FLUX);
    const int fb = sdk::persistent_grid(k_cflux<real, N, NV>, th, sf, c->nelem, c->device);
    k_cflux<real, N, NV><<<fb, th, sf, c->stream>>>(U, VS, Fh, geo, R, o, g, P, off0, off4);
    sdi_prof_end(c, SD_K_FLUX);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        sdi_set_error("curvilinear residual launch failed: %s", cudaGetErrorString(err));
        return SD_ECUDA;
    }
    return SD_OK;
}

template <typename real>
static sd_status residual_dispatch(sd_ctx* c, const real* U, real* R, int offset_in) {
    const bool ns = c->nvar == 5;
#define SDC_CASE(n_)                                                                                   \
    case n_:                                                                                           \
        return ns ? residual_impl<real, n_, 5>(c, U, R, offset_in) : residual_impl<real, n_, 1>(c, U, R, offset_in);
    switch (c->n) {
        SDC_CASE(2)
        SDC_CASE(3)
        SDC_CASE(4)
        SDC_CASE(5)
        SDC_CASE(6)
        SDC_CASE(7)
        SDC_CASE(8)
        SDC_CASE(9)
        default: return SD_EUNSUPPORTED;
    }
#undef SDC_CASE
}

template <int N, int NV>
static sd_status diag_impl(sd_ctx* c, const double* U) {
    using CS = CSizes<double, N, NV>;
    const COps<double, N> o = make_cops<double, N>(c);
    const Mesh g = cmesh(c);
    sdi_prof_begin(c, SD_K_OTHER);
    k_ctrace<double, N, NV><<<std::min(c->nelem, 148 * 32), 128, 0, c->stream>>>(U, c->Tu64, o, g, 0.0, 0.0);
    sdi_prof_end(c, SD_K_OTHER);
    const int th = elem_threads(N);
    const size_t smem = std::max<size_t>((size_t)CS::GRAD, (size_t)sdk::NDIAG * th) * sizeof(double);
    if (!sdk::set_smem(k_cdiag<N, NV>, smem)) return SD_EUNSUPPORTED;
    const int epb = (c->nelem + c->diag_blocks - 1) / c->diag_blocks;
    const int nb = (c->nelem + epb - 1) / epb;
    if (nb > c->diag_blocks) return SD_EINVAL;
    sdi_prof_begin(c, SD_K_OTHER);
    k_cdiag<N, NV><<<nb, th, smem, c->stream>>>(U, c->Tu64, c->cgeo64, o, g, c->dW, epb, c->partial);
    sdi_prof_end(c, SD_K_OTHER);
    c->diag_nb = nb;
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        sdi_set_error("curvilinear diagnostics launch failed: %s", cudaGetErrorString(err));
        return SD_ECUDA;
    }
    return SD_OK;
}

}  // namespace sdc

sd_status sdi_curv_residual_f32(sd_ctx* c, const float* U, float* R, int offset_in) {
    return sdc::residual_dispatch<float>(c, U, R, offset_in);
}

sd_status sdi_curv_residual_f64(sd_ctx* c, const double* U, double* R, int offset_in) {
    return sdc::residual_dispatch<double>(c, U, R, offset_in);
}

sd_status sdi_curv_diag_partials(sd_ctx* c, const double* U64) {
    const bool ns = c->nvar == 5;
    switch (c->n) {
        case 2: return ns ? sdc::diag_impl<2, 5>(c, U64) : sdc::diag_impl<2, 1>(c, U64);
        case 3: return ns ? sdc::diag_impl<3, 5>(c, U64) : sdc::diag_impl<3, 1>(c, U64);
        case 4: return ns ? sdc::diag_impl<4, 5>(c, U64) : sdc::diag_impl<4, 1>(c, U64);
        case 5: return ns ? sdc::diag_impl<5, 5>(c, U64) : sdc::diag_impl<5, 1>(c, U64);
        case 6: return ns ? sdc::diag_impl<6, 5>(c, U64) : sdc::diag_impl<6, 1>(c, U64);
        case 7: return ns ? sdc::diag_impl<7, 5>(c, U64) : sdc::diag_impl<7, 1>(c, U64);
        case 8: return ns ? sdc::diag_impl<8, 5>(c, U64) : sdc::diag_impl<8, 1>(c, U64);
        case 9: return ns ? sdc::diag_impl<9, 5>(c, U64) : sdc::diag_impl<9, 1>(c, U64);
        default: return SD_EUNSUPPORTED;
    }
}

// ------------------------------------------------------------------ grid set-up
// Reads the corner nodes, checks the periodic images and the Jacobian, and uploads the map
// coefficients (residual precision and FP64) and the interior-penalty scales.
sd_status sdi_curv_setup(sd_ctx* c, const double* nodes) {
    const int nx = c->ne[0], ny = c->ne[1], nz = c->ne[2];
    const int n = c->n;
    auto node = [&](int comp, int k, int j, int i) -> double {
        return nodes[(((size_t)comp * (nz + 1) + k) * (ny + 1) + j) * (nx + 1) + i];
    };
    // periodic images: one translation vector per axis
    double Tv[3][3];
    for (int comp = 0; comp < 3; ++comp) {
        Tv[0][comp] = node(comp, 0, 0, nx) - node(comp, 0, 0, 0);
        Tv[1][comp] = node(comp, 0, ny, 0) - node(comp, 0, 0, 0);
        Tv[2][comp] = node(comp, nz, 0, 0) - node(comp, 0, 0, 0);
    }
    double scale = 0.0;
    for (int a = 0; a < 3; ++a)
        scale = std::max(scale, std::sqrt(Tv[a][0] * Tv[a][0] + Tv[a][1] * Tv[a][1] + Tv[a][2] * Tv[a][2]));
    if (!(scale > 0.0) || !std::isfinite(scale)) {
        sdi_set_error("degenerate or non-finite node coordinates");
        return SD_EINVAL;
    }
    const double tol = 1e-10 * scale;
    for (int comp = 0; comp < 3; ++comp) {
        for (int k = 0; k <= nz; ++k)
            for (int j = 0; j <= ny; ++j)
                if (std::fabs(node(comp, k, j, nx) - node(comp, k, j, 0) - Tv[0][comp]) > tol) {
                    sdi_set_error("node (x=%d, y=%d, z=%d) is not the periodic image of (0, %d, %d)", nx, j, k, j, k);
                    return SD_EINVAL;
                }
        for (int k = 0; k <= nz; ++k)
            for (int i = 0; i <= nx; ++i)
                if (std::fabs(node(comp, k, ny, i) - node(comp, k, 0, i) - Tv[1][comp]) > tol) {
                    sdi_set_error("node (x=%d, y=%d, z=%d) is not the periodic image of (%d, 0, %d)", i, ny, k, i, k);
                    return SD_EINVAL;
                }
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i)
                if (std::fabs(node(comp, nz, j, i) - node(comp, 0, j, i) - Tv[2][comp]) > tol) {
                    sdi_set_error("node (x=%d, y=%d, z=%d) is not the periodic image of (%d, %d, 0)", i, j, nz, i, j);
                    return SD_EINVAL;
                }
    }
    const size_t E = (size_t)c->nelem;
    std::vector<double> geo(E * sdc::NGEO, 0.0);
    std::vector<double> vol(E, 0.0);
    const double* xs = c->xs;
    const double* ws = c->ws;
    auto tang = [](const double* cf, double x, double y, double z, double a[3][3]) {
        for (int k = 0; k < 3; ++k) {
            a[0][k] = cf[k] + cf[9 + k] * y + cf[15 + k] * z + cf[18 + k] * y * z;
            a[1][k] = cf[3 + k] + cf[9 + k] * x + cf[12 + k] * z + cf[18 + k] * x * z;
            a[2][k] = cf[6 + k] + cf[12 + k] * y + cf[15 + k] * x + cf[18 + k] * x * y;
        }
    };
    auto crs = [](const double* u, const double* v, double* w) {
        w[0] = u[1] * v[2] - u[2] * v[1];
        w[1] = u[2] * v[0] - u[0] * v[2];
        w[2] = u[0] * v[1] - u[1] * v[0];
    };
    for (int ez = 0; ez < nz; ++ez)
        for (int ey = 0; ey < ny; ++ey)
            for (int ex = 0; ex < nx; ++ex) {
                const size_t e = ((size_t)ez * ny + ey) * nx + ex;
                double* cf = geo.data() + e * sdc::NGEO;
                for (int comp = 0; comp < 3; ++comp) {
                    long double s[7] = {0, 0, 0, 0, 0, 0, 0};
                    for (int cc = 0; cc < 2; ++cc)
                        for (int b = 0; b < 2; ++b)
                            for (int a = 0; a < 2; ++a) {
                                const long double x = node(comp, ez + cc, ey + b, ex + a);
                                const int sa = 2 * a - 1, sb = 2 * b - 1, sc = 2 * cc - 1;
                                s[0] += sa * x;            // xi
                                s[1] += sb * x;            // eta
                                s[2] += sc * x;            // zeta
                                s[3] += sa * sb * x;       // xi eta
                                s[4] += sb * sc * x;       // eta zeta
                                s[5] += sa * sc * x;       // xi zeta
                                s[6] += sa * sb * sc * x;  // xi eta zeta
                            }
                    for (int t = 0; t < 7; ++t) cf[3 * t + comp] = (double)(s[t] / 8.0L);
                }
                double V = 0.0;
                for (int k = 0; k < n; ++k)
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i) {
                            double a[3][3], s3[3];
                            tang(cf, xs[i], xs[j], xs[k], a);
                            crs(a[1], a[2], s3);
                            const double J = a[0][0] * s3[0] + a[0][1] * s3[1] + a[0][2] * s3[2];
                            if (!(J > 0.0)) {
                                sdi_set_error("element (%d, %d, %d) has a non-positive Jacobian at a solution point",
                                              ex, ey, ez);
                                return SD_EINVAL;
                            }
                            V += ws[i] * ws[j] * ws[k] * J;
                        }
                vol[e] = V;
            }
    // interior-penalty scale of the -d face of each element: |A_f| / min(V_e, V_{e-d}),
    // A_f = 4 S_d at the face centre (S_d is bilinear on the face, so this is its integral)
    std::vector<double> ih(E * 3, 0.0);
    double vtot = 0.0;
    for (int ez = 0; ez < nz; ++ez)
        for (int ey = 0; ey < ny; ++ey)
            for (int ex = 0; ex < nx; ++ex) {
                const size_t e = ((size_t)ez * ny + ey) * nx + ex;
                vtot += vol[e];
                const double* cf = geo.data() + e * sdc::NGEO;
                for (int d = 0; d < 3; ++d) {
                    double r[3] = {0.0, 0.0, 0.0};
                    r[d] = -1.0;
                    double a[3][3], S[3];
                    tang(cf, r[0], r[1], r[2], a);
                    crs(a[(d + 1) % 3], a[(d + 2) % 3], S);
                    const double area = 4.0 * std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
                    int cidx[3] = {ex, ey, ez};
                    cidx[d] = (cidx[d] + c->ne[d] - 1) % c->ne[d];
                    const size_t en = ((size_t)cidx[2] * ny + cidx[1]) * nx + cidx[0];
                    ih[e * 3 + d] = area / std::min(vol[e], vol[en]);
                }
            }
    c->curv_volume = vtot;
    bool ok = true;
    auto alloc = [&](void** p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) ok = false;
    };
    const int NV = c->nvar, np = n * n * n, nq = n * n;
    alloc((void**)&c->cgeo64, E * sdc::NGEO * sizeof(double));
    if (c->prec == SD_F32) alloc(&c->cgeo, E * sdc::NGEO * sizeof(float));
    alloc(&c->cih, E * 3 * c->esize);
    alloc(&c->cvs, E * 3 * NV * np * c->esize);
    alloc(&c->cTg, E * 6 * 3 * NV * nq * c->esize);
    if (!ok) {
        cudaGetLastError();
        sdi_set_error("device allocation of the curvilinear grid data failed");
        return SD_ENOMEM;
    }
    if (c->prec == SD_F64) c->cgeo = c->cgeo64;
    cudaError_t err = cudaMemcpy(c->cgeo64, geo.data(), E * sdc::NGEO * sizeof(double), cudaMemcpyHostToDevice);
    if (err == cudaSuccess && c->prec == SD_F32) {
        std::vector<float> gf(geo.begin(), geo.end());
        err = cudaMemcpy(c->cgeo, gf.data(), E * sdc::NGEO * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (err == cudaSuccess) {
        if (c->prec == SD_F32) {
            std::vector<float> hf(ih.begin(), ih.end());
            err = cudaMemcpy(c->cih, hf.data(), E * 3 * sizeof(float), cudaMemcpyHostToDevice);
        } else {
            err = cudaMemcpy(c->cih, ih.data(), E * 3 * sizeof(double), cudaMemcpyHostToDevice);
        }
    }
    if (err != cudaSuccess) {
        sdi_set_error("upload of the curvilinear grid data failed: %s", cudaGetErrorString(err));
        return SD_ECUDA;
    }
    // the Cartesian gradient-trace buffer is not used on a curved grid (cTg replaces it)
    cudaFree(c->Tg);
    c->Tg = nullptr;
    c->curv = 1;
    return SD_OK;
}
