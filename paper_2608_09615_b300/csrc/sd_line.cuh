// Line-blocked residual kernels (the production path of sd_residual).
//
// Work decomposition. A block holds EB elements in shared memory. Direction-structured
// phases assign one warp (WPD warps when a face has more than 32 points) per direction
// per element group; inside it each lane owns one line of n points along that direction
// (lanes index the face point q, and for small n several elements share a warp). The
// direction is a template parameter, so every index into the per-thread arrays below is a
// compile-time constant and the arrays live in registers. A lane loads its line once and
// produces all n+1 flux-point values, the fluxes there and the divergence contribution
// to the n points of the line. The flux-point loop is not unrolled (its operator rows,
// with the grid metric folded in, are a __grid_constant__ kernel parameter), which keeps
// one copy of the flux code per direction.
//
// Kernels per residual (Sec. 2.3 steps 1-5):
//   k_line_trace  u at the 2*DIM faces (step 1, interface rows)            -> Tu
//   k_line_grad   common-solution corrections, v^S (Eq. w:e), own interface
//                 gradients (BR1 Eq. v:e / compact closed form)            -> Tg
//   k_face_flux   one thread per interface point, each interface once: the
//                 Riemann flux of the two traces minus the viscous flux of the
//                 averaged state and averaged gradient (Eqs. c:aux:v:2d, Sec. 4.4) -> Fh
//   k_line_flux   interior gradients (Eq. aux:v:std:2d), interior fluxes
//                 (Sec. 4.4 / Eq. pme) and the divergence with the interface
//                 fluxes Fh at the line ends                               -> R
// The three directions of k_line_flux add into R in the fixed order x, y, z, so results
// are deterministic. The interface flux is computed once per interface point, so it is
// single-valued and conservation holds to round-off.
//
// Navier-Stokes states enter the arithmetic with the reference offsets removed from rho and
// rho E (see ns_convective): as each lane loads its line, or in one pass over the staged
// values (see pipe_next); Tu holds traces of the offset state.
#pragma once

#include "sd_kernels.cuh"

// Threads per block the line kernels aim for (whole element groups of DIM warps): 96 for
// the trace and gradient kernels (one element group per block at n = 5, so a barrier waits
// for three warps; at 48^3 the gradient kernel measured 0.284 ms against 0.300 with 192
// threads and 0.307 with 384, the trace kernel 0.133 against 0.136), and 96 for
// k_line_flux with a register cap of 136 (further limited to what one block of the layout
// can use). For the FP32 Navier-Stokes n = 5 case on B300 this gives 5 resident flux
// blocks per SM without spills; it measured fastest among the layouts tried (on an
// earlier form of the kernel, per launch at 48^3: 192 threads / 143 registers 1.24 ms,
// 96 / 136 1.11 ms, 192 / 112 1.25 ms).
#ifndef SD_LINE_THREADS
#define SD_LINE_THREADS 96
#endif
#ifndef SD_FLUX_THREADS
#define SD_FLUX_THREADS 96
#endif
#ifndef SD_FLUX_MAXNREG
#define SD_FLUX_MAXNREG 136
#endif


namespace sdk {

// 1D operators of one n, in constant memory (uploaded once per device by the
// translation unit that launches the kernels).
template <typename real, int N>
struct OpTab {
    real L[(N + 1) * N];     // L[f*N + i]     = l_i(xi_{f-1/2})          (Eq. Lmat)
    real M[N * (N + 1)];     // M[i*(N+1) + f] = l'_{f-1/2}(xi_i)         (Eq. Mmat)
    real D[N * N];           // D = M L
    real LD[(N + 1) * N];    // LD[f*N + i] = (L D)[f][i]
    real LM0[N + 1];         // (L M)[f][0]
    real LMN[N + 1];         // (L M)[f][N]
};

template <typename real, int N>
__constant__ OpTab<real, N> c_op;

// per-grid scalars of the line kernels
template <typename real>
struct LineGeo {
    real two_h[3];           // 2/h_d
    real corrL[3];           // (2/h_d) alpha
    real corrR[3];           // (2/h_d) beta
    real off0, off4;         // offsets removed from variables 0 and 4 when staging
    real tip[3];             // interior penalty eta (p+1)^2 / h_d (0: off)
};

// Operator rows of the flux kernel with the grid's metric folded in, per direction d (a
// kernel parameter, read from the constant bank by the flux-point loop, so no per-point
// scaling by 2/h_d is left in the loop): the divergence weights -(2/h_d) M and the
// normal-derivative rows (2/h_d) L D, (2/h_d) (L M)[:,0], (2/h_d) (L M)[:,N] at the flux
// points.
template <typename real, int N>
struct FluxOps {
    real Mn[3][N][N + 1];    // -(2/h_d) M[i][f]
    real LDn[3][N + 1][N];   // (2/h_d) (L D)[f][i]
    real LM0n[3][N + 1];     // (2/h_d) (L M)[f][0]
    real LMNn[3][N + 1];     // (2/h_d) (L M)[f][N]
};

constexpr int round4(int x) { return (x + 3) / 4 * 4; }

template <int N, int DIM, int NV, int TGT = SD_LINE_THREADS>
struct LineLayout {
    static constexpr int NP = ipow(N, DIM);
    static constexpr int NQ = ipow(N, DIM - 1);
    static constexpr int NF = 2 * DIM;
    static constexpr int NG = NumGrad<NV>::value;
    static constexpr int EPW = NQ <= 32 ? 32 / NQ : 1;            // elements per warp
    static constexpr int WPD = NQ <= 32 ? 1 : (NQ + 31) / 32;     // warps per direction
    static constexpr int UNIT = DIM * WPD * 32;                   // threads per element group
    static constexpr int UPB = UNIT >= TGT ? 1 : TGT / UNIT;      // groups per block
    static constexpr int THREADS = UPB * UNIT;
    static constexpr int EB = UPB * EPW;                          // elements per block
    // Global scratch layouts: Tu[e][f][FST] and Fh[d][e][FST] hold [v][q] in the first NV*NQ
    // values of each block (scalars: then the diffusivity traces [q], see FST), Tg[e][f][GST] holds [c][q]; blocks are padded to a multiple of
    // 4 values so that each starts on a 16-byte boundary and is copied in 16-byte pieces.
    // (scalar blocks also hold the face traces of the porous-medium diffusivity at [NQ, 2 NQ))
    static constexpr int FST = round4(NV * NQ + (NV == 1 ? NQ : 0));
    static constexpr int GST = round4(NG * NQ);
    // per-element sizes of the contiguous element staging of the closure kernels
    static constexpr int S_U = NV * NP;
    static constexpr int S_TR = NF * NV * NQ;
    static constexpr int S_VS = NV * DIM * NP;
    // v^S components the residual kernels keep (vslot): 9 for Navier-Stokes, none for scalars
    static constexpr int S_VR = (NV == 5 ? 9 : 0) * NP;
    // per-direction residual contributions R_d[v][pt] (flux kernel, in its work area)
    static constexpr int S_RD = DIM * NV * NP;
    static constexpr int PER_GRAD = S_U + 2 * S_TR + S_VS;
    static constexpr int NBR_BYTES = ((EB * NF * 4 + 15) / 16) * 16;   // neighbour table
    static constexpr int REG_FIT = (65536 / THREADS) / 8 * 8;
    static constexpr int FLUX_REGS = SD_FLUX_MAXNREG < REG_FIT ? SD_FLUX_MAXNREG : (REG_FIT < 255 ? REG_FIT : 255);
};

// Strides of the staged arrays as the line functions see them: US between the variables
// of u, FS between the faces of the trace (and interface flux) arrays; within a face the
// layout is [v][q]. The residual kernels stage u variable-major over the block's elements
// (US = EB NP) and traces in the padded global face blocks (FS = FST); the closure
// kernels stage each element contiguously (US = NP, FS = NV NQ).
template <int US_, int FS_>
struct Strides {
    static constexpr int US = US_;
    static constexpr int FS = FS_;
};

// element groups of a launch: EB consecutive elements each, over [e_begin, e_end)
template <int EB>
__device__ __forceinline__ int num_groups(const Mesh& g) {
    return (g.e_end - g.e_begin + EB - 1) / EB;
}
template <int EB>
__device__ __forceinline__ int grp_first(const Mesh& g, int grp) {
    return g.e_begin + grp * EB;
}
template <int EB>
__device__ __forceinline__ int grp_count(const Mesh& g, int grp) {
    return min(EB, g.e_end - (g.e_begin + grp * EB));
}

struct LineId {
    int d;      // direction of this warp
    int eb;     // element slot in the block
    int q;      // face point index of the lane's line
    bool ok;    // lane carries a line
};

template <class LL>
__device__ __forceinline__ LineId line_id(int tid) {
    const int unit = tid / LL::UNIT;
    const int t = tid - unit * LL::UNIT;
    LineId r;
    r.d = t / (LL::WPD * 32);
    const int w = (t >> 5) % LL::WPD;
    const int lane = t & 31;
    if (LL::EPW > 1) {
        const int eu = lane / LL::NQ;
        r.q = lane - eu * LL::NQ;
        r.eb = unit * LL::EPW + eu;
        r.ok = eu < LL::EPW;
    } else {
        r.q = lane + 32 * w;
        r.eb = unit;
        r.ok = r.q < LL::NQ;
    }
    return r;
}

// point index of position i along compile-time direction D on line q
template <int N, int D>
__device__ __forceinline__ int lpt(int i, int q) {
    constexpr int lo = ipow(N, D);
    return (q % lo) + lo * i + lo * N * (q / lo);
}

// sum_i row[i] * x[i], one fixed fma sequence (row from constant memory)
template <typename real, int N>
__device__ __forceinline__ real dotc(const real* row, const real* x) {
    real s = row[0] * x[0];
#pragma unroll
    for (int i = 1; i < N; ++i) s = fma(row[i], x[i], s);
    return s;
}

// Slot of the v^S component (variable v, derivative direction m) the residual kernels
// keep: the derivative along m of rho and of the two momentum components across m. These
// are the transverse gradient components the lines of the other two directions need (the
// viscous flux along d uses d/dx_t of rho and rho u_d, t != d); a line's own normal
// derivatives are evaluated from u directly (dline).
__host__ __device__ constexpr int vslot(int v, int m) {
    return v == 0 ? 3 * m : (v - 1 == (m + 1) % 3 ? 3 * m + 1 : 3 * m + 2);
}

// derivative along the line of the variable with line values u[] at flux point f:
// L_f v = (2/h) L_f (D u + M[:,0] dl + M[:,N] dr) = (2/h) ((L D)_f u + (L M)_{f0} dl + (L M)_{fN} dr)
template <typename real, int N>
__device__ __forceinline__ real dline(const OpTab<real, N>& op, int f, const real* u, real dl, real dr,
                                      real two_h) {
    real a = dotc<real, N>(op.LD + f * N, u);
    a = fma(op.LM0[f], dl, a);
    a = fma(op.LMN[f], dr, a);
    return two_h * a;
}

// ---------------------------------------------------------------- staging helpers
// asynchronous global -> shared copy of one value (Ampere-style cp.async)
template <typename real>
__device__ __forceinline__ void cp_async(real* smem, const real* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(real) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// asynchronous copy of 16 bytes; both addresses must be 16-byte aligned
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// wait until at most NPEND of this thread's committed copy groups are still in flight
template <int NPEND>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// Contiguous element staging used by the closure kernels: u (offsets removed unless the
// input already carries them) and the neighbour traces of EB elements, each element's data
// at sm + eb * per in the layout Strides<NP, NV NQ>. Ends with a barrier.
template <typename real, class LL, int NV>
__device__ __forceinline__ void stage_load(const real* __restrict__ U, const real* __restrict__ Tu,
                                           const Mesh& g, int e0, real* sm, int per, real off0, real off4,
                                           int* nbr) {
    constexpr int NP = LL::NP, NQ = LL::NQ, NF = LL::NF;
    const int nloc = min(LL::EB, g.nelem - e0);
    for (int k = threadIdx.x; k < nloc * NF; k += blockDim.x) {
        const int eb = k / NF, f = k - eb * NF;
        nbr[k] = neighbour(g, e0 + eb, f >> 1, f & 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nloc * NV * NP; k += blockDim.x) {
        const int eb = k / (NV * NP);
        const int r = k - eb * NV * NP;
        const int v = r / NP, pt = r - v * NP;
        cp_async(&sm[eb * per + r], &U[(size_t)v * g.nelem * NP + (size_t)(e0 + eb) * NP + pt]);
    }
    for (int k = threadIdx.x; k < nloc * NF * NV * NQ; k += blockDim.x) {
        const int eb = k / (NF * NV * NQ);
        const int r = k - eb * NF * NV * NQ;
        const int f = r / (NV * NQ), rem = r - f * NV * NQ;
        const int en = nbr[eb * NF + f];
        cp_async(&sm[eb * per + LL::S_U + LL::S_TR + r], &Tu[((size_t)en * NF + (f ^ 1)) * LL::FST + rem]);
    }
    cp_async_wait_all();
    __syncthreads();
    if (NV == 5 && (off0 != real(0) || off4 != real(0))) {
        for (int k = threadIdx.x; k < nloc * NP; k += blockDim.x) {
            const int eb = k / NP, pt = k - eb * NP;
            sm[eb * per + pt] -= off0;
            sm[eb * per + 4 * NP + pt] -= off4;
        }
    }
}

// ---------------------------------------------------------------- pipelined staging
// The residual kernels are persistent: block b walks over the element groups b, b + grid,
// b + 2 grid, ... and keeps two shared-memory copies of the loaded data, so the copies of
// the next group are in flight while the current group is computed. A copy holds
//   u       [NV][EB][NP] (variable-major over the block's elements), padded to 4 values,
//   (NB_TR) the neighbour traces [EB][NF][FST],
//   (FH)    the interface fluxes of the element's faces [EB][NF][FST];
// the trace and flux blocks are copied as whole padded global blocks, in 16-byte pieces.
// The values the kernel computes itself (own traces [EB][NF][FST], v^S: WORK values per
// element) live in one work area. Where two copies do not fit in shared memory (the
// largest n in FP64) one copy is used and the loads of a group are not overlapped.
template <class LL, bool NB_TR, bool FH, typename real, int WORK>
struct Pipe {
    static constexpr int UPAD = round4(LL::S_U * LL::EB);
    static constexpr int TRB = LL::EB * LL::NF * LL::FST;            // one [EB][NF][FST] block
    static constexpr int OFF_TR = UPAD;                              // neighbour traces
    static constexpr int OFF_FH = UPAD + (NB_TR ? TRB : 0);          // interface fluxes
    static constexpr int LOAD = UPAD + (NB_TR ? TRB : 0) + (FH ? TRB : 0);   // per copy
    static constexpr int NBR_INTS = LL::NBR_BYTES / 4;
    static constexpr size_t bytes_n(int nbuf) {
        return 2 * (size_t)LL::NBR_BYTES + sizeof(real) * ((size_t)nbuf * LOAD + (size_t)LL::EB * WORK);
    }
    static constexpr int NBUF = bytes_n(2) <= 227 * 1024 ? 2 : 1;
    static constexpr size_t BYTES = bytes_n(NBUF);
};

template <typename real, class LL>
using TracePipe = Pipe<LL, false, false, real, 0>;
template <typename real, class LL>
using GradPipe = Pipe<LL, true, false, real, LL::S_VR>;
template <typename real, class LL>
struct FluxWork;
template <typename real, class LL>
using FluxPipe = Pipe<LL, true, true, real, FluxWork<real, LL>::value>;

// work values per element of the flux kernel: the kept v^S and the per-direction
// contributions R_d. FP32: R_d in a region of its own (SEP), so that writing it needs no
// barrier after the flux loops have read v^S and R can be written one iteration late. FP64:
// R_d over v^S behind one more barrier, which keeps the block's shared memory, and the
// resident blocks per SM, of the single-region layout.
template <typename real, class LL>
struct FluxWork {
    static constexpr bool SEP = sizeof(real) == 4;
    static constexpr int RD0 = SEP ? LL::S_VR : 0;           // offset of R_d in the work area
    static constexpr int value = SEP ? LL::S_VR + LL::S_RD : (LL::S_VR > LL::S_RD ? LL::S_VR : LL::S_RD);
};

template <class LL>
using ResStrides = Strides<LL::EB * LL::NP, LL::FST>;
template <class LL>
using ElemStrides = Strides<LL::NP, LL::S_TR / LL::NF>;

// neighbour element of every (element, face) of the group starting at e0 (no barrier)
template <class LL>
__device__ __forceinline__ void nbr_table(const Mesh& g, int e0, int nloc, int* nbr) {
    for (int k = threadIdx.x; k < nloc * LL::NF; k += blockDim.x) {
        const int eb = k / LL::NF, f = k - eb * LL::NF;
        nbr[k] = neighbour(g, e0 + eb, f >> 1, f & 1);
    }
}

// issue (do not wait for) the copies of one group into buf; nbr must be complete
template <typename real, class LL, class PL, int NV, bool NB_TR, bool FH>
__device__ __forceinline__ void stage_issue(const real* __restrict__ U, const real* __restrict__ Tu,
                                            const real* __restrict__ Fh, const Mesh& g, int e0, int nloc,
                                            real* buf, const int* nbr) {
    constexpr int NP = LL::NP, NF = LL::NF, FST = LL::FST, EB = LL::EB;
    constexpr int CH = 16 / (int)sizeof(real);          // values per 16-byte piece
    constexpr int CPB = FST / CH;                       // pieces per face block
    const int span = nloc * NP;                         // u values of one variable
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const real* src = U + (size_t)v * g.nelem * NP + (size_t)e0 * NP;
        real* dst = buf + v * EB * NP;
        for (int j = threadIdx.x; j < span; j += blockDim.x) cp_async(dst + j, src + j);
    }
    if (NB_TR) {
        for (int k = threadIdx.x; k < nloc * NF * CPB; k += blockDim.x) {
            const int c = k / CPB, w = k - c * CPB;     // c = eb * NF + f
            const int f = c % NF;
            const real* src = Tu + ((size_t)nbr[c] * NF + (f ^ 1)) * FST + w * CH;
            cp_async16(buf + PL::OFF_TR + c * FST + w * CH, src);
        }
    }
    if (FH) {
        for (int k = threadIdx.x; k < nloc * NF * CPB; k += blockDim.x) {
            const int c = k / CPB, w = k - c * CPB;
            const int eb = c / NF, f = c - eb * NF;
            // face 2d+1 is this element's +d face; face 2d is the +d face of its -d neighbour
            const int ef = (f & 1) ? e0 + eb : nbr[c];
            const real* src = Fh + ((size_t)(f >> 1) * g.nelem + ef) * FST + w * CH;
            cp_async16(buf + PL::OFF_FH + c * FST + w * CH, src);
        }
    }
}

// Pipeline steps. Iteration k of a block handles group g_k = blockIdx + k * grid. With two
// copies, iteration k waits for the copies of g_k, passes one barrier, and only then issues
// the copies of g_{k+1} into the other copy: every thread has finished reading that copy
// (group g_{k-1}) before the barrier, so no barrier is needed at the end of an iteration.
// The neighbour table of g_{k+2} is built in the same place, into the table g_k used (the
// tables alternate, nbr0 / nbr1 for even / odd k), so it is complete one barrier before
// its copies are issued. With one copy (the largest n in FP64) iteration k issues and waits
// for its own group, behind a barrier that ends the previous iteration's reads.
template <typename real, class LL, class PL, int NV, bool NB_TR, bool FH>
__device__ __forceinline__ void pipe_start(const real* __restrict__ U, const real* __restrict__ Tu,
                                           const real* __restrict__ Fh, const Mesh& g, int grp, int ngroups,
                                           real* buf0, int* nbr0, int* nbr1) {
    if (NB_TR || FH) {
        nbr_table<LL>(g, grp_first<LL::EB>(g, grp), grp_count<LL::EB>(g, grp), nbr0);
        const int gn = grp + gridDim.x;
        if (PL::NBUF == 2 && gn < ngroups) nbr_table<LL>(g, grp_first<LL::EB>(g, gn), grp_count<LL::EB>(g, gn), nbr1);
        __syncthreads();
    }
    if constexpr (PL::NBUF == 2) {
        stage_issue<real, LL, PL, NV, NB_TR, FH>(U, Tu, Fh, g, grp_first<LL::EB>(g, grp), grp_count<LL::EB>(g, grp),
                                                 buf0, nbr0);
        cp_async_commit();
    }
}

// top of iteration k (b = k & 1) for group grp: wait for this group's copies and make them
// visible to the block, then start the next group's copies (two copies). With OFFS the
// reference offsets are removed from the staged u in one pass (one more barrier); without,
// the staged u keeps the stored values and the line functions remove the offsets as they
// load their lines (the same FP32 subtraction, so the results are the same).
template <typename real, class LL, class PL, int NV, bool NB_TR, bool FH, bool OFFS = false>
__device__ __forceinline__ void pipe_next(const real* __restrict__ U, const real* __restrict__ Tu,
                                          const real* __restrict__ Fh, const Mesh& g, int grp, int ngroups, int b,
                                          bool first, real* buf0, real* buf1, int* nbr0, int* nbr1,
                                          real off0 = real(0), real off4 = real(0)) {
    real* buf = b ? buf1 : buf0;
    if constexpr (PL::NBUF == 1) {
        if (!first) __syncthreads();                 // the previous group's reads of buf0 are done
        stage_issue<real, LL, PL, NV, NB_TR, FH>(U, Tu, Fh, g, grp_first<LL::EB>(g, grp), grp_count<LL::EB>(g, grp),
                                                 buf, nbr0);
        cp_async_commit();
    }
    cp_async_wait_group<0>();
    __syncthreads();
    if constexpr (OFFS && NV == 5) {
        const int span = grp_count<LL::EB>(g, grp) * LL::NP;
        real* u0 = buf;
        real* u4 = buf + 4 * LL::EB * LL::NP;
        for (int k = threadIdx.x; k < span; k += blockDim.x) {
            u0[k] -= off0;
            u4[k] -= off4;
        }
        __syncthreads();
    }
    constexpr bool NB = NB_TR || FH;
    if constexpr (PL::NBUF == 2) {
        const int gn = grp + gridDim.x;
        if (gn < ngroups) {
            stage_issue<real, LL, PL, NV, NB_TR, FH>(U, Tu, Fh, g, grp_first<LL::EB>(g, gn), grp_count<LL::EB>(g, gn),
                                                     b ? buf0 : buf1, b ? nbr0 : nbr1);
            cp_async_commit();
        }
        const int ga = grp + 2 * gridDim.x;
        if (NB && ga < ngroups)
            nbr_table<LL>(g, grp_first<LL::EB>(g, ga), grp_count<LL::EB>(g, ga), b ? nbr1 : nbr0);
    } else {
        const int gn = grp + gridDim.x;
        if (NB && gn < ngroups) nbr_table<LL>(g, grp_first<LL::EB>(g, gn), grp_count<LL::EB>(g, gn), nbr0);
    }
}

// staged value of variable v with the reference offset removed (Navier-Stokes: rho - rho0
// and rho E - rho E0; the same FP32 subtraction wherever a line loads the point)
template <typename real, int NV>
__device__ __forceinline__ real unoffset(real x, int v, real off0, real off4) {
    if constexpr (NV == 5) {
        if (v == 0) return x - off0;
        if (v == 4) return x - off4;
    }
    return x;
}

// ---------------------------------------------------------------- line functions
// own traces at the two faces of direction D for every variable of line q; outL/outR
// point at the face blocks, ostride between variables
// (OFF: su holds the stored values and the reference offsets are removed here)
template <typename real, int N, int NQ, int NV, int D, class ST, bool OFF = false>
__device__ __forceinline__ void line_traces(const real* su, int q, real* outL, real* outR, int ostride,
                                            real off0 = real(0), real off4 = real(0)) {
    const OpTab<real, N>& op = c_op<real, N>;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        real u[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            u[i] = su[v * ST::US + lpt<N, D>(i, q)];
            if constexpr (OFF) u[i] = unoffset<real, NV>(u[i], v, off0, off4);
        }
        outL[v * ostride] = dotc<real, N>(op.L, u);
        outR[v * ostride] = dotc<real, N>(op.L + N * N, u);
    }
}

// face traces of the porous-medium diffusivity m |u|^(m-1) evaluated at the solution
// points of line q (Sec. 4.3 variant), for the interface flux
template <typename real, int N, int D, class ST>
__device__ __forceinline__ void coef_traces(const Phys<real>& P, const real* su, int q, real* outL, real* outR) {
    const OpTab<real, N>& op = c_op<real, N>;
    real a[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = scalar_coef(P, su[lpt<N, D>(i, q)]);
    *outL = dotc<real, N>(op.L, a);
    *outR = dotc<real, N>(op.L + N * N, a);
}

// v^S along D for every variable of line q (Eq. w:e in Cartesian form):
// v_D = (2/h_D) (D u + M[:,0] delta_L + M[:,N] delta_R)
template <typename real, int N, int DIM, int NV, int D, class ST>
__device__ __forceinline__ void line_vs(const LineGeo<real>& geo, const real* su, const real* tro,
                                        const real* trn, real* vS, int q) {
    constexpr int NP = ipow(N, DIM), NQ = ipow(N, DIM - 1);
    const OpTab<real, N>& op = c_op<real, N>;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        real u[N];
#pragma unroll
        for (int i = 0; i < N; ++i) u[i] = su[v * ST::US + lpt<N, D>(i, q)];
        const int il = (2 * D) * ST::FS + v * NQ + q, ir = (2 * D + 1) * ST::FS + v * NQ + q;
        const real dl = real(0.5) * (trn[il] - tro[il]);
        const real dr = real(0.5) * (trn[ir] - tro[ir]);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            real acc = dotc<real, N>(op.D + i * N, u);
            acc = fma(op.M[i * (N + 1)], dl, acc);
            acc = fma(op.M[i * (N + 1) + N], dr, acc);
            vS[(v * DIM + D) * NP + lpt<N, D>(i, q)] = geo.two_h[D] * acc;
        }
    }
}

// prologue of the closure kernels: own traces, then v^S (all components)
template <typename real, int N, int DIM, int NV, class ST>
__device__ __forceinline__ void prologue(const LineGeo<real>& geo, const LineId& id, bool live,
                                         real* su, real* tro, real* trn, real* vS) {
    constexpr int NQ = ipow(N, DIM - 1), FS = ST::FS;
    if (live) {
        real* o = tro + id.q;
        if (id.d == 0) line_traces<real, N, NQ, NV, 0, ST>(su, id.q, o, o + FS, NQ);
        if constexpr (DIM == 3) {
            if (id.d == 1) line_traces<real, N, NQ, NV, 1, ST>(su, id.q, o + 2 * FS, o + 3 * FS, NQ);
            if (id.d == 2) line_traces<real, N, NQ, NV, 2, ST>(su, id.q, o + 4 * FS, o + 5 * FS, NQ);
        }
    }
    __syncthreads();
    if (live) {
        if (id.d == 0) line_vs<real, N, DIM, NV, 0, ST>(geo, su, tro, trn, vS, id.q);
        if constexpr (DIM == 3) {
            if (id.d == 1) line_vs<real, N, DIM, NV, 1, ST>(geo, su, tro, trn, vS, id.q);
            if (id.d == 2) line_vs<real, N, DIM, NV, 2, ST>(geo, su, tro, trn, vS, id.q);
        }
    }
    __syncthreads();
}

// Residual kernels, per line (direction D, face point q): the line's u, its own face
// traces and the corrections delta stay in registers; the only shared-memory results are
// the kept v^S components, which the lines of the other directions read after a barrier.
//
// line_load: u of every variable, the own traces (L_0 u, L_n u, the same fma sequence as
// k_line_trace), delta_L = (trace_nb - trace_own)/2 at face 2D, delta_R at face 2D+1
// (Eq. c:flux), and (Navier-Stokes) v^S along D of rho and of the two momentum
// components across D (Eq. w:e; vslot)
template <typename real, int N, int DIM, int NV, int D, class ST, bool OFF>
__device__ __forceinline__ void line_load(const LineGeo<real>& geo, const real* su, const real* trn, real* vS,
                                          int q, real (&u)[NV][N], real (&dl)[NV], real (&dr)[NV]) {
    constexpr int NP = ipow(N, DIM), NQ = ipow(N, DIM - 1);
    const OpTab<real, N>& op = c_op<real, N>;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            u[v][i] = su[v * ST::US + lpt<N, D>(i, q)];
            if constexpr (OFF) u[v][i] = unoffset<real, NV>(u[v][i], v, geo.off0, geo.off4);
        }
        const real tl = dotc<real, N>(op.L, u[v]);
        const real tr = dotc<real, N>(op.L + N * N, u[v]);
        dl[v] = real(0.5) * (trn[(2 * D) * ST::FS + v * NQ + q] - tl);
        dr[v] = real(0.5) * (trn[(2 * D + 1) * ST::FS + v * NQ + q] - tr);
    }
    if constexpr (NV == 5) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int v = k == 0 ? 0 : 1 + (D + k) % 3;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                real acc = dotc<real, N>(op.D + i * N, u[v]);
                acc = fma(op.M[i * (N + 1)], dl[v], acc);
                acc = fma(op.M[i * (N + 1) + N], dr[v], acc);
                vS[vslot(v, D) * NP + lpt<N, D>(i, q)] = geo.two_h[D] * acc;
            }
        }
    }
}

// line_load for the warp's direction, then (Navier-Stokes) the barrier after which every
// kept v^S component is visible
template <typename real, int N, int DIM, int NV, class ST, bool OFF>
__device__ __forceinline__ void prologue_res(const LineGeo<real>& geo, const LineId& id, bool live,
                                             const real* su, const real* trn, real* vS, real (&u)[NV][N],
                                             real (&dl)[NV], real (&dr)[NV]) {
    if (live) {
        if (id.d == 0) line_load<real, N, DIM, NV, 0, ST, OFF>(geo, su, trn, vS, id.q, u, dl, dr);
        if constexpr (DIM == 3) {
            if (id.d == 1) line_load<real, N, DIM, NV, 1, ST, OFF>(geo, su, trn, vS, id.q, u, dl, dr);
            if (id.d == 2) line_load<real, N, DIM, NV, 2, ST, OFF>(geo, su, trn, vS, id.q, u, dl, dr);
        }
    }
    if constexpr (NV == 5) __syncthreads();
}

// own interface gradients of the two faces of direction D (written to the padded global
// blocks out[f][GST], [c][q] within a block): normal components from u and the corrections (BR1:
// L_s v^S; compact: the one-sided gradient keeps only the correction of face s, the
// closed form of Eqs. aux:cmp:lr:2d), transverse components from the kept v^S
template <typename real, int N, int DIM, int NV, int D>
__device__ __forceinline__ void grad_faces_res(const LineGeo<real>& geo, int compact, const real (&u)[NV][N],
                                               const real (&dl)[NV], const real (&dr)[NV], const real* vS,
                                               real* out, int q) {
    using LL = LineLayout<N, DIM, NV>;
    constexpr int NP = LL::NP, NQ = LL::NQ, NG = LL::NG, GST = LL::GST;
    const OpTab<real, N>& op = c_op<real, N>;
    const real th = geo.two_h[D];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        real aL, aR;
        if (compact) {
            aL = th * fma(op.LM0[0], dl[v], dotc<real, N>(op.LD, u[v]));
            aR = th * fma(op.LMN[N], dr[v], dotc<real, N>(op.LD + N * N, u[v]));
        } else {
            aL = dline<real, N>(op, 0, u[v], dl[v], dr[v], th);
            aR = dline<real, N>(op, N, u[v], dl[v], dr[v], th);
        }
        out[(2 * D) * GST + v * NQ + q] = aL;
        out[(2 * D + 1) * GST + v * NQ + q] = aR;
    }
#pragma unroll
    for (int c = NV; c < NG; ++c) {
        int v, m;
        comp_map<NV>(D, c, v, m);
        real gl[N];
#pragma unroll
        for (int i = 0; i < N; ++i) gl[i] = vS[vslot(v, m) * NP + lpt<N, D>(i, q)];
        out[(2 * D) * GST + c * NQ + q] = dotc<real, N>(op.L, gl);
        out[(2 * D + 1) * GST + c * NQ + q] = dotc<real, N>(op.L + N * N, gl);
    }
}

// ---------------------------------------------------------------- kernels
template <typename real, int N, int DIM, int NV>
__global__ void __launch_bounds__(LineLayout<N, DIM, NV>::THREADS)
k_line_trace(const real* __restrict__ U, real* __restrict__ Tu, LineGeo<real> geo, Mesh g, Phys<real> P) {
    using LL = LineLayout<N, DIM, NV>;
    using PL = TracePipe<real, LL>;
    using ST = ResStrides<LL>;
    constexpr int NP = LL::NP, NQ = LL::NQ, NF = LL::NF, FST = LL::FST;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* buf0 = reinterpret_cast<real*>(smem_raw + 2 * LL::NBR_BYTES);
    real* buf1 = buf0 + (PL::NBUF - 1) * PL::LOAD;
    const int ngroups = num_groups<LL::EB>(g);
    int grp = blockIdx.x;
    if (grp >= ngroups) return;
    const LineId id = line_id<LL>(threadIdx.x);
    pipe_start<real, LL, PL, NV, false, false>(U, nullptr, nullptr, g, grp, ngroups, buf0, nullptr, nullptr);
    for (int b = 0; grp < ngroups; grp += gridDim.x, b ^= 1) {
        real* buf = b ? buf1 : buf0;
        const int e0 = grp_first<LL::EB>(g, grp);
        // FP32: offsets removed per line (no shared pass, no second barrier); FP64: in one
        // shared pass (B300's FP64 rate makes the three-fold per-line subtraction the dearer)
        constexpr bool LOFF = sizeof(real) == 4;
        pipe_next<real, LL, PL, NV, false, false, !LOFF>(U, nullptr, nullptr, g, grp, ngroups, b,
                                                         grp == (int)blockIdx.x, buf0, buf1, nullptr, nullptr,
                                                         geo.off0, geo.off4);
        const int e = e0 + id.eb;
        if (id.ok && e < g.e_end) {
            const real* su = buf + id.eb * NP;
            real* out = Tu + (size_t)e * NF * FST + id.q;
            const real o0 = geo.off0, o4 = geo.off4;
            if (id.d == 0) line_traces<real, N, NQ, NV, 0, ST, LOFF>(su, id.q, out, out + FST, NQ, o0, o4);
            if constexpr (DIM == 3) {
                if (id.d == 1)
                    line_traces<real, N, NQ, NV, 1, ST, LOFF>(su, id.q, out + 2 * FST, out + 3 * FST, NQ, o0, o4);
                if (id.d == 2)
                    line_traces<real, N, NQ, NV, 2, ST, LOFF>(su, id.q, out + 4 * FST, out + 5 * FST, NQ, o0, o4);
            }
            if constexpr (NV == 1) {
                if (P.pme_sol) {
                    real* o = out + NQ;
                    if (id.d == 0) coef_traces<real, N, 0, ST>(P, su, id.q, o, o + FST);
                    if constexpr (DIM == 3) {
                        if (id.d == 1) coef_traces<real, N, 1, ST>(P, su, id.q, o + 2 * FST, o + 3 * FST);
                        if (id.d == 2) coef_traces<real, N, 2, ST>(P, su, id.q, o + 4 * FST, o + 5 * FST);
                    }
                }
            }
        }
    }
}

template <typename real, int N, int DIM, int NV>
__global__ void __launch_bounds__(LineLayout<N, DIM, NV>::THREADS)
k_line_grad(const real* __restrict__ U, const real* __restrict__ Tu, real* __restrict__ Tg,
            LineGeo<real> geo, Mesh g, int compact) {
    using LL = LineLayout<N, DIM, NV>;
    using PL = GradPipe<real, LL>;
    using ST = ResStrides<LL>;
    constexpr int NP = LL::NP, NF = LL::NF, GST = LL::GST;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* nbr0 = reinterpret_cast<int*>(smem_raw);
    int* nbr1 = nbr0 + PL::NBR_INTS;
    real* buf0 = reinterpret_cast<real*>(smem_raw + 2 * LL::NBR_BYTES);
    real* buf1 = buf0 + (PL::NBUF - 1) * PL::LOAD;
    real* work = buf0 + PL::NBUF * PL::LOAD;
    const int ngroups = num_groups<LL::EB>(g);
    int grp = blockIdx.x;
    if (grp >= ngroups) return;
    const LineId id = line_id<LL>(threadIdx.x);
    real* vS = work + id.eb * LL::S_VR;
    pipe_start<real, LL, PL, NV, true, false>(U, Tu, nullptr, g, grp, ngroups, buf0, nbr0, nbr1);
    for (int b = 0; grp < ngroups; grp += gridDim.x, b ^= 1) {
        real* buf = b ? buf1 : buf0;
        const int e0 = grp_first<LL::EB>(g, grp);
        // offsets: per line in FP32 (one barrier fewer per group: 0.280 against 0.285 ms
        // per launch at 48^3), one shared pass in FP64
        constexpr bool LOFF = sizeof(real) == 4;
        pipe_next<real, LL, PL, NV, true, false, !LOFF>(U, Tu, nullptr, g, grp, ngroups, b, grp == (int)blockIdx.x,
                                                        buf0, buf1, nbr0, nbr1, geo.off0, geo.off4);
        const int e = e0 + id.eb;
        const bool live = id.ok && e < g.e_end;
        const real* su = buf + id.eb * NP;
        const real* trn = buf + PL::OFF_TR + id.eb * NF * LL::FST;
        real u[NV][N], dl[NV], dr[NV];
        prologue_res<real, N, DIM, NV, ST, LOFF>(geo, id, live, su, trn, vS, u, dl, dr);
        if (live) {
            real* out = Tg + (size_t)e * NF * GST;
            if (id.d == 0) grad_faces_res<real, N, DIM, NV, 0>(geo, compact, u, dl, dr, vS, out, id.q);
            if constexpr (DIM == 3) {
                if (id.d == 1) grad_faces_res<real, N, DIM, NV, 1>(geo, compact, u, dl, dr, vS, out, id.q);
                if (id.d == 2) grad_faces_res<real, N, DIM, NV, 2>(geo, compact, u, dl, dr, vS, out, id.q);
            }
        }
    }
}

// common flux through one interface point along compile-time direction D: UL, gL are the
// traces and interface gradients of the element on the -D side, UR, gR of the one on the
// +D side (Eqs. c:flux, c:aux:v:2d; Sec. 4.4 option (a): Riemann flux of the two traces
// minus the viscous flux of the averaged state and gradient)
template <typename real, int NV, int NG, int D>
__device__ __forceinline__ void interface_flux(const LineGeo<real>& geo, const Phys<real>& P, const real* UL,
                                               const real* UR, const real* gL, const real* gR,
                                               const float* tauL, const float* tauR, real* F, real aL = real(0),
                                               real aR = real(0)) {
    if constexpr (NV == 1) {
        // scalar: -c v with the diffusivity c of the averaged state (option (a)) or of each
        // side (option (b)); with the diffusivity taken at the solution points, aL and aR
        // are the two sides' extrapolated values
        real g = real(0.5) * (gL[0] + gR[0]);
        real a = gL[0], b = gR[0];
        if (geo.tip[D] != real(0)) {
            g = fma(geo.tip[D], UR[0] - UL[0], g);
            a = fma(geo.tip[D], UR[0] - UL[0], a);
            b = fma(geo.tip[D], UR[0] - UL[0], b);
        }
        const bool sol = P.kind == 1 && P.pme_sol;
        if (P.vflux == 0) {
            const real c = sol ? real(0.5) * (aL + aR) : scalar_coef(P, real(0.5) * (UL[0] + UR[0]));
            F[0] = -c * g;
        } else {
            const real cl = sol ? aL : scalar_coef(P, UL[0]);
            const real cr = sol ? aR : scalar_coef(P, UR[0]);
            F[0] = real(0.5) * (-cl * a + -cr * b);
        }
        return;
    }
    real Fv[NV];
    if (P.vflux == 0) {
        // option (a): the flux of the averaged state and the averaged gradient
        real Uh[NV], vh[NG];
#pragma unroll
        for (int v = 0; v < NV; ++v) Uh[v] = real(0.5) * (UL[v] + UR[v]);
#pragma unroll
        for (int c = 0; c < NG; ++c) {
            vh[c] = real(0.5) * (gL[c] + gR[c]);
            // interior penalty on the normal derivative: tau_IP (u_R - u_L)
            if (c < NV && geo.tip[D] != real(0)) vh[c] = fma(geo.tip[D], UR[c] - UL[c], vh[c]);
        }
        ns_viscous(Uh, vh, D, P, Fv);
    } else {
        // option (b): the average of the two sides' fluxes, each from its own trace and
        // interface gradient (the penalty term on both sides' normal derivatives)
        real a[NG], b[NG], FL[NV], FR[NV];
#pragma unroll
        for (int c = 0; c < NG; ++c) {
            a[c] = gL[c];
            b[c] = gR[c];
            if (c < NV && geo.tip[D] != real(0)) {
                a[c] = fma(geo.tip[D], UR[c] - UL[c], a[c]);
                b[c] = fma(geo.tip[D], UR[c] - UL[c], b[c]);
            }
        }
        ns_viscous(UL, a, D, P, FL);
        ns_viscous(UR, b, D, P, FR);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fv[v] = real(0.5) * (FL[v] + FR[v]);
    }
    {
        ns_riemann(UL, UR, D, P, F);
        if (tauL) {
            // extra per-element flux: centred average of the two elements at the interface
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] += real(0.5) * ((real)tauL[3 * v + D] + (real)tauR[3 * v + D]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] -= Fv[v];
    }
}

template <typename real, int N, int DIM, int NV, int D>
__device__ __forceinline__ void face_point(const real* __restrict__ Tu, const real* __restrict__ Tg,
                                           real* __restrict__ Fh, const LineGeo<real>& geo, const Mesh& g,
                                           const Phys<real>& P, const float* __restrict__ tau, int e, int q) {
    using LL = LineLayout<N, DIM, NV>;
    constexpr int NQ = LL::NQ, NF = LL::NF, NG = LL::NG, FST = LL::FST, GST = LL::GST;
    const int en = neighbour(g, e, D, 1);
    const real* tl = Tu + ((size_t)e * NF + 2 * D + 1) * FST + q;
    const real* tr = Tu + ((size_t)en * NF + 2 * D) * FST + q;
    const real* gl = Tg + ((size_t)e * NF + 2 * D + 1) * GST + q;
    const real* gr = Tg + ((size_t)en * NF + 2 * D) * GST + q;
    real UL[NV], UR[NV], gL[NG], gR[NG], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        UL[v] = tl[v * NQ];
        UR[v] = tr[v * NQ];
    }
#pragma unroll
    for (int c = 0; c < NG; ++c) {
        gL[c] = gl[c * NQ];
        gR[c] = gr[c * NQ];
    }
    const float* tauL = nullptr;
    const float* tauR = nullptr;
    if (NV == 5 && tau) {
        tauL = tau + (size_t)e * 15;
        tauR = tau + (size_t)en * 15;
    }
    real aL = real(0), aR = real(0);
    if (NV == 1 && P.pme_sol) {
        aL = tl[NQ];
        aR = tr[NQ];
    }
    interface_flux<real, NV, NG, D>(geo, P, UL, UR, gL, gR, tauL, tauR, F, aL, aR);
    real* out = Fh + ((size_t)D * g.nelem + e) * FST + q;
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * NQ] = F[v];
}

// One thread per interface point; thread index (d, e, q) with q fastest, so the direction
// is uniform over long runs of threads and each direction has its own code path.
template <typename real, int N, int DIM, int NV>
__global__ void __launch_bounds__(256)
k_face_flux(const real* __restrict__ Tu, const real* __restrict__ Tg, real* __restrict__ Fh,
            LineGeo<real> geo, Mesh g, Phys<real> P, const float* __restrict__ tau) {
    constexpr int NQ = ipow(N, DIM - 1);
    const long long per_d = (long long)(g.e_end - g.e_begin) * NQ;
    const long long total = per_d * DIM;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(idx / per_d);
        const long long r = idx - d * per_d;
        const int el = (int)(r / NQ), q = (int)(r - (long long)el * NQ);
        const int e = g.e_begin + el;
        if (d == 0) face_point<real, N, DIM, NV, 0>(Tu, Tg, Fh, geo, g, P, tau, e, q);
        if constexpr (DIM == 3) {
            if (d == 1) face_point<real, N, DIM, NV, 1>(Tu, Tg, Fh, geo, g, P, tau, e, q);
            if (d == 2) face_point<real, N, DIM, NV, 2>(Tu, Tg, Fh, geo, g, P, tau, e, q);
        }
    }
}

// fluxes along D at the n+1 flux points of line q and their divergence on the line: the
// interface fluxes at f = 0 and f = N come from Fh, the n-1 interior ones are evaluated here.
// The flux-point loop is kept rolled (unrolling it for n = 5 measured 0.98 against 0.80 ms
// per launch at 48^3 on B300: the larger body costs more than the constant operands save).
template <typename real, int N, int DIM, int NV, int D, class ST>
__device__ __forceinline__ void line_flux(const FluxOps<real, N>& fo, const Phys<real>& P, const real (&u)[NV][N],
                                          const real (&dl)[NV], const real (&dr)[NV], const real* vS,
                                          const real* fh, int q, real (&r)[NV][N], const float* tau_own) {
    using LL = LineLayout<N, DIM, NV>;
    constexpr int NP = LL::NP, NQ = LL::NQ, NG = LL::NG;
    const OpTab<real, N>& op = c_op<real, N>;
    // interface flux points (f = 0 and f = N)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const real F0 = fh[(2 * D) * ST::FS + v * NQ + q];
        const real FN = fh[(2 * D + 1) * ST::FS + v * NQ + q];
#pragma unroll
        for (int i = 0; i < N; ++i) r[v][i] = fma(fo.Mn[D][i][N], FN, fo.Mn[D][i][0] * F0);
    }
    // interior flux points: extrapolated solution and gradient (Eq. aux:v:std:2d); the
    // normal derivatives come from u and the face corrections, the transverse ones from the
    // kept v^S
#pragma unroll 1
    for (int f = 1; f < N; ++f) {
        const real* Lr = op.L + f * N;
        real uf[NV], F[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) uf[v] = dotc<real, N>(Lr, u[v]);
        if constexpr (NV == 5) {
            real gf[NG];
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                real a = dotc<real, N>(fo.LDn[D][f], u[c]);
                a = fma(fo.LM0n[D][f], dl[c], a);
                gf[c] = fma(fo.LMNn[D][f], dr[c], a);
            }
#pragma unroll
            for (int c = NV; c < NG; ++c) {
                int v, m;
                comp_map<NV>(D, c, v, m);
                real gl[N];
#pragma unroll
                for (int i = 0; i < N; ++i) gl[i] = vS[vslot(v, m) * NP + lpt<N, D>(i, q)];
                gf[c] = dotc<real, N>(Lr, gl);
            }
            ns_flux_point(uf, gf, D, P, F);
            if (tau_own) {
#pragma unroll
                for (int v = 0; v < NV; ++v) F[v] += (real)tau_own[3 * v + D];
            }
        } else {
            real gfn = dotc<real, N>(fo.LDn[D][f], u[0]);
            gfn = fma(fo.LM0n[D][f], dl[0], gfn);
            gfn = fma(fo.LMNn[D][f], dr[0], gfn);
            if (P.kind == 1 && P.pme_sol) {
                // diffusivity from the solution points, extrapolated to the flux point
                real a[N];
#pragma unroll
                for (int i = 0; i < N; ++i) a[i] = scalar_coef(P, u[0][i]);
                F[0] = -dotc<real, N>(Lr, a) * gfn;
            } else {
                F[0] = scalar_flux(P, uf[0], gfn);
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int i = 0; i < N; ++i) r[v][i] = fma(fo.Mn[D][i][f], F[v], r[v][i]);
    }
}

template <int N, int DIM, int NV>
using FluxLayout = LineLayout<N, DIM, NV, SD_FLUX_THREADS>;

template <typename real, int N, int DIM, int NV>
__global__ void __maxnreg__((FluxLayout<N, DIM, NV>::FLUX_REGS))
k_line_flux(const real* __restrict__ U, const real* __restrict__ Tu, const real* __restrict__ Fh,
            real* __restrict__ R, LineGeo<real> geo, Mesh g, Phys<real> P, const float* __restrict__ tau,
            const __grid_constant__ FluxOps<real, N> fo) {
    using LL = FluxLayout<N, DIM, NV>;
    using PL = FluxPipe<real, LL>;
    using ST = ResStrides<LL>;
    constexpr int NP = LL::NP, NF = LL::NF, EB = LL::EB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int* nbr0 = reinterpret_cast<int*>(smem_raw);
    int* nbr1 = nbr0 + PL::NBR_INTS;
    real* buf0 = reinterpret_cast<real*>(smem_raw + 2 * LL::NBR_BYTES);
    real* buf1 = buf0 + (PL::NBUF - 1) * PL::LOAD;
    real* work = buf0 + PL::NBUF * PL::LOAD;
    const int ngroups = num_groups<EB>(g);
    int grp = blockIdx.x;
    if (grp >= ngroups) return;
    const LineId id = line_id<LL>(threadIdx.x);
    using FW = FluxWork<real, LL>;
    constexpr int WPE = FW::value;                             // work values per element
    real* vS = work + id.eb * WPE;
    // R of a group: the three directions' contributions, added in the fixed order x, y, z
    // (deterministic sums). FP32 (FW::SEP): run one iteration late, after the next group's
    // first barrier, so that no barrier of its own is needed; FP64: at the end of the group
    // behind a barrier.
    auto write_r = [&](int pe0, int pnloc) {
        for (int k = threadIdx.x; k < pnloc * NV * NP; k += blockDim.x) {
            const int eb = k / (NV * NP);
            const int rr = k - eb * NV * NP;
            const int v = rr / NP, pt = rr - v * NP;
            const real* rd = work + eb * WPE + FW::RD0 + v * NP + pt;
            real acc = rd[0];
            if constexpr (DIM == 3) {
                acc = acc + rd[NV * NP];
                acc = acc + rd[2 * NV * NP];
            }
            R[(size_t)v * g.nelem * NP + (size_t)(pe0 + eb) * NP + pt] = acc;
        }
    };
    pipe_start<real, LL, PL, NV, true, true>(U, Tu, Fh, g, grp, ngroups, buf0, nbr0, nbr1);
    int pe0 = 0, pnloc = 0;                                     // the group whose R is pending
    for (int b = 0; grp < ngroups; grp += gridDim.x, b ^= 1) {
        real* buf = b ? buf1 : buf0;
        const int e0 = grp_first<EB>(g, grp), nloc = grp_count<EB>(g, grp);
        // offsets: per line in FP32, one shared pass in FP64 (as in k_line_trace)
        constexpr bool LOFF = sizeof(real) == 4;
        pipe_next<real, LL, PL, NV, true, true, !LOFF>(U, Tu, Fh, g, grp, ngroups, b, grp == (int)blockIdx.x, buf0,
                                                       buf1, nbr0, nbr1, geo.off0, geo.off4);
        if constexpr (FW::SEP) {
            write_r(pe0, pnloc);
            // Navier-Stokes: the barrier in prologue_res orders these reads of the work area
            // before this group's writes to it; scalars have no such barrier
            if constexpr (NV != 5) __syncthreads();
        }
        const int e = e0 + id.eb;
        const bool live = id.ok && e < g.e_end;
        const real* su = buf + id.eb * NP;
        const real* trn = buf + PL::OFF_TR + id.eb * NF * LL::FST;
        const real* fh = buf + PL::OFF_FH + id.eb * NF * LL::FST;
        real u[NV][N], dl[NV], dr[NV];
        prologue_res<real, N, DIM, NV, ST, LOFF>(geo, id, live, su, trn, vS, u, dl, dr);

        real r[NV][N];
        if (live) {
            const float* t0 = (NV == 5 && tau) ? tau + (size_t)e * 15 : nullptr;
            if (id.d == 0) line_flux<real, N, DIM, NV, 0, ST>(fo, P, u, dl, dr, vS, fh, id.q, r, t0);
            if constexpr (DIM == 3) {
                if (id.d == 1) line_flux<real, N, DIM, NV, 1, ST>(fo, P, u, dl, dr, vS, fh, id.q, r, t0);
                if (id.d == 2) line_flux<real, N, DIM, NV, 2, ST>(fo, P, u, dl, dr, vS, fh, id.q, r, t0);
            }
        }
        if constexpr (!FW::SEP) __syncthreads();                // every line has read v^S
        if (live) {
            // this line's contribution R_d[v][pt] in the work area
            real* rd = vS + FW::RD0 + id.d * NV * NP;
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    int pt;
                    if (id.d == 0) pt = lpt<N, 0>(i, id.q);
                    else if (id.d == 1) pt = lpt<N, (DIM == 3 ? 1 : 0)>(i, id.q);
                    else pt = lpt<N, (DIM == 3 ? 2 : 0)>(i, id.q);
                    rd[v * NP + pt] = r[v][i];
                }
        }
        if constexpr (FW::SEP) {
            pe0 = e0;
            pnloc = nloc;
        } else {
            __syncthreads();
            write_r(e0, nloc);
        }
    }
    if constexpr (FW::SEP) {
        __syncthreads();
        write_r(pe0, pnloc);
    }
}

}  // namespace sdk
