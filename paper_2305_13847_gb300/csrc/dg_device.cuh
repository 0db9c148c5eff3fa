// Device code of the moist DG right-hand side and SSPRK(4,3) stage update.
//
// Method: Hittmeir, Lederer, Schoeberl, von Wahl, "A discontinuous Galerkin
// approach for atmospheric flows with implicit condensation" (arXiv 2305.13847).
// Equation numbers below refer to that paper.
//
// Kernels (templated on dimension D, order K, rain switch and storage type):
//   k_prepare  per node: implicit-condensation split Eq. (2.8) -> derived
//              fields; per face point: traces of U and of (T, rho_v, p') on
//              all 2D faces of the element, written to a trace buffer.
//   k_stage    per element: volume term of Eq. (3.2) by sum factorisation,
//              Lax-Friedrichs face fluxes (Section 3.2, Eq. (3.4)) against the
//              neighbours' traces, sources (Eq. (2.4) and gravity), diagonal
//              M^{-1}; then either writes dU/dt, or performs the SSPRK(4,3)
//              stage combination and, fused, the next stage's split and traces.
//   k_split    per node split only (dg_saturation_split).
//   k_init_bubble, k_reduce_*  workload set-up and diagnostics.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dg_math.cuh"

namespace dgm {

// ---------------------------------------------------------------------------
// Physical constants: Table 1 (Appendix A) and Section 2.1 of the paper.
// ---------------------------------------------------------------------------
constexpr double kCl = 4218.0;     // specific heat of liquid water
constexpr double kCpd = 1005.0;    // dry air, constant pressure
constexpr double kCpv = 1850.0;    // vapour, constant pressure
constexpr double kCvd = 718.0;     // dry air, constant volume
constexpr double kCvv = 1390.0;    // vapour, constant volume
constexpr double kEref = 610.7;    // e_s(T_ref)
constexpr double kLref = 2.835e6;  // latent heat at T_ref
constexpr double kRd = 287.05;
constexpr double kRv = 461.51;
constexpr double kTref = 273.15;
constexpr double kPref = 1.0e5;
// Eq. (2.6): e_s = e_ref (T/T_ref)^a exp(b (1/T_ref - 1/T))
constexpr double kEsA = (kCpv - kCl) / kRv;
constexpr double kEsB = (kLref - (kCpv - kCl) * kTref) / kRv;
constexpr double kLprime = kLref - kRv * kTref;      // rho_v coefficient of Eq. (2.3)
constexpr double kInvTref = 1.0 / kTref;
constexpr double kRvs0 = kEref / (kRv * kTref);      // rho_vs(T_ref)
// Eq. (2.4), q_au = 0
constexpr double kSevA = 3.86e-3;
constexpr double kSevB = 9.41e-5;
constexpr double kSevC = 9.1;
constexpr double kSau = 1.0e-3;
constexpr double kSac = 1.72;

// Linearisation (adjoint) only: fractional rain powers are differentiated at
// max(rho_r, kRainFloorLin).  Their derivatives are unbounded as rho_r -> 0+,
// and the rain that the DG discretisation leaks into cloud-free elements
// (1e-20 .. 1e-9 kg/m^3) makes the exact linearisation grow without bound over
// a few dozen steps; below 1e-12 kg/m^3 (1e-9 g/m^3) no rain is physical.
constexpr double kRainFloorLin = 1e-12;

constexpr int kMaxNewton = 50;
constexpr double kNewtonTol = 1e-12;

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// ---------------------------------------------------------------------------
// Parameter blocks (passed by value; they live in the kernel-parameter bank)
// ---------------------------------------------------------------------------
struct MeshData {
    int n[3];
    int ne;
    int periodic[3];
    int nzlev_node, nzlev_face;
    double two_over_h[3];  // 2 / h_j: d(xi)/dx
    double h[3];
    double g;
    double rho_w;          // <= 0: rho_m + rho_r
    double kvr;            // v0 Gamma(4.5)/6 (pi N0)^(-1/8)
    double jac;            // |K| / 2^d
    double rain_floor;     // linearisation only: rain powers differentiated at max(rho_r, floor)
    double rain_d8, rain_d16;  // d rho_r^(1/8) / d rho_r and d rho_r^(1/16) / d rho_r at the floor
    int pert_split;        // float32 state: 1 = split in perturbation variables (DG_FP32_PERT)
    int newton_cap;        // iteration cap of every Newton loop of the split (default kMaxNewton)
    // faces normal to e_j: a grid of nfn[j] (= n_j, + 1 with walls) x the other n,
    // nfaces[j] of them; face c lies between the elements at coordinates c - 1
    // and c along e_j.  The face kernel covers direction j with fblk[j] CTAs
    // and stores, per element, the outward flux of each of its faces
    // (fbuf [ne][2D][NFP][NFP1], NFP = NF, or 2 NF with the diffusion's
    // symmetry terms), so that a stage tile reads one contiguous block.
    int nfn[3];
    int nfaces[3];
    int fblk[3];
    // artificial diffusion (Section 3.5): vertex grid of the continuous Q1
    // coefficient (n_j vertices per row if periodic, n_j + 1 with walls),
    // alpha_K = alpha_pre ||w||_{0,K} with alpha_pre = gamma 0.5 h^(1 - d/2),
    // interior-penalty factor sigma k^2 / h_j per direction
    int nv[3];
    double alpha_pre;
    double sigma_pen[3];
    // float32 copies of the constants the float32 forms use in their hot
    // loops (a float64 -> float32 conversion occupies the FP64 pipe)
    float two_over_h_f[3];
    float g_f, kvr_f, rho_w_f, jac_f, alpha_pre_f;
    float sigma_pen_f[3];
};

// a mesh constant in the storage type: the float64 value, or its float32 copy
template <typename Real>
__device__ __forceinline__ Real mconst(double d, float f) {
    return sizeof(Real) == sizeof(double) ? (Real)d : (Real)f;
}

template <typename Real>
struct RefData {
    Real dhat[6][6];   // dhat[a][i] = (w_i / w_a) l_a'(xi_i): weak derivative of basis a
    Real lm[6], lp[6];       // l_a(-1), l_a(+1)
    Real liftm[6], liftp[6]; // l_a(-1)/w_a, l_a(+1)/w_a
    Real xi[6], w[6];
    // artificial diffusion: nodal derivative matrix dmat[i][a] = l_a'(xi_i),
    // l_a'(-1), l_a'(+1) and their lifts l_a'(+-1)/w_a
    Real dmat[6][6];
    Real dlm[6], dlp[6];
    Real dliftm[6], dliftp[6];
    // dhat_s[j] = (2/h_j) dhat of this mesh, so that the volume contraction
    // needs no separate scaling (read from the mesh's own kernel arguments,
    // also where the other tables are shared between meshes)
    Real dhat_s[3][6][6];
    Real liftm_s[3][6], liftp_s[3][6];    // (2/h_j) l_a(-+1)/w_a
    Real dliftm_s[3][6], dliftp_s[3][6];  // (2/h_j)^2 l_a'(-+1)/w_a
};

template <typename Real>
struct KArgs {
    MeshData M;
    RefData<Real> ref;
    const Real *Uin;       // state the operator is evaluated on (ABI layout)
    const Real *Un;        // U^n for the stage combination (may equal Uin)
    Real *Uout;            // MODE_RHS: dU/dt; MODE_STAGE: new stage state
    Real *derived;         // [ND][nodes]
    const Real *trace_in;  // traces of Uin:   [2D][NTR][ne][NFP1]
    Real *trace_out;       // traces of Uout (MODE_STAGE)
    const Real *bnode;     // base at node levels [4][nzlev_node]: rho_d, rho_m, E, p
    const Real *bface;     // base at face levels [4][nzlev_face]
    const double *bnode_d; // float64 copy for the split
    const double *rvs_tab; // rho_vs Taylor table: [kTabN][kTabStride] (dg_math.cuh)
    const float *bsplit;   // DG_FP32_PERT: split of the base state per node level [kBsN][nzlev_node]
    Real *fbuf;            // face pass: G along +e_j of every face, face-major [faces][NFP][NFP1]
                           // (faces normal to e_0, then e_1, e_2); with diffusion NFP = 2 NF:
                           // flux, then S = alpha [[u]] / 2
    const int *ftab;       // face pass: index in fbuf of each element's 2D faces [ne][2D]
    Real *alphaK;          // diffusion: [2][ne] alpha_u, alpha_r per element (of the state produced)
    const Real *alphaV;    // diffusion: [2][nv] continuous coefficient at the vertices
    const Real *dtrace_in; // diffusion: d/dx_j traces of Uin  [2D][NF][ne][NFP1]
    Real *dtrace_out;      // diffusion: d/dx_j traces of Uout
    const Real *sponge;    // sponge delta_R at the node levels (last stage of a step) or null
    Real alpha, beta, gdt; // Uout = alpha Un + beta Uin + gdt dU/dt
    unsigned long long *flags;  // [0] Newton failures, [1] non-physical nodes
    // rain fall-out (time steps with rain): per point of the bottom and top
    // wall faces, the time integral of the outward water flux
    // [2 (bottom, top)][faces per wall][NFP1], float64; fall_w = this stage's
    // weight in the step (dt/6, dt/6, dt/6, dt/2); null when not accumulating
    double *fallout;
    double fall_w;
    // k_prepare and k_stage over element tiles [tile0, tile0 + ntiles)
    // (ntiles 0: all), so that an upload is split while its chunks arrive
    // and a download starts while the last stage still runs
    int tile0, ntiles;
};

// float64 value of a storage-type value (widen: integer pipe)
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return widen(x); }

// Fall-out: add this stage's outward water flux (rho_m + rho_r, outward
// normal) at point q of a bottom (top = false) or top wall face over
// horizontal element position h.  Each wall face point has one writer per
// stage, so the sum is deterministic.
template <class S, typename Real>
__device__ __forceinline__ void add_fallout(const KArgs<Real> &A, bool top, int h, int q,
                                            double out_water) {
    const int nh = S::D == 3 ? A.M.n[0] * A.M.n[1] : A.M.n[0];
    double *p = A.fallout + ((size_t)(top ? nh : 0) + h) * S::NFP1 + q;
    *p = fma(A.fall_w, out_water, *p);
}

// ---------------------------------------------------------------------------
// Compile-time layout of one (D, K, RAIN) configuration
// ---------------------------------------------------------------------------
// TT_: the threads a stage tile aims at, EPB = TT_ / NP elements (at least
// one).  128 in 3-D: a warp that waits at a tile barrier holds up three
// others, not seven (measured: float32 steps -5 % against 256).
// FF_: float64 storage type with the stage kernel's volume and lift
// contractions as compensated float32-pair sums (DG_FP64_FFC, dg_math.cuh)
template <int D_, int K_, bool RAIN_, int TT_ = (D_ == 3 ? 128 : 256), bool FF_ = false>
struct Shape {
    static constexpr int D = D_;
    static constexpr int K = K_;
    static constexpr bool RAIN = RAIN_;
    static constexpr bool FF = FF_;
    static constexpr int P1 = K + 1;
    static constexpr int NP = ipow(P1, D);        // nodes per element
    static constexpr int NFP1 = ipow(P1, D - 1);  // points per face
    static constexpr int NFACE = 2 * D;
    static constexpr int NF = (RAIN ? 4 : 3) + D; // unknowns
    static constexpr int IM = RAIN ? 3 : 2;       // first momentum field
    static constexpr int IE = IM + D;             // energy field
    static constexpr int ND = RAIN ? 5 : 3;       // derived: T, rho_v, p' [, G_rm, v_r]
    static constexpr int NTR = NF + 3;            // traced: U, T, rho_v, p'
    static constexpr int EPB = (TT_ / NP) > 0 ? (TT_ / NP) : 1;   // elements per CTA
    static constexpr int NT = ((EPB * NP + 31) / 32) * 32;          // threads per CTA
    static constexpr int VERT = D - 1;
    static constexpr int NCORNER = 1 << D;                          // element vertices
};

template <int D, int P1>
__device__ __forceinline__ int digit(int a, int j) {
    if (j == 0) return a % P1;
    if (j == 1) return (D == 2) ? a / P1 : (a / P1) % P1;
    return a / (P1 * P1);
}

template <int P1>
__device__ __forceinline__ int stride_of(int j) { return j == 0 ? 1 : (j == 1 ? P1 : P1 * P1); }

// index of the face point of node a on the faces normal to e_j
template <int D, int P1>
__device__ __forceinline__ int face_q(int a, int j) {
    if (D == 2) return j == 0 ? digit<D, P1>(a, 1) : digit<D, P1>(a, 0);
    if (j == 0) return digit<D, P1>(a, 1) + P1 * digit<D, P1>(a, 2);
    if (j == 1) return digit<D, P1>(a, 0) + P1 * digit<D, P1>(a, 2);
    return digit<D, P1>(a, 0) + P1 * digit<D, P1>(a, 1);
}

// node at position i along direction j through face point q
template <int D, int P1>
__device__ __forceinline__ int line_node(int j, int q, int i) {
    if (D == 2) return j == 0 ? i + P1 * q : q + P1 * i;
    const int q0 = q % P1, q1 = q / P1;
    if (j == 0) return i + P1 * (q0 + P1 * q1);
    if (j == 1) return q0 + P1 * (i + P1 * q1);
    return q0 + P1 * (q1 + P1 * i);
}

// vertical node digit of face point q of a face normal to e_j (j not vertical)
template <int D, int P1>
__device__ __forceinline__ int face_q_vert(int j, int q) {
    if (D == 2) return q;           // j == 0: remaining direction is the vertical
    return q / P1;                  // j = 0 or 1: remaining (., vertical)
}

// A CTA's copy of the mesh's scaled reference tables, per direction j:
// dhat_s[j][a][0 .. P1) for each a, then liftm_s[j], liftp_s[j], dliftm_s[j],
// dliftp_s[j].  A thread indexes them by its own a_j; in shared memory the
// threads of a warp read their different entries in one access, where the
// kernel-parameter bank serves one address at a time.  The float64 tile
// reads them here (measured -1.4 % per step); the float32 tile, whose
// shared-memory pipe is the busier one, from the parameter bank.
template <class S>
struct Coef {
    static constexpr int ROWS = S::P1 * S::P1;
    static constexpr int LM = ROWS, LP = ROWS + S::P1, DLM = ROWS + 2 * S::P1, DLP = ROWS + 3 * S::P1;
    static constexpr int BLK = (ROWS + 4 * S::P1 + 3) / 4 * 4;   // whole 16-byte groups (float)
    static constexpr int N = S::D * BLK;
};

template <class S, typename Real>
__device__ __forceinline__ void coef_fill(const RefData<Real> &r, Real *s_cf) {
    using C = Coef<S>;
    for (int i = threadIdx.x; i < C::N; i += blockDim.x) {
        const int j = i / C::BLK, k = i - j * C::BLK;
        Real v = Real(0);
        if (k < C::LM) v = r.dhat_s[j][k / S::P1][k % S::P1];
        else if (k < C::LP) v = r.liftm_s[j][k - C::LM];
        else if (k < C::DLM) v = r.liftp_s[j][k - C::LP];
        else if (k < C::DLP) v = r.dliftm_s[j][k - C::DLM];
        else if (k < C::DLP + S::P1) v = r.dliftp_s[j][k - C::DLP];
        s_cf[i] = v;
    }
}

// Nodal-flux words per node and direction.  float32 stores the fields as
// interleaved pairs (2p, 2p + 1), the last pair padded when n_f is odd,
// [D][(n_f + 1) / 2][STR][2]: the volume term then runs on 64-bit shared
// loads and paired fmas (fma.rn.f32x2, each lane the scalar fma).  float64
// keeps [D][n_f][STR].
template <class S, typename Real>
__host__ __device__ constexpr int fl_words() {
    return (sizeof(Real) == sizeof(float) || S::FF) ? 2 * ((S::NF + 1) / 2) : S::NF;
}

// index of field f of direction j at tile node t in the nodal fluxes
template <class S, typename Real, int STR>
__device__ __forceinline__ int fl_index(int j, int f, int t) {
    if constexpr (sizeof(Real) == sizeof(float))
        return ((j * ((S::NF + 1) / 2) + (f >> 1)) * STR + t) * 2 + (f & 1);
    else
        return (j * S::NF + f) * STR + t;
}

// the fluxes F[0 .. n_f) of direction j at tile node t
template <class S, typename Real, int STR>
__device__ __forceinline__ void fl_store(Real *s_fl, int j, int t, const Real *F) {
    if constexpr (sizeof(Real) == sizeof(float)) {
        constexpr int NPR = (S::NF + 1) / 2;
        float2 *fl2 = reinterpret_cast<float2 *>(s_fl);
#pragma unroll
        for (int p = 0; p < NPR; ++p)
            fl2[(j * NPR + p) * STR + t] = make_float2(F[2 * p], 2 * p + 1 < S::NF ? F[2 * p + 1] : 0.0f);
    } else {
#pragma unroll
        for (int f = 0; f < S::NF; ++f) s_fl[(j * S::NF + f) * STR + t] = F[f];
    }
}

// Volume term of Eq. (3.2), sum factorised, at node a of local element el:
// R_a += sum_i dhat_s[j][a_j][i] F_j(line node i) for every direction j, from
// the nodal fluxes s_fl [D][NF][STR]; coefficients from s_cf (Coef, float64)
// or from the kernel arguments (float32)
template <class S, typename Real, int STR>
__device__ __forceinline__ void volume_term(const KArgs<Real> &A, const Real *s_fl,
                                            const Real *s_cf, int el, int a, Real *R) {
#pragma unroll
    for (int j = 0; j < S::D; ++j) {
        const int aj = digit<S::D, S::P1>(a, j);
        const int st = stride_of<S::P1>(j);
        const int b0 = el * S::NP + a - aj * st;
        if constexpr (sizeof(Real) == sizeof(double)) {
            Real c[S::P1];
#pragma unroll
            for (int i = 0; i < S::P1; ++i) c[i] = s_cf[j * Coef<S>::BLK + aj * S::P1 + i];
#pragma unroll
            for (int f = 0; f < S::NF; ++f) {
                const Real *fl = s_fl + (j * S::NF + f) * STR + b0;
                Real acc = R[f];
#pragma unroll
                for (int i = 0; i < S::P1; ++i) acc = fma(c[i], fl[i * st], acc);
                R[f] = acc;
            }
        } else {
            // field pairs: lane x is field 2p, lane y field 2p + 1, each the
            // same fma chain as one field at a time
            constexpr int NPR = (S::NF + 1) / 2;
            const float2 *fl2 = reinterpret_cast<const float2 *>(s_fl);
            float2 c[S::P1];
#pragma unroll
            for (int i = 0; i < S::P1; ++i) {
                const float ci = A.ref.dhat_s[j][aj][i];
                c[i] = make_float2(ci, ci);
            }
#pragma unroll
            for (int p = 0; p < NPR; ++p) {
                const float2 *fl = fl2 + (j * NPR + p) * STR + b0;
                float2 acc = make_float2(R[2 * p], 2 * p + 1 < S::NF ? R[2 * p + 1] : 0.0f);
#pragma unroll
                for (int i = 0; i < S::P1; ++i) acc = __ffma2_rn(c[i], fl[i * st], acc);
                R[2 * p] = acc.x;
                if (2 * p + 1 < S::NF) R[2 * p + 1] = acc.y;
            }
        }
    }
}

// ---- float-float contractions of the float64 form (DG_FP64_FFC) ----------
// The coefficient tables of Coef as float32 pairs (ff_split of the float64
// entries), in the same slots.
template <class S>
__device__ __forceinline__ void coef_fill_ff(const RefData<double> &r, float2 *s_cf) {
    using C = Coef<S>;
    for (int i = threadIdx.x; i < C::N; i += blockDim.x) {
        const int j = i / C::BLK, k = i - j * C::BLK;
        double v = 0.0;
        if (k < C::LM) v = r.dhat_s[j][k / S::P1][k % S::P1];
        else if (k < C::LP) v = r.liftm_s[j][k - C::LM];
        else if (k < C::DLM) v = r.liftp_s[j][k - C::LP];
        else if (k < C::DLP) v = r.dliftm_s[j][k - C::DLM];
        else if (k < C::DLP + S::P1) v = r.dliftp_s[j][k - C::DLP];
        s_cf[i] = ff_split(v);
    }
}

// Volume term of Eq. (3.2) as in volume_term, every product and sum as a
// compensated float32-pair operation, two fields at a time: (Rs, Re)[p] +=
// sum_i dhat_s[j][a_j][i] F_j(line node i) for the fields 2p (lane x) and
// 2p + 1 (lane y).  fl4 [D][(NF + 1) / 2][STR] holds (hi_2p, hi_2p+1, lo_2p,
// lo_2p+1) per node, the coefficients are pairs (coef_fill_ff); the terms of
// each field are taken in the float64 form's order.
template <class S, int STR>
__device__ __forceinline__ void volume_term_ff(const float4 *fl4, const float2 *cf2, int el, int a,
                                               float2 *Rs, float2 *Re) {
    constexpr int NPR = (S::NF + 1) / 2;
#pragma unroll
    for (int j = 0; j < S::D; ++j) {
        const int aj = digit<S::D, S::P1>(a, j);
        const int st = stride_of<S::P1>(j);
        const int b0 = el * S::NP + a - aj * st;
        float2 c[S::P1];
#pragma unroll
        for (int i = 0; i < S::P1; ++i) c[i] = cf2[j * Coef<S>::BLK + aj * S::P1 + i];
#pragma unroll
        for (int p = 0; p < NPR; ++p) {
            const float4 *fl = fl4 + (j * NPR + p) * STR + b0;
#pragma unroll
            for (int i = 0; i < S::P1; ++i) {
                const float4 x = fl[i * st];
                ff_madd2(c[i], make_float2(x.x, x.y), make_float2(x.z, x.w), Rs[p], Re[p]);
            }
        }
    }
}

// Lift of the face fluxes (phase 3 of the stage tile) with float32 pairs, two
// fields at a time: (Rs, Re) -= (2/h_j) l_a(+1)/w_a Fhat(j, +) and += (2/h_j)
// l_a(-1)/w_a times the low face's value (the outward flux inline, G along
// +e_j with the face pass, hence the sign), the high face first as in the
// float64 form.  fh2 holds the face fluxes as (hi, lo) per field.
template <class S, bool PF>
__device__ __forceinline__ void lift_ff(const float2 *fh2, const float2 *cf2, int el, int a,
                                        float2 *Rs, float2 *Re) {
    constexpr int NPR = (S::NF + 1) / 2;
#pragma unroll
    for (int j = 0; j < S::D; ++j) {
        const int aj = digit<S::D, S::P1>(a, j);
        const int q = face_q<S::D, S::P1>(a, j);
        const float2 *fm = fh2 + ((el * S::NFACE + 2 * j) * S::NF) * S::NFP1 + q;
        const float2 *fp = fh2 + ((el * S::NFACE + 2 * j + 1) * S::NF) * S::NFP1 + q;
        const float2 cm = cf2[j * Coef<S>::BLK + Coef<S>::LM + aj];
        const float2 cp = ff_neg(cf2[j * Coef<S>::BLK + Coef<S>::LP + aj]);
        const float2 cmo = PF ? cm : ff_neg(cm);
#pragma unroll
        for (int p = 0; p < NPR; ++p) {
            const bool two = 2 * p + 1 < S::NF;
            const float2 p0 = fp[2 * p * S::NFP1], m0 = fm[2 * p * S::NFP1];
            const float2 p1 = two ? fp[(2 * p + 1) * S::NFP1] : make_float2(0.0f, 0.0f);
            const float2 m1 = two ? fm[(2 * p + 1) * S::NFP1] : make_float2(0.0f, 0.0f);
            ff_madd2(cp, make_float2(p0.x, p1.x), make_float2(p0.y, p1.y), Rs[p], Re[p]);
            ff_madd2(cmo, make_float2(m0.x, m1.x), make_float2(m0.y, m1.y), Rs[p], Re[p]);
        }
    }
}

__device__ __forceinline__ void elem_multi(const MeshData &M, int e, int &i0, int &i1, int &i2) {
    i0 = e % M.n[0];
    const int r = e / M.n[0];
    i1 = r % M.n[1];
    i2 = r / M.n[1];
}

// neighbour across face (j, s) or -1 at a wall
template <int D>
__device__ __forceinline__ int neighbour(const MeshData &M, int e, int j, int s) {
    int i[3];
    elem_multi(M, e, i[0], i[1], i[2]);
    int v = i[j] + s;
    if (v < 0 || v >= M.n[j]) {
        if (!M.periodic[j]) return -1;
        v = (v < 0) ? v + M.n[j] : v - M.n[j];
    }
    i[j] = v;
    return i[0] + M.n[0] * (i[1] + M.n[1] * (D == 3 ? i[2] : 0));
}

template <int D>
__device__ __forceinline__ int vert_index(const MeshData &M, int e) {
    int i0, i1, i2;
    elem_multi(M, e, i0, i1, i2);
    return D == 2 ? i1 : i2;
}

// ---------------------------------------------------------------------------
// Thermodynamics (float64): Eq. (2.3), (2.6), (2.8)
// ---------------------------------------------------------------------------
// rho_vs(T) = e_s(T) / (R_v T) = rho_vs(T_ref) (T/T_ref)^(a-1) exp(b (1/T_ref - 1/T))
__device__ __forceinline__ double rho_vs(double T, double invT) {
    return kRvs0 * exp((kEsA - 1.0) * log(T * kInvTref) + kEsB * (kInvTref - invT));
}

// float32 rho_vs for the pre-solve: rho_vs(T_ref) 2^((a-1) log2(T/T_ref) + b log2(e) (1/T_ref - 1/T))
__device__ __forceinline__ float rho_vs_f32(float T) {
    const float l2e = 1.4426950408889634f;
    return (float)kRvs0 * exp2f((float)(kEsA - 1.0) * __log2f(T * (float)kInvTref) +
                                (float)kEsB * l2e * ((float)kInvTref - __frcp_rn(T)));
}

// float64 rho_vs(T) and d rho_vs / dT from the Taylor table (dg_math.cuh).
// Outside the table range the closed form is evaluated directly.  The
// entry is chosen from the float32-rounded T (within 3e-5 K of T, so
// |T - T_i| <= 1/256 K + 3e-5 K, where the series is still exact to
// float64 rounding); T_i = 150 + i/128 is exact in float32 and widened
// exactly, so the offset needs no float64 <-> integer conversion.
__device__ __forceinline__ double rho_vs_tab(double T, const double *__restrict__ tab, double &d1) {
    const float tf = narrow(T);
    if (!(tf >= (float)kTabT0 && tf <= (float)(kTabT1 - 1.0))) {
        const double invT = 1.0 / T;
        const double v = rho_vs(T, invT);
        d1 = v * invT * fma(kEsB, invT, kEsA - 1.0);
        return v;
    }
    const int i = __float2int_rn((tf - (float)kTabT0) * (float)kTabInvStep);
    const double d = T - widen((float)kTabT0 + (float)i * (float)(1.0 / kTabInvStep));
    const double2 *e = reinterpret_cast<const double2 *>(tab + (size_t)kTabStride * i);
    const double2 c01 = __ldg(e), c23 = __ldg(e + 1), c45 = __ldg(e + 2), c67 = __ldg(e + 3);
    d1 = fma(d, fma(d, c67.y, c67.x), c01.y);
    return fma(d, fma(d, fma(d, fma(d, fma(d, c45.y, c45.x), c23.y), c23.x), c01.y), c01.x);
}

// The same at a float32 temperature t (T = (double)t exactly): the index,
// the range check and the offset d = t - T_i are exact in float32 (T_i =
// 150 + i/128 has 16 significant bits, and t - T_i is exact by Sterbenz's
// lemma), so only the two polynomials run in float64.
__device__ __forceinline__ double rho_vs_tab(float t, const double *__restrict__ tab, double &d1) {
    if (!(t >= (float)kTabT0 && t <= (float)(kTabT1 - 1.0))) return rho_vs_tab(widen(t), tab, d1);
    const int i = __float2int_rn((t - (float)kTabT0) * (float)kTabInvStep);
    const float Ti = (float)kTabT0 + (float)i * (float)(1.0 / kTabInvStep);
    const double d = widen(t - Ti);
    const double2 *e = reinterpret_cast<const double2 *>(tab + (size_t)kTabStride * i);
    const double2 c01 = __ldg(e), c23 = __ldg(e + 1), c45 = __ldg(e + 2), c67 = __ldg(e + 3);
    d1 = fma(d, fma(d, c67.y, c67.x), c01.y);
    return fma(d, fma(d, fma(d, fma(d, fma(d, c45.y, c45.x), c23.y), c23.x), c01.y), c01.x);
}

// float64 rho_vs at a float32 temperature t, value only, for the FP32-bulk
// split: c_0 + c_1 d in float64 and the curvature d^2 (c_2 + c_3 d + c_4 d^2)
// in float32.  The curvature is at most 6.4e-7 of rho_vs (at 150 K; 3e-8 at
// 280 K) and c_5 d^5 below 1e-17, so float32 arithmetic on coefficients
// truncated to float32 leaves below 3e-13 relative (1e-14 above 250 K): two
// float64 fmas instead of the five of the full series.  All of c_0 .. c_4 are
// positive and within the float32 normal range over the table.
__device__ __forceinline__ double rho_vs_bulk(float t, const double *__restrict__ tab) {
    if (!(t >= (float)kTabT0 && t <= (float)(kTabT1 - 1.0))) {
        double d1;
        return rho_vs_tab(widen(t), tab, d1);
    }
    const int i = __float2int_rn((t - (float)kTabT0) * (float)kTabInvStep);
    const float df = t - ((float)kTabT0 + (float)i * (float)(1.0 / kTabInvStep));   // exact
    const double2 *e = reinterpret_cast<const double2 *>(tab + (size_t)kTabStride * i);
    const double2 c01 = __ldg(e), c23 = __ldg(e + 1);
    const float c4 = trunc_f32(__ldg(tab + (size_t)kTabStride * i + 4));
    const float q = fmaf(df, fmaf(df, c4, trunc_f32(c23.y)), trunc_f32(c23.x)) * (df * df);
    return fma(widen(df), c01.y, c01.x) + widen(q);
}

// d rho_vs / dT = rho_vs ((a-1)/T + b/T^2) in float32, from a float32 rho_vs
// and 1/T (the FP32-bulk split's Newton derivative and Taylor step)
__device__ __forceinline__ float drho_vs_f32(float rvs, float invT) {
    return rvs * invT * ((float)(kEsA - 1.0) + (float)kEsB * invT);
}

struct SplitResult {
    double T, rv, deficit;  // deficit = rho_vs(T) - rho_v (0 at saturation)
    bool converged;
};

// Eq. (2.8): T, rho_v from totals rho_d, rho_m, rho_r and internal energy re.
// Unsaturated candidate T_u in closed form; if rho_m > rho_vs(T_u) the vapour
// is saturated and T solves
//   H(T) = (c_vd rd + c_vv rvs + c_l (rm - rvs + rr)) (T - T_ref) + rvs L' - re = 0,
// H increasing and convex.  The saturation test is decided in float32 unless
// rho_m is within 1e-5 of rho_vs (then in float64); the float64 rho_vs(T_u)
// is formed only where the caller needs the evaporation deficit of an
// unsaturated node.  Saturated: Newton's method in float32 from T_u (to
// ~1e-7), then one third-order (Chebyshev) step in float64,
//   d = -H/H',  T = T0 + d - (H''/(2 H')) d^2,
// with H and H' in float64 and the H'' term in float32: from |d| <= 3e-4 K
// (the pre-solve lands within ~5e-5 K) the step leaves an error of order
// (H''/H')^2 d^3 < 2e-13 K, so one float64
// evaluation of rho_vs gives T and rho_v = rho_vs(T) (second-order Taylor
// from T0) to float64 rounding.  A larger |d| falls back to the bracketed
// float64 Newton iteration (cap kMaxNewton).
template <bool NEED_DEFICIT>
__device__ __forceinline__ SplitResult split_point(double rd, double rm, double rr, double re,
                                                   const double *__restrict__ tab,
                                                   int cap = kMaxNewton) {
    SplitResult r;
    // T_u = T_ref + X / C_u.  X (a difference of large terms) is float64; the
    // float32 T_u decides saturation (with a 1e-5 margin) and starts the
    // pre-solve, and the float64 T_u is formed only where it is the answer or
    // the decision is close (saturated nodes need only the float32 value: their
    // root lies above T_u, and the pre-solve ends there)
    // (float32 copies by narrow(), float64 ones of float32 values by widen():
    // integer operations, which keep the FP64 pipe for the arithmetic; the
    // decisions against the float32 rho_vs are float32 compares of the
    // float32-rounded rho_m, exact up to the 1e-5 margin)
    const double X = fma(-rm, kLprime, re);
    const float rmf = narrow(rm);
    const float cuf = (float)kCvd * narrow(rd) + (float)kCvv * rmf + (float)kCl * narrow(rr);
    const float tuf = fmaf(narrow(X), __frcp_rn(cuf), (float)kTref);
    const float rvs32 = rho_vs_f32(tuf);
    bool sat;
    double rvs_u = 0.0, tu = 0.0;
    const bool close = fabsf(rmf - rvs32) <= 1e-5f * rmf || !(tuf > 0.0f);
    if (close || (NEED_DEFICIT && !(rmf > rvs32))) {
        tu = fma(X, recip(kCvd * rd + kCvv * rm + kCl * rr), kTref);
        double d1u;
        rvs_u = rho_vs_tab(tu, tab, d1u);
        sat = rm > rvs_u;
    } else {
        sat = rmf > rvs32;
        if (!sat) tu = fma(X, recip(kCvd * rd + kCvv * rm + kCl * rr), kTref);
    }
    if (!sat) {
        r.T = tu;
        r.rv = rm;
        r.deficit = NEED_DEFICIT ? rvs_u - rm : 0.0;
        r.converged = true;
        return r;
    }
    const double cdry = kCvd * rd + kCl * (rm + rr);
    const float clv = (float)(kCvv - kCl), lp = (float)kLprime;
    const float am1 = (float)(kEsA - 1.0), bb = (float)kEsB;
    // float32 pre-solve
    float t = tuf;
    {
        const float cdf = narrow(cdry), ref = narrow(re), tref = (float)kTref;
        const int n32 = cap < 30 ? cap : 30;
        for (int it = 0; it < n32; ++it) {
            const float rvs = rho_vs_f32(t);
            const float it_ = __frcp_rn(t);
            const float drvs = rvs * it_ * (am1 + bb * it_);
            const float heat = cdf + clv * rvs;
            const float h = heat * (t - tref) + rvs * lp - ref;
            const float dh = heat + (clv * (t - tref) + lp) * drvs;
            const float dt = h * __frcp_rn(dh);
            t -= dt;
            if (fabsf(dt) <= 2e-6f * t) break;
        }
    }
    r.deficit = 0.0;
    // one float64 third-order step from T0
    {
        // t > T_u after a pre-solve from the left of the root; otherwise
        // (pre-solve cut short) start from the float64 T_u
        const bool tf = t > tuf;
        const double t0 = tf ? widen(t) : fma(X, recip(kCvd * rd + kCvv * rm + kCl * rr), kTref);
        double drvs;
        const double rvs = tf ? rho_vs_tab(t, tab, drvs) : rho_vs_tab(t0, tab, drvs);
        const double heat = fma(kCvv - kCl, rvs, cdry);
        const double lat = fma(kCvv - kCl, t0 - kTref, kLprime);
        const double h = fma(heat, t0 - kTref, fma(rvs, kLprime, -re));
        const double dh = fma(lat, drvs, heat);
        const double d = -h * recip(dh);
        if (abs_le(d, 3e-4)) {
            // H'' = 2 (c_vv - c_l) rho_vs' + (c_vv - c_l)(T - T_ref) + L') rho_vs'',
            // rho_vs'' = rho_vs (phi1^2 + phi1'), phi1' = -(a-1)/T^2 - 2b/T^3
            const float itf = __frcp_rn(tf ? t : narrow(t0)), rvf = narrow(rvs);
            const float p1f = itf * (am1 + bb * itf);               // (ln rho_vs)
            const float d2rvs = rvf * (p1f * p1f - itf * itf * (am1 + 2.0f * bb * itf));
            const float d2h = 2.0f * clv * (rvf * p1f) + narrow(lat) * d2rvs;
            const float df = narrow(d);
            const float c2 = -0.5f * d2h / narrow(dh) * df * df;   // second-order term of the step
            const double dc = d + widen(c2);
            const float dcf = narrow(dc);
            r.T = t0 + dc;
            r.rv = fma(drvs, dc, rvs) + widen(0.5f * d2rvs * dcf * dcf);
            r.converged = true;
            return r;
        }
    }
    // fallback: bracketed float64 Newton iteration
    tu = fma(X, recip(kCvd * rd + kCvv * rm + kCl * rr), kTref);
    double tn0 = ((double)t > tu) ? (double)t : tu;
    double lo = tu, hi = INFINITY, rvs = 0.0, drvs = 0.0, step = INFINITY;
    bool done = false;
    for (int it = 0; it < cap; ++it) {
        rvs = rho_vs_tab(tn0, tab, drvs);
        const double heat = fma(kCvv - kCl, rvs, cdry);
        const double h = fma(heat, tn0 - kTref, fma(rvs, kLprime, -re));
        const double dh = fma(fma(kCvv - kCl, tn0 - kTref, kLprime), drvs, heat);
        if (h < 0.0) lo = tn0;
        if (h > 0.0) hi = tn0;
        double tn = tn0 - h * recip(dh);
        if (!(tn >= lo && tn <= hi)) tn = isinf(hi) ? tn0 + 10.0 : 0.5 * (lo + hi);
        step = tn - tn0;
        tn0 = tn;
        if (it >= 1 && fabs(step) <= 1e-10 * tn0) {
            done = true;
            break;
        }
    }
    r.T = tn0;
    // rho_vs at the final T from the last evaluation: the step is below
    // 1e-10 T, so the neglected second-order term is below 1e-20 relative
    r.rv = fma(drvs, step, rvs);
    r.converged = done;
    return r;
}

// v_r = v0 Gamma(4.5)/6 (pi rho_w N0)^(-1/8) rho_r^(1/8) = kvr (rho_r / rho_w)^(1/8) (Section 2.1)
__device__ __forceinline__ double rain_velocity(double rr, double rm, const MeshData &M) {
    const double rw = gt0(M.rho_w) ? M.rho_w : rm + rr;
    if (!gt0(rr) || !gt0(rw)) return 0.0;
    const double rrp = rr;
    const double t = rrp * recip(rw);
    const double y = inv_root8(t);                          // t^(-1/8)
    const double y2 = y * y, y4 = y2 * y2;
    return M.kvr * t * (y4 * y2 * y);                       // t^(1/8) = t y^7
}

__device__ __forceinline__ float rain_velocity(float rr, float rm, const MeshData &M) {
    const float rrp = rr > 0.0f ? rr : 0.0f;
    const float rw = M.rho_w_f > 0.0f ? M.rho_w_f : rm + rr;
    if (!(rrp > 0.0f) || !(rw > 0.0f)) return 0.0f;
    return M.kvr_f * exp2f(0.125f * __log2f(rrp * __frcp_rn(rw)));
}

// Per-node split plus the node-local quantities the next operator needs.
struct NodeDerived {
    double T, rv, pp, gm, vr;
    float Tf, rvf, ppf, gmf, vrf;   // float32 copies (FP32-bulk form)
    float rcf;                      // rho_m - rho_v, perturbation form only
    bool conv, phys;
};

template <bool RAIN>
__device__ __forceinline__ NodeDerived node_derived(double rd, double rm, double rr, double E,
                                                    double msq, double pbar, const MeshData &M,
                                                    const double *__restrict__ tab) {
    NodeDerived o;
    const double rho = rd + rm + rr;
    const double re = E - 0.5 * msq * recip(rho);
    const SplitResult s = split_point<RAIN>(rd, rm, rr, re, tab, M.newton_cap);
    o.T = s.T;
    o.rv = s.rv;
    o.conv = s.converged;
    o.pp = (rd * kRd + s.rv * kRv) * s.T - pbar;
    o.phys = gt0(rd) && gt0(rho) && gt(s.T, 50.0) && lt(s.T, 1000.0) && finite(o.pp);
    o.gm = 0.0;
    o.vr = 0.0;
    if (RAIN) {
        // Eq. (2.4): the rain powers from x = max(rho_r, 0)^(1/16) = r y^15, y = r^(-1/16)
        const bool rpos = gt0(rr);
        const double rrp = rpos ? rr : 0.0;
        double x = 0.0;
        if (rpos) {
            const double y = inv_root16(rrp);
            const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
            x = rrp * (y8 * y4 * y2 * y);
        }
        const double x2 = x * x, x3 = x2 * x, x4 = x2 * x2, x8 = x4 * x4, x14 = x8 * x4 * x2;
        const double rc = rm - s.rv;
        const double s_ev = (kSevA - kSevB * (s.T - kTref)) * (1.0 + kSevC * x3) * s.deficit * x8;
        const double s_au = kSau * (gt0(rc) ? rc : 0.0);
        const double s_ac = kSac * rc * x14;
        o.gm = s_ev - s_au - s_ac;
        // v_r = kvr (rho_r / rho_w)^(1/8) = kvr x^2 rho_w^(-1/8) (Section 2.1)
        const double rw = gt0(M.rho_w) ? M.rho_w : rm + rr;
        o.vr = (rpos && gt0(rw)) ? M.kvr * x2 * inv_root8(rw) : 0.0;
    }
    return o;
}

// T_u = T_ref + X / C_u in float64 from its float32 estimate tuf and
// rcu ~ 1/C_u: with t0 = tuf (exact), the residual X - C_u (t0 - T_ref) is
// C_u times the estimate's error (~1e-5 K), and its float32 quotient
// completes T_u to ~1e-11 K (C_u and three float64 operations instead of a
// float64 reciprocal)
__device__ __forceinline__ double t_unsaturated(double X, double cu, float tuf, float rcu) {
    const double t0 = widen(tuf);
    return t0 + widen(narrow(fma(-cu, t0 - kTref, X)) * rcu);
}

// Split of the FP32-bulk form: the state is float32; the temperature recovery
// from the total energy (the cancellation-prone balance E - |m|^2/(2 rho) -
// rho_m L') and the Newton solve for the saturated vapour density run in
// float64.  Newton iterates in float32 from T_u to ~1e-7, then one float64
// Newton correction with the float64 rho_vs (table, rho_vs_bulk) gives T to
// ~1e-13 and rho_v = rho_vs(T) to ~1e-12, so vapour is never supersaturated
// by more than ~1e-12 relative.  Rain sources and v_r are bulk (float32)
// arithmetic.
template <bool RAIN>
__device__ __forceinline__ NodeDerived node_derived_bulk(const float *u, int im, int ie, int d,
                                                         double brd, double brm, double bE,
                                                         double pbar, float brdf, float brmf,
                                                         const MeshData &M,
                                                         const double *__restrict__ tab,
                                                         float Tprev = -1.0f) {
    NodeDerived o;
    // float32 totals for the saturation test, the pre-solve and the checks
    const float rdf = brdf + u[0], rmf = brmf + u[1], rrf = RAIN ? u[2] : 0.0f;
    const float rhof = rdf + rmf + rrf;
    float msq = 0.0f;
    for (int j = 0; j < d; ++j) msq = fmaf(u[im + j], u[im + j], msq);
    // float64 temperature recovery: T_u = T_ref + (E - |m|^2/(2 rho) - rho_m L') / C_u
    const double rd = brd + widen(u[0]);
    const double rm = brm + widen(u[1]);
    const double rr = RAIN ? widen(u[2]) : 0.0;
    const double re = (bE + widen(u[ie])) - widen(0.5f * msq * __frcp_rn(rhof));
    // T_u = T_ref + X / C_u, X = E_int - rho_m L'.  The float32 T_u (from the
    // float32 X, within ~1e-5 K) decides saturation and starts the pre-solve;
    // X and T_u in float64 are formed only where T = T_u (unsaturated) or the
    // decision is close
    const float ref = narrow(re);
    const float cuf = (float)kCvd * rdf + (float)kCvv * rmf + (float)kCl * rrf;
    const float rcu = __frcp_rn(cuf);
    const float tuf = fmaf(fmaf(-rmf, (float)kLprime, ref), rcu, (float)kTref);
    const float rvs32 = rho_vs_f32(tuf);
    bool sat;
    double tu = 0.0;
    const bool close = fabsf(rmf - rvs32) <= 1e-5f * rmf || !(tuf > 0.0f);
    if (close) {
        tu = t_unsaturated(fma(-rm, kLprime, re), fma(kCvd, rd, fma(kCvv, rm, kCl * rr)), tuf, rcu);
        double d1u;
        sat = rm > rho_vs_tab(tu, tab, d1u);      // close call: decide in float64
    } else {
        sat = rmf > rvs32;
    }
    float deficit = 0.0f, rvf, Tf;
    o.conv = true;
    if (!sat) {
        if (!close)
            tu = t_unsaturated(fma(-rm, kLprime, re), fma(kCvd, rd, fma(kCvv, rm, kCl * rr)), tuf,
                               rcu);
        o.T = tu;
        o.rv = rm;
        Tf = narrow(tu);
        rvf = rmf;
        deficit = rho_vs_f32(Tf) - rmf;
    } else {
        // explicit fma: a contraction left to the compiler may differ between
        // the stage kernel and the ensemble's tile functions
        const float cdf = fmaf((float)kCvd, rdf, (float)kCl * (rmf + rrf));
        const float tref = (float)kTref;
        const float clv = (float)(kCvv - kCl), lp = (float)kLprime;
        // start at this node's temperature of the previous stage when there
        // is one (not below T_u, which lies below the saturated root)
        float t = Tprev > tuf ? Tprev : tuf;
        bool conv = false;
        const int n32 = M.newton_cap < 40 ? M.newton_cap : 40;
        for (int it = 0; it < n32; ++it) {
            const float rvs = rho_vs_f32(t);
            const float drvs = drho_vs_f32(rvs, __frcp_rn(t));
            const float heat = cdf + clv * rvs;
            const float h = heat * (t - tref) + rvs * lp - ref;
            const float dh = heat + (clv * (t - tref) + lp) * drvs;
            const float dt = h * __frcp_rn(dh);
            t -= dt;
            // a step of at most 2e-3 K leaves at most (H''/2H') dt^2 < 2e-7 K;
            // the float64 correction below takes the rest
            if (fabsf(dt) <= 2e-3f) {
                conv = true;
                break;
            }
        }
        // one float64 Newton correction of T: the residual H(t) in float64
        // with the float64 rho_vs(t), the step H/H' in float32 (|dT| is below
        // ~3e-5 K, so its float32 rounding moves T by < 1e-11 K), and
        // rho_v = rho_vs(t) - rho_vs'(t) dT with the float32 derivative (the
        // product is below 2e-6 of rho_vs, so < 1e-12 relative)
        const double T32 = widen(t);
        const double rvs = rho_vs_bulk(t, tab);
        const double cdry = fma(kCvd, rd, kCl * (rm + rr));
        const double h = fma(fma(kCvv - kCl, rvs, cdry), T32 - kTref, fma(rvs, kLprime, -re));
        const float rvsf = narrow(rvs);
        const float drvs = drho_vs_f32(rvsf, __frcp_rn(t));
        const float dh = cdf + clv * rvsf + (clv * (t - tref) + lp) * drvs;
        const float dT = narrow(h) / dh;
        o.T = T32 - widen(dT);
        o.rv = rvs - widen(drvs * dT);
        Tf = narrow(o.T);
        rvf = narrow(o.rv);
        o.conv = conv && fabsf(dT) <= 1e-4f * t;
    }
    // p' = (rho_d R_d + rho_v R_v) T - p_bar in float64 (cancellation against p_bar)
    o.pp = fma(fma(rd, kRd, o.rv * kRv), o.T, -pbar);
    const float ppf = narrow(o.pp);
    o.phys = (rdf > 0.0f) && (rhof > 0.0f) && (Tf > 50.0f) && (Tf < 1000.0f) && isfinite(ppf);
    o.gm = 0.0;
    o.vr = 0.0;
    o.Tf = Tf;
    o.rvf = rvf;
    o.ppf = ppf;
    if (RAIN) {
        const float rrp = rrf > 0.0f ? rrf : 0.0f;
        const float x = rrp > 0.0f ? exp2f(0.0625f * __log2f(rrp)) : 0.0f;
        const float x2 = x * x, x3 = x2 * x, x4 = x2 * x2, x8 = x4 * x4, x14 = x8 * x4 * x2;
        const float rc = rmf - rvf;
        const float s_ev = ((float)kSevA - (float)kSevB * (Tf - (float)kTref)) *
                           (1.0f + (float)kSevC * x3) * deficit * x8;
        const float s_au = (float)kSau * (rc > 0.0f ? rc : 0.0f);
        const float s_ac = (float)kSac * rc * x14;
        o.gmf = s_ev - s_au - s_ac;
        o.vrf = rain_velocity(rrf, rmf, M);
    }
    return o;
}

// ---------------------------------------------------------------------------
// Split in perturbation variables (DG_FP32_PERT)
// ---------------------------------------------------------------------------
// With the base state split once in float64 at every node level
// (T_bar, rho_v_bar), the unknowns are the perturbations tau = T - T_bar and
// nu = rho_v - rho_v_bar.  Subtracting the base identity
// E_bar = C_bar (T_bar - T_ref) + rho_v_bar L' from Eq. (2.8a) leaves
//   H(tau) = C tau + (C - C_bar)(T_bar - T_ref) + nu L' - E' + |m|^2/(2 rho),
//   C - C_bar = c_vd rho_d' + c_l (rho_m' + rho_r') + (c_vv - c_l) nu,
// and Eq. (2.6) gives rho_vs(T_bar + tau) = R_bar (1 + expm1(phi(tau))),
//   phi = (a-1) log1p(tau/T_bar) + (b/T_bar) tau / (T_bar + tau).
// Every term is a perturbation, so float32 resolves T and rho_v to about
// 1e-7 of tau and nu (T to ~1e-9 relative) without the cancellation of the
// direct form; p' = R_d (rho_d' T + rho_d_bar tau) + R_v (nu T + rho_v_bar tau)
// + (p(base split) - p_bar) likewise.
// The float32-rounded base split (T_bar, rho_v_bar) is taken as the exact
// reference; the float64 residuals of its identities are tabulated, so the
// rounding of the reference enters no result.
constexpr int kBsN = 12;  // 0 T_bar, 1 rho_v_bar, 2 R_bar = rho_vs(T_bar), 3 rho_m_bar - R_bar,
                          // 4 R_bar - rho_v_bar, 5 p residual (rho_d R_d + rho_v R_v) T - p, 6 C_bar,
                          // 7 T_bar - T_ref, 8 energy residual E_bar - C_bar (T_bar - T_ref) - rho_v_bar L',
                          // 9 rho_m_bar - rho_v_bar, 10 1/T_bar, 11 b/T_bar

// phi(tau) = (a-1) log1p(tau/T_bar) + (b/T_bar) tau/T with T = T_bar + tau;
// iTb = 1/T_bar and bTb = b/T_bar from the table, iT = 1/T (no divisions)
__device__ __forceinline__ float phi_of(float tau, float iTb, float bTb, float iT) {
    const float am1 = (float)(kEsA - 1.0);
    return am1 * log1pf(tau * iTb) + bTb * (tau * iT);
}

template <bool RAIN>
__device__ __forceinline__ NodeDerived node_derived_pert(const float *u, int im, int ie, int d,
                                                         float brd, float brm, const float *bs,
                                                         int nl, const MeshData &M,
                                                         float Tprev = -1.0f) {
    NodeDerived o;
    const float Tb = bs[0], rvb = bs[nl], Rb = bs[2 * nl], Qb = bs[3 * nl], Db = bs[4 * nl];
    const float pres = bs[5 * nl], Cb = bs[6 * nl], dTb = bs[7 * nl], eres = bs[8 * nl];
    const float cqb = bs[9 * nl], iTb = bs[10 * nl], bTb = bs[11 * nl];
    const float cvd = (float)kCvd, cvv = (float)kCvv, cl = (float)kCl, lp = (float)kLprime;
    const float rdp = u[0], rmp = u[1], rrp = RAIN ? u[2] : 0.0f;
    const float rho = brd + brm + rdp + rmp + rrp;
    float msq = 0.0f;
    for (int j = 0; j < d; ++j) msq = fmaf(u[im + j], u[im + j], msq);
    // rho e - (base identity) = E' - |m|^2/(2 rho) + energy residual
    const float de = (u[ie] - 0.5f * msq * __frcp_rn(rho)) + eres;
    const float c0 = cvd * rdp + cl * (rmp + rrp);            // C - C_bar without the nu part
    // unsaturated candidate: rho_v = rho_m, nu_u = rho_m' + (rho_m_bar - rho_v_bar)
    const float nu_u = rmp + cqb;
    const float Cu = Cb + c0 + (cvv - cl) * nu_u;
    const float tau_u = (de - (c0 + (cvv - cl) * nu_u) * dTb - nu_u * lp) * __frcp_rn(Cu);
    // saturated iff rho_m > rho_vs(T_u) <=> rho_m' + Q_bar - R_bar expm1(phi(tau_u)) > 0
    const float em_u = expm1f(phi_of(tau_u, iTb, bTb, __frcp_rn(Tb + tau_u)));
    const bool sat = rmp + Qb - Rb * em_u > 0.0f;
    float tau, nu, deficit = 0.0f;
    bool conv = true;
    if (!sat) {
        tau = tau_u;
        nu = nu_u;
        deficit = (Db + Rb * em_u) - nu_u;                     // rho_vs(T) - rho_v
    } else {
        // start at this node's temperature of the previous stage (a stage
        // moves it by ~1e-3 K), else at the base temperature; not below T_u,
        // which lies below the saturated root.  Where the base state is
        // cloudy T_u lies ~ rho_c L'/C (a few K) below the root, while the
        // root is usually within a fraction of a K of T_bar.  H is increasing
        // and convex, so Newton converges from either side.
        const float tau_p = Tprev > 0.0f ? Tprev - Tb : 0.0f;
        tau = tau_u > tau_p ? tau_u : tau_p;
        conv = false;
        const float am1 = (float)(kEsA - 1.0), bb = (float)kEsB;
        float prev = 3.0e38f;
        bool have_nu = false;
        const int n32 = M.newton_cap < 40 ? M.newton_cap : 40;
        for (int it = 0; it < n32; ++it) {
            const float T = Tb + tau;
            const float iT = __frcp_rn(T);
            const float em = expm1f(phi_of(tau, iTb, bTb, iT));
            const float nus = Db + Rb * em;                     // rho_vs(T) - rho_v_bar
            const float p1 = iT * (am1 + bb * iT);              // d phi / d tau
            const float dnu = Rb * (1.0f + em) * p1;
            const float C = Cb + c0 + (cvv - cl) * nus;
            const float h = C * tau + (c0 + (cvv - cl) * nus) * dTb + nus * lp - de;
            const float dh = C + ((cvv - cl) * (tau + dTb) + lp) * dnu;
            const float step = h * __frcp_rn(dh);
            tau -= step;
            // done once the step s is at most 2e-3 K: Newton leaves an error
            // of at most (H''/2H') s^2, and H''/2H' < 0.05 /K on the saturated
            // branch (0.023 /K at 300 K), so at most 2e-7 K remains; or once
            // the step stops shrinking (float32 rounding of h then decides
            // the last bits and the iteration only dithers)
            const float as = fabsf(step);
            if (as <= 2e-3f || (as <= 1e-2f && as >= 0.5f * prev)) {
                // nu at the new tau by Taylor from this evaluation:
                // nu'' = R_bar e^phi (phi'^2 + phi''), and the omitted third-order
                // term, ~ rho_vs phi'^3 s^3 / 6, is below 1e-12 kg/m^3 for |s| <= 1e-2 K
                const float p2 = -iT * iT * (am1 + 2.0f * bb * iT);
                const float d2nu = Rb * (1.0f + em) * (p1 * p1 + p2);
                nu = fmaf(0.5f * d2nu * step, step, fmaf(-dnu, step, nus));
                have_nu = true;
                conv = true;
                break;
            }
            prev = as;
        }
        if (!have_nu) nu = Db + Rb * expm1f(phi_of(tau, iTb, bTb, __frcp_rn(Tb + tau)));
    }
    const float T = Tb + tau;
    o.Tf = T;
    o.rvf = rvb + nu;
    o.rcf = rmp + cqb - nu;                                    // exactly 0 when unsaturated
    // p' = (rho_d R_d + rho_v R_v) T - p_bar in perturbation form
    o.ppf = (float)kRd * (rdp * T + brd * tau) + (float)kRv * (nu * T + rvb * tau) + pres;
    o.T = (double)Tb + (double)tau;
    o.rv = (double)rvb + (double)nu;
    o.pp = (double)o.ppf;
    o.conv = conv;
    o.phys = (brd + rdp > 0.0f) && (rho > 0.0f) && (T > 50.0f) && (T < 1000.0f) && isfinite(o.ppf);
    o.gm = 0.0;
    o.vr = 0.0;
    o.gmf = 0.0f;
    o.vrf = 0.0f;
    if (RAIN) {
        const float rr = rrp > 0.0f ? rrp : 0.0f;
        const float x = rr > 0.0f ? exp2f(0.0625f * __log2f(rr)) : 0.0f;
        const float x2 = x * x, x3 = x2 * x, x4 = x2 * x2, x8 = x4 * x4, x14 = x8 * x4 * x2;
        const float rc = o.rcf;
        const float s_ev = ((float)kSevA - (float)kSevB * (T - (float)kTref)) *
                           (1.0f + (float)kSevC * x3) * deficit * x8;
        const float s_au = (float)kSau * (rc > 0.0f ? rc : 0.0f);
        const float s_ac = (float)kSac * rc * x14;
        o.gmf = s_ev - s_au - s_ac;
        o.vrf = rain_velocity(rrp, brm + rmp, M);
    }
    return o;
}

// float64 split of the base state at every node level -> the tables above
static __global__ void k_base_split(const double *bnode, int nl, float *bs, const double *tab) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const double rd = bnode[l], rm = bnode[nl + l], E = bnode[2 * nl + l], p = bnode[3 * nl + l];
    const SplitResult r = split_point<false>(rd, rm, 0.0, E, tab);
    const double T = (double)(float)r.T, rv = (double)(float)r.rv;   // the float32 reference
    const double R = rho_vs(T, 1.0 / T);
    const double C = kCvd * rd + kCvv * rv + kCl * (rm - rv);
    bs[l] = (float)T;
    bs[nl + l] = (float)rv;
    bs[2 * nl + l] = (float)R;
    bs[3 * nl + l] = (float)(rm - R);
    bs[4 * nl + l] = (float)(R - rv);
    bs[5 * nl + l] = (float)((rd * kRd + rv * kRv) * T - p);
    bs[6 * nl + l] = (float)C;
    bs[7 * nl + l] = (float)(T - kTref);
    bs[10 * nl + l] = (float)(1.0 / T);
    bs[11 * nl + l] = (float)(kEsB / T);
    bs[8 * nl + l] = (float)(E - C * (T - kTref) - rv * kLprime);
    bs[9 * nl + l] = (float)(rm - rv);
}

// ---------------------------------------------------------------------------
// Pointwise flux of Eq. (2.11) and the wave-speed bound of Eq. (3.4)
// ---------------------------------------------------------------------------
template <int D, bool RAIN, typename Real>
struct Prim {
    Real rd, rm, rr, rho, irho, E, p, pp, T, rv, vr;
    Real m[D], u[D];
};

template <class S, typename Real>
__device__ __forceinline__ void make_prim(Prim<S::D, S::RAIN, Real> &P, const Real *U, Real brd,
                                          Real brm, Real bE, Real bp, Real T, Real rv, Real pp) {
    P.rd = brd + U[0];
    P.rm = brm + U[1];
    P.rr = S::RAIN ? U[2] : Real(0);
    P.rho = P.rd + P.rm + P.rr;
    const Real inv = recip(P.rho);
    P.irho = inv;
#pragma unroll
    for (int j = 0; j < S::D; ++j) {
        P.m[j] = U[S::IM + j];
        P.u[j] = P.m[j] * inv;
    }
    P.E = bE + U[S::IE];
    P.pp = pp;
    P.p = bp + pp;
    P.T = T;
    P.rv = rv;
    P.vr = Real(0);
}

// F_j(U): rho_d u_j, rho_m u_j, rho_r (u_j - v_r d_jz), m_i u_j - rho_r v_r u_i d_jz + p' d_ij,
//         (E + p) u_j - (c_l (T - T_ref) + |u|^2/2) rho_r v_r d_jz
template <class S, typename Real>
__device__ __forceinline__ void flux_dir(const Prim<S::D, S::RAIN, Real> &P, int j, Real *F) {
    const bool vert = (j == S::VERT);
    const Real uj = P.u[j];
    F[0] = P.rd * uj;
    F[1] = P.rm * uj;
    const Real rvr = (S::RAIN && vert) ? P.rr * P.vr : Real(0);
    if (S::RAIN) F[2] = P.rr * uj - rvr;
#pragma unroll
    for (int i = 0; i < S::D; ++i) {
        Real f = P.m[i] * uj;
        if (S::RAIN && vert) f -= rvr * P.u[i];
        if (i == j) f += P.pp;
        F[S::IM + i] = f;
    }
    Real fe = (P.E + P.p) * uj;
    if (S::RAIN && vert) {
        Real ke = Real(0);
#pragma unroll
        for (int i = 0; i < S::D; ++i) ke += P.u[i] * P.u[i];
        fe -= (Real(kCl) * (P.T - Real(kTref)) + Real(0.5) * ke) * rvr;
    }
    F[S::IE] = fe;
}

// |u.n| + |v_r e_z.n| + c_m, c_m = sqrt(gamma_m p / rho), gamma_m = (c_v + R)/c_v
// (c_v, R per unit volume: c_vd rho_d + c_vv rho_v + c_l (rho_c + rho_r), R_d rho_d + R_v rho_v)
template <class S, int J, typename Real>
__device__ __forceinline__ Real wave_speed(const Prim<S::D, S::RAIN, Real> &P) {
    const Real rc = P.rm - P.rv;
    const Real cv = Real(kCvd) * P.rd + Real(kCvv) * P.rv + Real(kCl) * (rc + P.rr);
    // c_m = sqrt(num / den) = num / sqrt(num den): one reciprocal square root
    const Real num = (cv + Real(kRd) * P.rd + Real(kRv) * P.rv) * P.p;
    const Real nd = num * (cv * P.rho);
    Real lam = fabs(P.u[J]) + (gt0(nd) ? num * rsqrt_nr(nd) : Real(0));
    if (S::RAIN && J == S::VERT) lam += fabs(P.vr);
    return lam;
}

// a + b rounded once, never fused with the products that formed a or b: the
// face flux sums F- + F+ this way so that the result does not depend on the
// order of the two sides
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// trace of a nodal field on face (j, s) at face point q: sum_i l_i(s) v(line node i)
template <class S, typename Real>
__device__ __forceinline__ Real interp_face(const Real *v, const Real *ls, int j, int q) {
    Real acc = Real(0);
#pragma unroll
    for (int i = 0; i < S::P1; ++i) acc = fma(ls[i], v[line_node<S::D, S::P1>(j, q, i)], acc);
    return acc;
}

// Which trace fields a face carries: T enters the face flux only through the
// rain's energy flux on faces normal to e_z, so the other faces hold no
// temperature trace (its slot in the trace buffer is neither written nor read)
template <class S>
__host__ __device__ constexpr bool has_trace(int fld, int j) {
    return fld != S::NF || j == S::VERT;
}

// ---------------------------------------------------------------------------
// k_prepare: split at every node and traces of every face
// ---------------------------------------------------------------------------
// Traces on the two faces normal to e_J through face point q of element el:
// the k+1 node values of the line are read once and interpolated to both
// ends (same fma chain as interp_face).  DIFF: also the traces of
// d/dx_J U, (2/h_J) sum_i l_i'(+-1) U(line node i), for the interior-penalty
// terms.
template <class S, typename Real, bool DIFF, int J>
__device__ __forceinline__ void write_line(const KArgs<Real> &A, const RefData<Real> &ref,
                                           const Real *s_tr, Real *trace_out, int el, int e, int q) {
    constexpr int STR = S::EPB * S::NP;
    const int ne = A.M.ne;
    const int b0 = el * S::NP + line_node<S::D, S::P1>(J, q, 0);
    constexpr int st = J == 0 ? 1 : (J == 1 ? S::P1 : S::P1 * S::P1);
    Real *om = trace_out + ((size_t)(2 * J) * S::NTR * ne + e) * S::NFP1 + q;
    Real *op = trace_out + ((size_t)(2 * J + 1) * S::NTR * ne + e) * S::NFP1 + q;
    const size_t fs = (size_t)ne * S::NFP1;
#pragma unroll
    for (int fld = 0; fld < S::NTR; ++fld) {
        if (!has_trace<S>(fld, J)) continue;
        Real v[S::P1];
#pragma unroll
        for (int i = 0; i < S::P1; ++i) v[i] = s_tr[fld * STR + b0 + i * st];
        Real am = Real(0), ap = Real(0);
#pragma unroll
        for (int i = 0; i < S::P1; ++i) {
            am = fma(ref.lm[i], v[i], am);
            ap = fma(ref.lp[i], v[i], ap);
        }
        om[fld * fs] = am;
        op[fld * fs] = ap;
        if (DIFF && fld < S::NF) {
            Real dm = Real(0), dp = Real(0);
#pragma unroll
            for (int i = 0; i < S::P1; ++i) {
                dm = fma(ref.dlm[i], v[i], dm);
                dp = fma(ref.dlp[i], v[i], dp);
            }
            const Real sc = mconst<Real>(A.M.two_over_h[J], A.M.two_over_h_f[J]);
            A.dtrace_out[(((size_t)(2 * J) * S::NF + fld) * ne + e) * S::NFP1 + q] = sc * dm;
            A.dtrace_out[(((size_t)(2 * J + 1) * S::NF + fld) * ne + e) * S::NFP1 + q] = sc * dp;
        }
    }
}

// One thread per face point: the float64 form, whose FP64 pipe is the bound,
// runs faster with the trace work spread over more threads (measured).
template <class S, typename Real, bool DIFF>
__device__ __forceinline__ void write_traces_points(const KArgs<Real> &A, const RefData<Real> &ref,
                                                    const Real *s_tr, Real *trace_out, int bidx) {
    const int ne = A.M.ne;
    for (int item = threadIdx.x; item < S::EPB * S::NFACE * S::NFP1; item += S::NT) {
        const int el = item / (S::NFACE * S::NFP1);
        const int rem = item - el * (S::NFACE * S::NFP1);
        const int face = rem / S::NFP1;
        const int q = rem - face * S::NFP1;
        const int e = bidx * S::EPB + el;
        if (e >= ne) continue;
        const int j = face >> 1;
        const Real *ls = (face & 1) ? ref.lp : ref.lm;
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) {
            if (!has_trace<S>(fld, j)) continue;
            const Real *v = s_tr + (size_t)fld * S::EPB * S::NP + el * S::NP;
            trace_out[(((size_t)face * S::NTR + fld) * ne + e) * S::NFP1 + q] =
                interp_face<S, Real>(v, ls, j, q);
        }
        if (DIFF) {
            const Real *dls = (face & 1) ? ref.dlp : ref.dlm;
            const Real sc = mconst<Real>(A.M.two_over_h[j], A.M.two_over_h_f[j]);
#pragma unroll
            for (int fld = 0; fld < S::NF; ++fld) {
                const Real *v = s_tr + (size_t)fld * S::EPB * S::NP + el * S::NP;
                A.dtrace_out[(((size_t)face * S::NF + fld) * ne + e) * S::NFP1 + q] =
                    sc * interp_face<S, Real>(v, dls, j, q);
            }
        }
    }
}

// Traces of the tile's state on all 2D faces.  float32: one thread per line
// (both ends; the float32 tile is bound by instruction issue, and this halves
// the shared-memory reads and index work, measured -22 % per step);
// float64: one thread per face point (write_traces_points).
template <class S, typename Real, bool DIFF = false>
__device__ __forceinline__ void write_traces(const KArgs<Real> &A, const RefData<Real> &ref,
                                             const Real *s_tr, Real *trace_out, int bidx) {
    if (sizeof(Real) == sizeof(double)) {
        write_traces_points<S, Real, DIFF>(A, ref, s_tr, trace_out, bidx);
        return;
    }
    const int ne = A.M.ne;
    for (int item = threadIdx.x; item < S::EPB * S::D * S::NFP1; item += S::NT) {
        const int el = item / (S::D * S::NFP1);
        const int rem = item - el * (S::D * S::NFP1);
        const int j = rem / S::NFP1;
        const int q = rem - j * S::NFP1;
        const int e = bidx * S::EPB + el;
        if (e >= ne) continue;
        switch (j) {
            case 0: write_line<S, Real, DIFF, 0>(A, ref, s_tr, trace_out, el, e, q); break;
            case 1: write_line<S, Real, DIFF, 1>(A, ref, s_tr, trace_out, el, e, q); break;
            default:
                write_line<S, Real, DIFF, (S::D == 3 ? 2 : 1)>(A, ref, s_tr, trace_out, el, e, q);
                break;
        }
    }
}

// ---------------------------------------------------------------------------
// Artificial diffusion helpers (Section 3.5)
// ---------------------------------------------------------------------------
// weight W_a |K|/2^d of node a times |u|^2 and |u - v_r e_z|^2, added to the
// element's sums s_red[0..1] (shared memory)
template <class S, typename Real>
__device__ __forceinline__ void alpha_accumulate(const KArgs<Real> &A, const RefData<Real> &ref,
                                                 const Real *u, Real vr, int a, int lev,
                                                 Real *s_red) {
    const int nl = A.M.nzlev_node;
    const Real rho = (A.bnode[lev] + u[0]) + (A.bnode[nl + lev] + u[1]) + (S::RAIN ? u[2] : Real(0));
    const Real inv = recip(rho);
    Real wq = mconst<Real>(A.M.jac, A.M.jac_f);
#pragma unroll
    for (int j = 0; j < S::D; ++j) wq *= ref.w[digit<S::D, S::P1>(a, j)];
    Real w2u = Real(0), w2r = Real(0);
#pragma unroll
    for (int j = 0; j < S::D; ++j) {
        const Real uj = u[S::IM + j] * inv;
        w2u = fma(uj, uj, w2u);
        const Real ur = (j == S::VERT) ? uj - vr : uj;
        w2r = fma(ur, ur, w2r);
    }
    atomicAdd(&s_red[0], wq * w2u);
    if (S::RAIN) atomicAdd(&s_red[1], wq * w2r);
}

// alpha_K = alpha_pre ||w||_{0,K} from the element sums (threads t < EPB)
template <class S, typename Real>
__device__ __forceinline__ void alpha_store(const KArgs<Real> &A, const Real *s_red, int bidx) {
    const int t = threadIdx.x;
    if (t < S::EPB) {
        const int e = bidx * S::EPB + t;
        if (e < A.M.ne) {
            const Real pre = mconst<Real>(A.M.alpha_pre, A.M.alpha_pre_f);
            A.alphaK[e] = pre * sqrt(s_red[2 * t]);
            A.alphaK[A.M.ne + e] = S::RAIN ? pre * sqrt(s_red[2 * t + 1]) : Real(0);
        }
    }
}

// the element's 2^d vertex values of the continuous coefficient (alpha_u, then
// alpha_r), corner c = sum_j b_j 2^j at vertex im + b
template <class S, typename Real>
__device__ __forceinline__ void alpha_corners(const KArgs<Real> &A, const int *im, Real *out) {
    const MeshData &M = A.M;
    const int nvt = M.nv[0] * M.nv[1] * (S::D == 3 ? M.nv[2] : 1);
#pragma unroll
    for (int c = 0; c < S::NCORNER; ++c) {
        int v[3] = {0, 0, 0};
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            v[j] = im[j] + ((c >> j) & 1);
            if (v[j] >= M.nv[j]) v[j] -= M.n[j];     // periodic wrap (nv = n)
        }
        const int flat = v[0] + M.nv[0] * (v[1] + M.nv[1] * v[2]);
        out[c] = A.alphaV[flat];
        out[S::NCORNER + c] = A.alphaV[nvt + flat];
    }
}

// Q1 interpolant at reference point xi[0..D) of corner values cv[NCORNER]
// (corner c = sum_j b_j 2^j): D rounds of linear interpolation, first along
// x (2^(D-1) pairs), then y, then z
template <class S, typename Real>
__device__ __forceinline__ Real q1_interp(const Real *cv, const Real *xi) {
    Real v[S::NCORNER];
#pragma unroll
    for (int c = 0; c < S::NCORNER; ++c) v[c] = cv[c];
#pragma unroll
    for (int j = 0; j < S::D; ++j) {
        const Real t = Real(0.5) * (Real(1) + xi[j]);
#pragma unroll
        for (int k = 0; k < (S::NCORNER >> (j + 1)); ++k) v[k] = fma(t, v[2 * k + 1] - v[2 * k], v[2 * k]);
    }
    return v[0];
}

// vertex values of the continuous coefficient: mean of alpha_K over the
// elements sharing the vertex (lumped L2 projection onto continuous Q1)
template <int D, typename Real>
__global__ void k_alpha_vertex(MeshData M, const Real *alphaK, Real *alphaV) {
    const int nvt = M.nv[0] * M.nv[1] * (D == 3 ? M.nv[2] : 1);
    for (int gid = blockIdx.x * blockDim.x + threadIdx.x; gid < nvt; gid += gridDim.x * blockDim.x) {
        int v[3];
        v[0] = gid % M.nv[0];
        const int r = gid / M.nv[0];
        v[1] = D == 3 ? r % M.nv[1] : r;
        v[2] = D == 3 ? r / M.nv[1] : 0;
        Real su = Real(0), sr = Real(0);
        int cnt = 0;
        for (int c = 0; c < (1 << D); ++c) {
            int ei[3] = {0, 0, 0};
            bool ok = true;
            for (int j = 0; j < D; ++j) {
                int x = v[j] - 1 + ((c >> j) & 1);
                if (M.periodic[j]) {
                    if (x < 0) x += M.n[j];
                } else if (x < 0 || x >= M.n[j]) {
                    ok = false;
                }
                ei[j] = x;
            }
            if (!ok) continue;
            const int e = ei[0] + M.n[0] * (ei[1] + M.n[1] * ei[2]);
            su += alphaK[e];
            sr += alphaK[M.ne + e];
            ++cnt;
        }
        alphaV[gid] = su / Real(cnt);
        alphaV[nvt + gid] = sr / Real(cnt);
    }
}

// Tprev: this node's temperature at the previous stage (a start for the
// float32 Newton iterations), or <= 0 when there is none
template <class S>
__device__ __forceinline__ NodeDerived derive_node(const double *u, const KArgs<double> &A, int lev,
                                                   double Tprev = -1.0) {
    (void)Tprev;
    const int nl = A.M.nzlev_node;
    double msq = 0.0;
#pragma unroll
    for (int j = 0; j < S::D; ++j) msq += u[S::IM + j] * u[S::IM + j];
    return node_derived<S::RAIN>(A.bnode_d[lev] + u[0], A.bnode_d[nl + lev] + u[1],
                                 S::RAIN ? u[2] : 0.0, A.bnode_d[2 * nl + lev] + u[S::IE], msq,
                                 A.bnode_d[3 * nl + lev], A.M, A.rvs_tab);
}

template <class S>
__device__ __forceinline__ NodeDerived derive_node(const float *u, const KArgs<float> &A, int lev,
                                                   float Tprev = -1.0f) {
    const int nl = A.M.nzlev_node;
    if (A.M.pert_split)
        return node_derived_pert<S::RAIN>(u, S::IM, S::IE, S::D, A.bnode[lev], A.bnode[nl + lev],
                                          A.bsplit + lev, nl, A.M, Tprev);
    return node_derived_bulk<S::RAIN>(u, S::IM, S::IE, S::D, A.bnode_d[lev], A.bnode_d[nl + lev],
                                      A.bnode_d[2 * nl + lev], A.bnode_d[3 * nl + lev],
                                      A.bnode[lev], A.bnode[nl + lev], A.M, A.rvs_tab, Tprev);
}

// STRIDE: nodes per field row of s_tr (0: the stage tile's EPB NP)
template <class S, typename Real, bool DIFF = false, int STRIDE = 0>
__device__ __forceinline__ void split_and_store(const KArgs<Real> &A, const Real *u, int e, int a,
                                                int iz, Real *s_tr, int t, Real *s_red = nullptr,
                                                Real Tprev = Real(-1)) {
    const size_t nodes = (size_t)A.M.ne * S::NP;
    const size_t gi = (size_t)e * S::NP + a;
    const int lev = iz * S::P1 + digit<S::D, S::P1>(a, S::VERT);
    const NodeDerived nd = derive_node<S>(u, A, lev, Tprev);
    if (!nd.conv) atomicAdd(&A.flags[0], 1ull);
    if (!nd.phys) atomicAdd(&A.flags[1], 1ull);
    Real T, rv, pp, gm, vr;
    if (sizeof(Real) == sizeof(float)) {
        T = (Real)nd.Tf;
        rv = (Real)nd.rvf;
        pp = (Real)nd.ppf;
        gm = (Real)nd.gmf;
        vr = (Real)nd.vrf;
    } else {
        T = (Real)nd.T;
        rv = (Real)nd.rv;
        pp = (Real)nd.pp;
        gm = (Real)nd.gm;
        vr = (Real)nd.vr;
    }
    A.derived[gi] = T;
    A.derived[nodes + gi] = rv;
    A.derived[2 * nodes + gi] = pp;
    if (S::RAIN) {
        A.derived[3 * nodes + gi] = gm;
        A.derived[4 * nodes + gi] = vr;
    }
    if (DIFF) alpha_accumulate<S, Real>(A, A.ref, u, vr, a, lev, s_red + 2 * (t / S::NP));
    const int str = STRIDE > 0 ? STRIDE : S::EPB * S::NP;
#pragma unroll
    for (int f = 0; f < S::NF; ++f) s_tr[f * str + t] = u[f];
    s_tr[S::NF * str + t] = T;
    s_tr[(S::NF + 1) * str + t] = rv;
    s_tr[(S::NF + 2) * str + t] = pp;
}

// DIFF: also the element coefficients alpha_K and the derivative traces
template <class S, typename Real, bool DIFF>
__global__ void __launch_bounds__(S::NT) k_prepare(KArgs<Real> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *s_tr = reinterpret_cast<Real *>(smem_raw);  // [NTR][EPB*NP]
    Real *s_red = s_tr + S::NTR * S::EPB * S::NP;    // [EPB][2]
    const int t = threadIdx.x;
    const int el = t / S::NP, a = t - el * S::NP;
    const int bidx = blockIdx.x + A.tile0;
    const int e = bidx * S::EPB + el;
    const bool valid = (t < S::EPB * S::NP) && (e < A.M.ne);
    if (DIFF) {
        if (t < 2 * S::EPB) s_red[t] = Real(0);
        __syncthreads();
    }
    if (valid) {
        const size_t nodes = (size_t)A.M.ne * S::NP;
        const size_t gi = (size_t)e * S::NP + a;
        Real u[S::NF];
#pragma unroll
        for (int f = 0; f < S::NF; ++f) u[f] = A.Uin[f * nodes + gi];
        split_and_store<S, Real, DIFF>(A, u, e, a, vert_index<S::D>(A.M, e), s_tr, t, s_red);
    }
    __syncthreads();
    if (DIFF) alpha_store<S, Real>(A, s_red, bidx);
    write_traces<S, Real, DIFF>(A, A.ref, s_tr, A.trace_out, bidx);
}

// ---------------------------------------------------------------------------
// k_stage: dU/dt of Eq. (3.2) per element, then MODE_RHS or MODE_STAGE
// ---------------------------------------------------------------------------
constexpr int MODE_RHS = 0;
constexpr int MODE_STAGE = 1;

// Shared memory of a stage tile: nodal fluxes s_fl (fl_index), node
// values for the traces s_tr [NTR][EPB NP], outward face fluxes s_fh
// [EPB][2D][NFP][NFP1] (with diffusion NFP = 2 NF: the fluxes, then the
// symmetry terms), per-element indices, with diffusion the element's vertex
// coefficients [EPB][2][2^D] and its alpha sums [EPB][2], and (float64) the
// coefficient tables s_cf (Coef).  s_tr is needed before the volume phase
// only when the float32 inline form interpolates its own traces in the face
// phase, or with diffusion (the derivatives of the node values); otherwise
// it is filled after the volume phase and shares s_fl.
template <class S, typename Real, bool PF, bool DIFF = false>
__host__ __device__ constexpr bool tr_shares_fl() {
    return (PF || sizeof(Real) == sizeof(double)) && !DIFF;
}

// byte offset of s_fh (16-byte aligned for the asynchronous copy of the face fluxes)
template <class S, typename Real, bool PF, bool DIFF>
__host__ __device__ constexpr size_t stage_fh_offset() {
    constexpr size_t FL = (size_t)S::D * fl_words<S, Real>();
    return ((sizeof(Real) * (tr_shares_fl<S, Real, PF, DIFF>()
                                 ? (FL > (size_t)S::NTR ? FL : (size_t)S::NTR)
                                 : FL + S::NTR) *
             S::EPB * S::NP) + 15) / 16 * 16;
}

// byte offset of the coefficient tables s_cf (Coef; 16-byte aligned)
template <class S, typename Real, bool PF, bool DIFF>
__host__ __device__ constexpr size_t stage_cf_offset() {
    constexpr size_t fh = (size_t)S::EPB * S::NFACE * (DIFF ? 2 * S::NF : S::NF) * S::NFP1;
    return (stage_fh_offset<S, Real, PF, DIFF>() + sizeof(Real) * fh +
            sizeof(int) * 16 * (size_t)S::EPB +  // per element: 2D neighbours, vertical index
            (DIFF ? sizeof(Real) * (size_t)S::EPB * (2 * S::NCORNER + 2) : 0) + 15) / 16 * 16;
}

template <class S, typename Real, bool PF = false, bool DIFF = false>
constexpr size_t stage_smem_bytes() {
    return stage_cf_offset<S, Real, PF, DIFF>() +
           (sizeof(Real) == sizeof(double) ? sizeof(Real) * (size_t)Coef<S>::N : 0);
}

// completes the asynchronous copies issued by this thread
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The tile's face values from the face pass's face-major buffer
// (fbuf [faces][NFP][NFP1]; ftab [ne][2D] gives each element's faces) to
// s_fh [EPB][2D][NFP][NFP1]: one contiguous block per face, copied
// asynchronously in CHUNK-byte pieces by all threads; completed by
// cp_async_wait_all.
template <class S, typename Real, int NFP>
__device__ __forceinline__ void cp_async_faces(const Real *fbuf, const int *ftab, Real *s_fh,
                                               int bidx, int nel) {
    constexpr size_t FB = sizeof(Real) * (size_t)NFP * S::NFP1;   // bytes per face
    constexpr int CHUNK = FB % 16 == 0 ? 16 : (FB % 8 == 0 ? 8 : 4);
    constexpr int NCH = (int)(FB / CHUNK);
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(s_fh);
    const char *g = reinterpret_cast<const char *>(fbuf);
    for (int item = threadIdx.x; item < nel * S::NFACE * NCH; item += blockDim.x) {
        const int ef = item / NCH, ch = item - ef * NCH;            // (element, face), piece
        const int fidx = __ldg(ftab + (size_t)bidx * S::EPB * S::NFACE + ef);
        const char *src = g + (size_t)fidx * FB + (size_t)ch * CHUNK;
        const unsigned dst = sbase + (unsigned)((size_t)ef * FB + (size_t)ch * CHUNK);
        if (CHUNK == 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
        else if (CHUNK == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src));
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src));
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

// neighbour element across face (j, s) from the element's multi-index, or -1 (wall)
template <int D>
__device__ __forceinline__ int neighbour_of(const MeshData &M, const int *im, int j, int s) {
    int v = im[j] + s;
    if (v < 0 || v >= M.n[j]) {
        if (!M.periodic[j]) return -1;
        v = (v < 0) ? v + M.n[j] : v - M.n[j];
    }
    const int i0 = j == 0 ? v : im[0], i1 = j == 1 ? v : im[1], i2 = j == 2 ? v : im[2];
    return i0 + M.n[0] * (i1 + M.n[1] * (D == 3 ? i2 : 0));
}

template <class S, typename Real>
__device__ __forceinline__ void load_base(const Real *tab, int nlev, int lev, Real &rd, Real &rm,
                                          Real &E, Real &p) {
    rd = tab[lev];
    rm = tab[nlev + lev];
    E = tab[2 * nlev + lev];
    p = tab[3 * nlev + lev];
}

// Lax-Friedrichs flux F_n = {{F}}.n + Lambda/2 [[U]] (Section 3.2) at face point q of
// face (J, s) of element e2, in the outward direction s e_J; own trace from
// shared memory, neighbour trace from the trace buffer, slip-wall ghost state
// m+ = m- - 2 (m-.n) n with everything else copied.
template <class S, typename Real, int J>
__device__ __forceinline__ void face_point(const KArgs<Real> &A, const RefData<Real> &ref,
                                           const Real *s_tr, Real *s_fh, int el2, int face, int q,
                                           int e2, int nb, int iz) {
    constexpr int STR = S::EPB * S::NP;
    const MeshData &M = A.M;
    const int ne = M.ne;
    const int s = (face & 1) ? 1 : -1;
    const Real *ls = (face & 1) ? ref.lp : ref.lm;
    Real tm[S::NTR], tp[S::NTR];
    if (sizeof(Real) == sizeof(double)) {
        // float64 form: the own trace was written with the same interpolation
        // when this state was produced; reading it back saves float64 work
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            tm[fld] = has_trace<S>(fld, J)
                          ? A.trace_in[(((size_t)face * S::NTR + fld) * ne + e2) * S::NFP1 + q]
                          : Real(0);
    } else {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            tm[fld] = interp_face<S, Real>(s_tr + fld * STR + el2 * S::NP, ls, J, q);
    }
    if (nb >= 0) {
        const int fo = 2 * J + (s > 0 ? 0 : 1);
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            tp[fld] = has_trace<S>(fld, J)
                          ? A.trace_in[(((size_t)fo * S::NTR + fld) * ne + nb) * S::NFP1 + q]
                          : Real(0);
    } else {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) tp[fld] = tm[fld];
        tp[S::IM + J] = -tm[S::IM + J];
    }
    Real brd, brm, bE, bp;
    if (J == S::VERT) {
        load_base<S, Real>(A.bface, M.nzlev_face, iz + (s > 0 ? 1 : 0), brd, brm, bE, bp);
    } else {
        load_base<S, Real>(A.bnode, M.nzlev_node, iz * S::P1 + face_q_vert<S::D, S::P1>(J, q), brd,
                           brm, bE, bp);
    }
    Prim<S::D, S::RAIN, Real> Pm, Pp;
    make_prim<S, Real>(Pm, tm, brd, brm, bE, bp, tm[S::NF], tm[S::NF + 1], tm[S::NF + 2]);
    make_prim<S, Real>(Pp, tp, brd, brm, bE, bp, tp[S::NF], tp[S::NF + 1], tp[S::NF + 2]);
    if (S::RAIN) {
        Pm.vr = rain_velocity(Pm.rr, Pm.rm, M);
        Pp.vr = rain_velocity(Pp.rr, Pp.rm, M);
    }
    Real Fm[S::NF], Fp[S::NF];
    flux_dir<S, Real>(Pm, J, Fm);
    flux_dir<S, Real>(Pp, J, Fp);
    const Real lm = wave_speed<S, J, Real>(Pm), lpp = wave_speed<S, J, Real>(Pp);
    const Real lam = max_nonneg(lm, lpp);
    const Real hs = Real(0.5) * Real(s), hl = Real(0.5) * lam;
    Real *out = s_fh + ((el2 * S::NFACE + face) * S::NF) * S::NFP1 + q;
    // one explicit fma, as in face_flux: both schedules round identically
    Real o[S::NF];
#pragma unroll
    for (int f = 0; f < S::NF; ++f) {
        o[f] = fma(hs, add_rn(Fm[f], Fp[f]), hl * (tm[f] - tp[f]));
        out[f * S::NFP1] = o[f];
    }
    if (S::RAIN && J == S::VERT && nb < 0 && A.fallout) {
        const int nh = S::D == 3 ? M.n[0] * M.n[1] : M.n[0];
        add_fallout<S, Real>(A, s > 0, e2 % nh, q, to_f64(o[1]) + to_f64(o[2]));
    }
}

// ---------------------------------------------------------------------------
// Face pass: the Lax-Friedrichs flux of Section 3.2 once per face point
// ---------------------------------------------------------------------------
// G = {{F_J}} + Lambda/2 (U_lo - U_hi) along +e_J at one face point from the
// traces tl (element at the lower coordinate) and th (upper) and the base
// state at the point.  The sum F_lo + F_hi is an unfused add and G one
// explicit fma, so G does not depend on which side evaluates it, and the
// inline schedule's outward fluxes are +G and -G exactly.
template <class S, typename Real, int J>
__device__ __forceinline__ void lf_flux(const Real *tl, const Real *th, Real brd, Real brm, Real bE,
                                        Real bp, const MeshData &M, Real *G) {
    Prim<S::D, S::RAIN, Real> Pl, Ph;
    make_prim<S, Real>(Pl, tl, brd, brm, bE, bp, tl[S::NF], tl[S::NF + 1], tl[S::NF + 2]);
    make_prim<S, Real>(Ph, th, brd, brm, bE, bp, th[S::NF], th[S::NF + 1], th[S::NF + 2]);
    if (S::RAIN) {
        Pl.vr = rain_velocity(Pl.rr, Pl.rm, M);
        Ph.vr = rain_velocity(Ph.rr, Ph.rm, M);
    }
    Real Fl[S::NF], Fh[S::NF];
    flux_dir<S, Real>(Pl, J, Fl);
    flux_dir<S, Real>(Ph, J, Fh);
    const Real ll = wave_speed<S, J, Real>(Pl), lh = wave_speed<S, J, Real>(Ph);
    const Real lam = max_nonneg(ll, lh);
    const Real hl = Real(0.5) * lam;
#pragma unroll
    for (int fld = 0; fld < S::NF; ++fld)
        G[fld] = fma(Real(0.5), add_rn(Fl[fld], Fh[fld]), hl * (tl[fld] - th[fld]));
}

// G = {{F_j}} + Lambda/2 (U_lo - U_hi) along +e_j from the traces of the two
// elements (lo at coordinate c - 1, hi at c); a slip wall stands in for a
// missing element with the ghost state m -> m - 2 (m.n) n.  The element on
// the lo side lifts +G, the one on the hi side -G, so the two contributions
// cancel exactly in the sums of the conserved quantities.
template <class S, typename Real, int J, bool DIFF>
__device__ __forceinline__ void face_flux(const KArgs<Real> &A, int f, int q) {
    const MeshData &M = A.M;
    const int ne = M.ne;
    int im[3];
    {
        const int n0 = J == 0 ? M.nfn[0] : M.n[0], n1 = J == 1 ? M.nfn[1] : M.n[1];
        im[0] = f % n0;
        const int r = f / n0;
        im[1] = S::D == 3 ? r % n1 : r;
        im[2] = S::D == 3 ? r / n1 : 0;
    }
    const int c = im[J];
    int lo[3] = {im[0], im[1], im[2]};
    int e_lo = -1, e_hi = -1;
    if (c > 0 || M.periodic[J]) {
        lo[J] = c > 0 ? c - 1 : M.n[J] - 1;
        e_lo = lo[0] + M.n[0] * (lo[1] + M.n[1] * (S::D == 3 ? lo[2] : 0));
    }
    if (c < M.n[J]) e_hi = im[0] + M.n[0] * (im[1] + M.n[1] * (S::D == 3 ? im[2] : 0));
    Real tl[S::NTR], th[S::NTR];
    if (e_lo >= 0) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            tl[fld] = has_trace<S>(fld, J)
                          ? A.trace_in[(((size_t)(2 * J + 1) * S::NTR + fld) * ne + e_lo) * S::NFP1 + q]
                          : Real(0);
    }
    if (e_hi >= 0) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            th[fld] = has_trace<S>(fld, J)
                          ? A.trace_in[(((size_t)(2 * J) * S::NTR + fld) * ne + e_hi) * S::NFP1 + q]
                          : Real(0);
    }
    if (e_lo < 0) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) tl[fld] = th[fld];
        tl[S::IM + J] = -th[S::IM + J];
    }
    if (e_hi < 0) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) th[fld] = tl[fld];
        th[S::IM + J] = -tl[S::IM + J];
    }
    Real brd, brm, bE, bp;
    if (J == S::VERT) {
        load_base<S, Real>(A.bface, M.nzlev_face, c, brd, brm, bE, bp);
    } else {
        load_base<S, Real>(A.bnode, M.nzlev_node, im[S::VERT] * S::P1 + face_q_vert<S::D, S::P1>(J, q),
                           brd, brm, bE, bp);
    }
    // face-major: [faces normal to e_0 | e_1 | e_2][NFP fields][NFP1 points],
    // one block per face
    constexpr int NFP = DIFF ? 2 * S::NF : S::NF;
    const size_t fg = (size_t)(J > 0 ? M.nfaces[0] : 0) + (J > 1 ? M.nfaces[1] : 0) + f;
    Real *out = A.fbuf + fg * NFP * S::NFP1 + q;
    Real G[S::NF];
    lf_flux<S, Real, J>(tl, th, brd, brm, bE, bp, M, G);
    if (DIFF) {
        // interior penalty (Eq. (3.7)) on interior faces: viscous flux along +e_j
        //   V = -alpha {{du/dx_j}} + sigma k^2/h_j alpha [[u]],  [[u]] = u_lo - u_hi,
        // added to G, and S = alpha [[u]] / 2 for the symmetry term, lifted by
        // both elements with l_a'(+-1)/w_a; walls carry no diffusive flux
        Real Sx[S::NF];
#pragma unroll
        for (int fld = 0; fld < S::NF; ++fld) Sx[fld] = Real(0);
        if (e_lo >= 0 && e_hi >= 0) {
            // continuous coefficient at the face point: Q1 over the face's vertices
            const int nvt = M.nv[0] * M.nv[1] * (S::D == 3 ? M.nv[2] : 1);
            Real au = Real(0), ar = Real(0);
            int qd[3] = {0, 0, 0};
            {
                int r = q, o = 0;
#pragma unroll
                for (int i = 0; i < S::D; ++i) {
                    if (i == J) continue;
                    qd[i] = (o + 1 < S::D - 1) ? r % S::P1 : r;
                    r /= S::P1;
                    ++o;
                }
            }
#pragma unroll
            for (int c = 0; c < (1 << (S::D - 1)); ++c) {
                int v[3] = {0, 0, 0};
                Real wgt = Real(1);
                int o = 0;
#pragma unroll
                for (int i = 0; i < S::D; ++i) {
                    if (i == J) {
                        v[i] = im[J];          // the face coordinate c
                        continue;
                    }
                    const int b = (c >> o) & 1;
                    ++o;
                    v[i] = im[i] + b;
                    if (v[i] >= M.nv[i]) v[i] -= M.n[i];
                    const Real x = A.ref.xi[qd[i]];
                    wgt *= b ? Real(0.5) * (Real(1) + x) : Real(0.5) * (Real(1) - x);
                }
                const int flat = v[0] + M.nv[0] * (v[1] + M.nv[1] * v[2]);
                au = fma(wgt, A.alphaV[flat], au);
                ar = fma(wgt, A.alphaV[nvt + flat], ar);
            }
            const Real sig = mconst<Real>(M.sigma_pen[J], M.sigma_pen_f[J]);
#pragma unroll
            for (int fld = 0; fld < S::NF; ++fld) {
                const Real al = (S::RAIN && fld == 2) ? ar : au;
                const Real dl =
                    A.dtrace_in[(((size_t)(2 * J + 1) * S::NF + fld) * ne + e_lo) * S::NFP1 + q];
                const Real dh = A.dtrace_in[(((size_t)(2 * J) * S::NF + fld) * ne + e_hi) * S::NFP1 + q];
                const Real jump = tl[fld] - th[fld];
                G[fld] += al * (sig * jump - Real(0.5) * (dl + dh));
                Sx[fld] = Real(0.5) * al * jump;
            }
        }
#pragma unroll
        for (int fld = 0; fld < S::NF; ++fld) out[(S::NF + fld) * S::NFP1] = Sx[fld];
    }
    // G along +e_J: the outward flux of the element below the face; the one
    // above lifts -G (the sign sits in its lift coefficient)
#pragma unroll
    for (int fld = 0; fld < S::NF; ++fld) out[fld * S::NFP1] = G[fld];
    if (S::RAIN && J == S::VERT && (e_lo < 0 || e_hi < 0) && A.fallout) {
        // outward normal -e_z at the bottom wall, +e_z at the top
        const int nh = S::D == 3 ? M.n[0] * M.n[1] : M.n[0];
        const double gw = to_f64(G[1]) + to_f64(G[2]);
        add_fallout<S, Real>(A, e_lo >= 0, f - c * nh, q, e_lo < 0 ? -gw : gw);
    }
}

constexpr int kFaceThreads = 128;

template <class S, typename Real, bool DIFF>
__global__ void __launch_bounds__(kFaceThreads) k_face(KArgs<Real> A) {
    int b = blockIdx.x, J = 0;
    if (b >= A.M.fblk[0]) {
        b -= A.M.fblk[0];
        J = 1;
        if (S::D == 3 && b >= A.M.fblk[1]) {
            b -= A.M.fblk[1];
            J = 2;
        }
    }
    const long long gid = (long long)b * kFaceThreads + threadIdx.x;
    const int f = (int)(gid / S::NFP1), q = (int)(gid - (long long)f * S::NFP1);
    if (f >= A.M.nfaces[J]) return;
    switch (J) {
        case 0: face_flux<S, Real, 0, DIFF>(A, f, q); break;
        case 1: face_flux<S, Real, 1, DIFF>(A, f, q); break;
        default: face_flux<S, Real, (S::D == 3 ? 2 : 1), DIFF>(A, f, q); break;
    }
}

// One tile of EPB consecutive elements (tile index bidx) of the stage
// kernel; every thread of the CTA takes part (the body has barriers).
// PF: the face fluxes come from the face pass (k_face) instead of being
// evaluated here on both sides of every face.
template <class S, typename Real, int MODE, bool PF = false, bool DIFF = false>
__device__ __forceinline__ void stage_block(const KArgs<Real> &A, const RefData<Real> &ref, int bidx,
                                            unsigned char *smem_raw) {
    static_assert(!DIFF || PF, "artificial diffusion runs with the face pass");
    constexpr int STR = S::EPB * S::NP;
    constexpr bool SHARE = tr_shares_fl<S, Real, PF, DIFF>();
    constexpr int NFP = DIFF ? 2 * S::NF : S::NF;             // per face: fluxes [, symmetry terms]
    constexpr int EB = S::NFACE * NFP * S::NFP1;              // face values of one element
    // float64 form with float-float contractions: nodal fluxes, coefficient
    // tables and face fluxes held as float32 pairs in the float64 slots, the
    // tendencies accumulated as pairs (Rs, Re) through the volume term and the
    // lift, then formed in float64 for the stage update
    constexpr bool FFC = S::FF && sizeof(Real) == sizeof(double) && !DIFF;
    Real *s_fl = reinterpret_cast<Real *>(smem_raw);          // nodal fluxes (fl_index)
    Real *s_tr = SHARE ? s_fl : s_fl + S::D * fl_words<S, Real>() * STR;   // [NTR][STR]
    Real *s_fh = reinterpret_cast<Real *>(smem_raw + stage_fh_offset<S, Real, PF, DIFF>());  // [EPB][EB]
    int *s_info = reinterpret_cast<int *>(s_fh + S::EPB * EB);                            // [EPB][16]
    Real *s_al = reinterpret_cast<Real *>(s_info + 16 * S::EPB);        // DIFF: [EPB][2][NCORNER]
    Real *s_red = s_al + S::EPB * 2 * S::NCORNER;                       // DIFF: [EPB][2]
    Real *s_cf = reinterpret_cast<Real *>(smem_raw + stage_cf_offset<S, Real, PF, DIFF>());
    const MeshData &M = A.M;
    const int ne = M.ne;
    const size_t nodes = (size_t)ne * S::NP;
    const int t = threadIdx.x;
    const int el = t / S::NP, a = t - el * S::NP;
    const int e = bidx * S::EPB + el;
    const bool valid = (t < STR) && (e < ne);

    // the node's state and derived fields: loads issued first, so that their
    // latency overlaps the set-up below
    Real u[S::NF], R[S::NF], dT = Real(0), drv = Real(0), dpp = Real(0), dgm = Real(0), dvr = Real(0);
    if (valid) {
        const size_t gi = (size_t)e * S::NP + a;
#pragma unroll
        for (int f = 0; f < S::NF; ++f) u[f] = A.Uin[f * nodes + gi];
        dT = A.derived[gi];
        drv = A.derived[nodes + gi];
        dpp = A.derived[2 * nodes + gi];
        if (S::RAIN) {
            dgm = A.derived[3 * nodes + gi];
            dvr = A.derived[4 * nodes + gi];
        }
    }

    // face pass: copy the tile's face values to shared memory while the
    // nodal phases run (one contiguous block per face)
    if (PF) cp_async_faces<S, Real, NFP>(A.fbuf, A.ftab, s_fh, bidx, min(S::EPB, ne - bidx * S::EPB));

    if constexpr (FFC)
        coef_fill_ff<S>(A.ref, reinterpret_cast<float2 *>(s_cf));
    else if (sizeof(Real) == sizeof(double))
        coef_fill<S, Real>(A.ref, s_cf);

    // per element: neighbours across the 2D faces (inline faces) and the
    // vertical index
    if (t < S::EPB) {
        const int e0 = bidx * S::EPB + t;
        if (e0 < ne) {
            int im[3];
            elem_multi(M, e0, im[0], im[1], im[2]);
            if (!PF) {
#pragma unroll
                for (int j = 0; j < S::D; ++j) {
                    s_info[t * 16 + 2 * j] = neighbour_of<S::D>(M, im, j, -1);
                    s_info[t * 16 + 2 * j + 1] = neighbour_of<S::D>(M, im, j, 1);
                }
            }
            s_info[t * 16 + 6] = im[S::VERT];
            if (DIFF) alpha_corners<S, Real>(A, im, s_al + t * 2 * S::NCORNER);
        }
        if (DIFF) {
            s_red[2 * t] = Real(0);
            s_red[2 * t + 1] = Real(0);
        }
    }
    __syncthreads();

    // ---- phase 1: nodal fluxes, sources, node values for own traces
    if (valid) {
        const Real T = dT, rv = drv, pp = dpp;
        const int lev = s_info[el * 16 + 6] * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        Real brd, brm, bE, bp;
        load_base<S, Real>(A.bnode, M.nzlev_node, lev, brd, brm, bE, bp);
        Prim<S::D, S::RAIN, Real> P;
        make_prim<S, Real>(P, u, brd, brm, bE, bp, T, rv, pp);
        if (S::RAIN) P.vr = dvr;
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            Real F[S::NF];
            flux_dir<S, Real>(P, j, F);
            if constexpr (FFC) {
                // (hi, hi, lo, lo) of the field pairs (2p, 2p + 1), the last
                // padded with zeros when n_f is odd
                constexpr int NPR = (S::NF + 1) / 2;
                float4 *fl4 = reinterpret_cast<float4 *>(s_fl);
#pragma unroll
                for (int p = 0; p < NPR; ++p) {
                    const float2 v0 = ff_split(to_f64(F[2 * p]));
                    const float2 v1 =
                        2 * p + 1 < S::NF ? ff_split(to_f64(F[2 * p + 1])) : make_float2(0.0f, 0.0f);
                    fl4[(j * NPR + p) * STR + t] = make_float4(v0.x, v1.x, v0.y, v1.y);
                }
            } else {
                fl_store<S, Real, STR>(s_fl, j, t, F);
            }
        }
#pragma unroll
        for (int f = 0; f < S::NF; ++f) R[f] = Real(0);
        // node values for the own traces (the float64 form reads them back
        // from the trace buffer) or for the derivatives of the diffusion
        if (DIFF) {
#pragma unroll
            for (int f = 0; f < S::NF; ++f) s_tr[f * STR + t] = u[f];
        } else if (!PF && sizeof(Real) == sizeof(float)) {
#pragma unroll
            for (int f = 0; f < S::NF; ++f) s_tr[f * STR + t] = u[f];
            s_tr[S::NF * STR + t] = T;
            s_tr[(S::NF + 1) * STR + t] = rv;
            s_tr[(S::NF + 2) * STR + t] = pp;
        }
        // sources G (Eq. (2.11)): microphysics and gravity
        if (S::RAIN) {
            R[1] = dgm;
            R[2] = -dgm;
        }
        const Real g = mconst<Real>(M.g, M.g_f);
        R[S::IM + S::VERT] = -g * (u[0] + u[1] + (S::RAIN ? u[2] : Real(0)));
        R[S::IE] = -g * u[S::IM + S::VERT];
    }
    __syncthreads();

    // ---- phase 1b (diffusion): F_j -= alpha du/dx_j at the node, so that the
    // volume term below also carries (alpha grad u, grad phi_a) of Eq. (3.7)
    if (DIFF) {
        if (valid) {
            Real xi[3];
#pragma unroll
            for (int j = 0; j < S::D; ++j) xi[j] = ref.xi[digit<S::D, S::P1>(a, j)];
            const Real *cv = s_al + el * 2 * S::NCORNER;
            const Real au = q1_interp<S, Real>(cv, xi), ar = q1_interp<S, Real>(cv + S::NCORNER, xi);
#pragma unroll
            for (int j = 0; j < S::D; ++j) {
                const int aj = digit<S::D, S::P1>(a, j);
                const int st = stride_of<S::P1>(j);
                const int b0 = el * S::NP + a - aj * st;
                const Real sc = mconst<Real>(M.two_over_h[j], M.two_over_h_f[j]);
#pragma unroll
                for (int f = 0; f < S::NF; ++f) {
                    const Real *v = s_tr + f * STR + b0;
                    Real du = Real(0);
#pragma unroll
                    for (int i = 0; i < S::P1; ++i) du = fma(ref.dmat[aj][i], v[i * st], du);
                    const Real al = (S::RAIN && f == 2) ? ar : au;
                    s_fl[fl_index<S, Real, STR>(j, f, t)] -= al * (sc * du);
                }
            }
        }
        __syncthreads();
    }

    // ---- phase 2a: volume term, sum factorised: R_a += (2/h_j) sum_i dhat[a_j][i] F_j(i)
    constexpr int NPR = (S::NF + 1) / 2;
    float2 Rs[NPR], Re[NPR];     // FFC: the tendencies of the field pairs (2p, 2p + 1)
    if constexpr (FFC) {
        if (valid) {
#pragma unroll
            for (int p = 0; p < NPR; ++p) {
                const float2 r0 = ff_split(to_f64(R[2 * p]));
                const float2 r1 =
                    2 * p + 1 < S::NF ? ff_split(to_f64(R[2 * p + 1])) : make_float2(0.0f, 0.0f);
                Rs[p] = make_float2(r0.x, r1.x);
                Re[p] = make_float2(r0.y, r1.y);
            }
            volume_term_ff<S, STR>(reinterpret_cast<const float4 *>(s_fl),
                                   reinterpret_cast<const float2 *>(s_cf), el, a, Rs, Re);
        }
    } else {
        if (valid) volume_term<S, Real, STR>(A, s_fl, s_cf, el, a, R);
    }

    // ---- phase 2b: Lax-Friedrichs flux at every face point of the CTA's elements
    if (PF) {
        // outward fluxes of the face pass, copied asynchronously since the start
        cp_async_wait_all();
    } else {
        // face points in direction-major order (direction, element, side,
        // point): the lanes of a warp mostly share the direction, so each
        // direction-specialised face_point body runs with full warps
        constexpr int PER_J = S::EPB * 2 * S::NFP1;
        for (int item = t; item < S::EPB * S::NFACE * S::NFP1; item += S::NT) {
            const int jd = item / PER_J;
            const int r = item - jd * PER_J;
            const int el2 = r / (2 * S::NFP1);
            const int r2 = r - el2 * (2 * S::NFP1);
            const int face = 2 * jd + r2 / S::NFP1;
            const int q = r2 - (face & 1) * S::NFP1;
            const int e2 = bidx * S::EPB + el2;
            if (e2 >= ne) continue;
            const int nb = s_info[el2 * 16 + face], iz2 = s_info[el2 * 16 + 6];
            switch (face >> 1) {
                case 0: face_point<S, Real, 0>(A, ref, s_tr, s_fh, el2, face, q, e2, nb, iz2); break;
                case 1: face_point<S, Real, 1>(A, ref, s_tr, s_fh, el2, face, q, e2, nb, iz2); break;
                default:
                    face_point<S, Real, (S::D == 3 ? 2 : 1)>(A, ref, s_tr, s_fh, el2, face, q, e2, nb,
                                                             iz2);
                    break;
            }
        }
    }
    __syncthreads();
    if constexpr (FFC) {
        // the tile's face fluxes as float32 pairs, in place (each thread
        // rewrites the slots it reads)
        const int nv = min(S::EPB, ne - bidx * S::EPB) * EB;
        float2 *fh2 = reinterpret_cast<float2 *>(s_fh);
        for (int i = t; i < nv; i += S::NT) fh2[i] = ff_split(to_f64(s_fh[i]));
        __syncthreads();
    }

    // ---- phase 3: lift the face fluxes, R_a -= (2/h_j) l_a(s)/w_a Fhat(j, s)
    if (valid) {
        if constexpr (FFC) {
            lift_ff<S, PF>(reinterpret_cast<const float2 *>(s_fh), reinterpret_cast<const float2 *>(s_cf),
                           el, a, Rs, Re);
#pragma unroll
            for (int f = 0; f < S::NF; ++f)
                R[f] = (f & 1) ? ff_value(Rs[f >> 1].y, Re[f >> 1].y) : ff_value(Rs[f >> 1].x, Re[f >> 1].x);
        }
#pragma unroll
        for (int j = 0; j < (FFC ? 0 : S::D); ++j) {
            const int aj = digit<S::D, S::P1>(a, j);
            const int q = face_q<S::D, S::P1>(a, j);
            const Real *fm = s_fh + ((el * S::NFACE + 2 * j) * NFP) * S::NFP1 + q;
            const Real *fp = s_fh + ((el * S::NFACE + 2 * j + 1) * NFP) * S::NFP1 + q;
            const Real *cf = s_cf + j * Coef<S>::BLK;
            Real cm, cp;
            if constexpr (sizeof(Real) == sizeof(double)) {
                cm = cf[Coef<S>::LM + aj];
                cp = cf[Coef<S>::LP + aj];
            } else {
                cm = A.ref.liftm_s[j][aj];
                cp = A.ref.liftp_s[j][aj];
            }
            // the low face holds the outward flux (inline) or G along +e_j,
            // which is minus this element's outward flux (face pass):
            // fma(-c, -G, r) = fma(c, G, r) exactly, so both schedules round
            // alike.  Two fmas per face and field (a sum of the two products
            // first would cost a multiply and an add more).
            const Real cmo = PF ? cm : -cm;
#pragma unroll
            for (int f = 0; f < S::NF; ++f)
                R[f] = fma(cmo, fm[f * S::NFP1], fma(-cp, fp[f * S::NFP1], R[f]));
            if (DIFF) {
                // symmetry term of Eq. (3.7): + (2/h_j)^2 l_a'(s)/w_a S on both faces
                const Real *sm = fm + S::NF * S::NFP1;
                const Real *sp = fp + S::NF * S::NFP1;
                Real dm, dp;
                if constexpr (sizeof(Real) == sizeof(double)) {
                    dm = cf[Coef<S>::DLM + aj];
                    dp = cf[Coef<S>::DLP + aj];
                } else {
                    dm = A.ref.dliftm_s[j][aj];
                    dp = A.ref.dliftp_s[j][aj];
                }
#pragma unroll
                for (int f = 0; f < S::NF; ++f)
                    R[f] = fma(dm, sm[f * S::NFP1], fma(dp, sp[f * S::NFP1], R[f]));
            }
        }
        const size_t gi = (size_t)e * S::NP + a;
        if (MODE == MODE_RHS) {
#pragma unroll
            for (int f = 0; f < S::NF; ++f) A.Uout[f * nodes + gi] = R[f];
        } else {
            Real un[S::NF];
#pragma unroll
            for (int f = 0; f < S::NF; ++f) {
                // one explicit fma: every stage kernel rounds the update alike;
                // beta u is u itself when beta = 1 (three stages in four)
                Real v = fma(A.gdt, R[f], is_one(A.beta) ? u[f] : A.beta * u[f]);
                if (nonzero(A.alpha)) v = fma(A.alpha, A.Un[f * nodes + gi], v);
                un[f] = v;
            }
            if (A.sponge) {
                // Eq. (3.8) at the end of the step: relax rho_m', rho_r', m, E'
                // towards 0 and add the moisture removed to rho_d' (Section 3.6)
                const Real dl = A.sponge[s_info[el * 16 + 6] * S::P1 + digit<S::D, S::P1>(a, S::VERT)];
                if (dl != Real(0)) {
                    const Real om = Real(1) - dl;
                    Real removed = dl * un[1];
                    if (S::RAIN) removed = add_rn(removed, dl * un[2]);
                    un[0] = un[0] + removed;
#pragma unroll
                    for (int f = 1; f < S::NF; ++f) un[f] = om * un[f];
                }
            }
#pragma unroll
            for (int f = 0; f < S::NF; ++f) A.Uout[f * nodes + gi] = un[f];
            split_and_store<S, Real, DIFF>(A, un, e, a, s_info[el * 16 + 6], s_tr, t, s_red, dT);
        }
    }
    if (MODE == MODE_STAGE) {
        __syncthreads();
        if (DIFF) alpha_store<S, Real>(A, s_red, bidx);
        write_traces<S, Real, DIFF>(A, ref, s_tr, A.trace_out, bidx);
    }
}

template <class S, typename Real, int MODE, bool PF, bool DIFF>
__global__ void __launch_bounds__(S::NT) k_stage(KArgs<Real> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stage_block<S, Real, MODE, PF, DIFF>(A, A.ref, blockIdx.x + A.tile0, smem_raw);
}

// The float32 face-pass tile (64, 128 or 256 threads) with its register
// budget sized for 1280 threads per SM in 3-D (48 registers) and 1536 in
// 2-D (40 registers; measured: the 256-member 2-D ensemble 18.8 -> 18.1 ms
// per step, while 3-D tiles run 2 % slower at 40 registers)
template <class S>
constexpr int f32pf_min_blocks() {
    return (S::D == 3 ? 1280 : 1536) / S::NT;
}

template <class S, int MODE>
__global__ void __launch_bounds__(S::NT, f32pf_min_blocks<S>()) k_stage_f32pf(KArgs<float> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    stage_block<S, float, MODE, true, false>(A, A.ref, blockIdx.x + A.tile0, smem_raw);
}

// ---------------------------------------------------------------------------
// k_split: derived fields only (float64 outputs)
// ---------------------------------------------------------------------------
template <class S, typename Real>
__global__ void k_split(KArgs<Real> A, double *oT, double *orv, double *orc, double *opp) {
    const size_t nodes = (size_t)A.M.ne * S::NP;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < nodes;
         gi += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(gi / S::NP), a = (int)(gi - (size_t)e * S::NP);
        const int lev = vert_index<S::D>(A.M, e) * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        const int nl = A.M.nzlev_node;
        Real u[S::NF];
#pragma unroll
        for (int f = 0; f < S::NF; ++f) u[f] = A.Uin[f * nodes + gi];
        const NodeDerived nd = derive_node<S>(u, A, lev);
        const double rm = A.bnode_d[nl + lev] + (double)u[1];
        if (!nd.conv) atomicAdd(&A.flags[0], 1ull);
        if (!nd.phys) atomicAdd(&A.flags[1], 1ull);
        if (oT) oT[gi] = nd.T;
        if (orv) orv[gi] = nd.rv;
        // the perturbation form decides saturation in float32: rho_c is 0
        // exactly where it found the node unsaturated
        if (orc) orc[gi] = (A.M.pert_split && !(nd.rcf > 0.0f)) ? 0.0 : rm - nd.rv;
        if (opp) opp[gi] = nd.pp;
    }
}

// ---------------------------------------------------------------------------
// k_init_bubble: warm bubble at fixed pressure and mixing ratio
// ---------------------------------------------------------------------------
struct BubbleArgs {
    double theta, qt0, H, amplitude;
    double centre[3], radius[3];
    const double *noise;  // device, [e][a] or NULL
};

template <class S, typename Real>
__global__ void k_init_bubble(KArgs<Real> A, BubbleArgs B) {
    const size_t nodes = (size_t)A.M.ne * S::NP;
    const double kappa = kRd / kCpd;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < nodes;
         gi += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(gi / S::NP), a = (int)(gi - (size_t)e * S::NP);
        int im[3];
        elem_multi(A.M, e, im[0], im[1], im[2]);
        double x[3] = {0.0, 0.0, 0.0};
        double r2 = 0.0;
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            const int aj = digit<S::D, S::P1>(a, j);
            x[j] = im[j] * A.M.h[j] + (1.0 + (double)A.ref.xi[aj]) * A.M.h[j] * 0.5;
            const double d = (x[j] - B.centre[j]) / B.radius[j];
            r2 += d * d;
        }
        const double Lb = fmin(sqrt(r2), 1.0);
        const double cb = cos(0.5 * M_PI * Lb);
        const double thp = B.amplitude * cb * cb;
        const int nl = A.M.nzlev_node;
        const int lev = im[S::VERT] * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        const double pbar = A.bnode_d[3 * nl + lev];
        const double ex = pow(pbar / kPref, kappa);
        double T = (B.theta + thp) * ex;
        if (B.noise) T += B.noise[gi];
        const double qt = B.qt0 * (1.0 - x[S::VERT] / B.H);
        // p = (rho_d R_d + rho_v R_v) T with rho_v = min(rho_vs(T), qt rho_d)
        const double rvs = rho_vs(T, 1.0 / T);
        double rd = pbar / (T * (kRd + qt * kRv));
        double rv = qt * rd;
        if (qt * rd > rvs) {
            rd = (pbar - rvs * kRv * T) / (kRd * T);
            rv = rvs;
        }
        const double rm = qt * rd;
        const double E = (kCvd * rd + kCvv * rv + kCl * (rm - rv)) * (T - kTref) + rv * kLprime;
        A.Uout[gi] = (Real)(rd - A.bnode_d[lev]);
        A.Uout[nodes + gi] = (Real)(rm - A.bnode_d[nl + lev]);
        for (int f = 2; f < S::NF; ++f) A.Uout[f * nodes + gi] = Real(0);
        A.Uout[S::IE * nodes + gi] = (Real)(E - A.bnode_d[2 * nl + lev]);
    }
}

// ---------------------------------------------------------------------------
// Reductions (deterministic: fixed per-block tree, then one block in order)
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kNRed = 9;

template <class S, typename Real>
__global__ void __launch_bounds__(kRedThreads) k_reduce_partial(KArgs<Real> A, double *partials) {
    __shared__ double sh[kNRed][kRedThreads];
    const size_t nodes = (size_t)A.M.ne * S::NP;
    double acc[kNRed];
#pragma unroll
    for (int r = 0; r < kNRed; ++r) acc[r] = 0.0;
    acc[5] = 0.0;
    acc[6] = -INFINITY;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < nodes;
         gi += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(gi / S::NP), a = (int)(gi - (size_t)e * S::NP);
        double W = A.M.jac;
#pragma unroll
        for (int j = 0; j < S::D; ++j) W *= (double)A.ref.w[digit<S::D, S::P1>(a, j)];
        const int nl = A.M.nzlev_node;
        const int lev = vert_index<S::D>(A.M, e) * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        const double urd = (double)A.Uin[gi], urm = (double)A.Uin[nodes + gi];
        const double urr = S::RAIN ? (double)A.Uin[2 * nodes + gi] : 0.0;
        const double rd = A.bnode_d[lev] + urd, rm = A.bnode_d[nl + lev] + urm, rr = urr;
        // the split's float64 T, rho_v, p' (the float32 forms store their
        // derived fields in float32, whose rounding of T alone moves rho_vs(T)
        // by ~2e-6 relative: too coarse for the supersaturation diagnostic)
        Real u[S::NF];
#pragma unroll
        for (int f = 0; f < S::NF; ++f) u[f] = A.Uin[f * nodes + gi];
        const NodeDerived nd = derive_node<S>(u, A, lev);
        const double T = nd.T, rv = nd.rv, pp = nd.pp;
        const double rho = rd + rm + rr;
        double msq = 0.0;
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            const double m = (double)A.Uin[(S::IM + j) * nodes + gi];
            msq += m * m;
        }
        acc[0] += W * urd;
        acc[1] += W * (urm + urr);
        acc[2] += W * (double)A.Uin[S::IM * nodes + gi];
        acc[3] += W * (rm - rv);
        acc[4] += W * urr;
        const double p = A.bnode_d[3 * nl + lev] + pp;
        const double rc = rm - rv;
        const double cv = kCvd * rd + kCvv * rv + kCl * (rc + rr);
        const double cm = sqrt((cv + kRd * rd + kRv * rv) / cv * p / rho);
        const double vr = S::RAIN ? rain_velocity(rr, rm, A.M) : 0.0;
        acc[5] = fmax(acc[5], sqrt(msq) / rho + fabs(vr) + cm);
        const double rvs = rho_vs(T, 1.0 / T);
        acc[6] = fmax(acc[6], (rv - rvs) / rvs);
        acc[7] += W * (double)A.Uin[S::IE * nodes + gi];
    }
    // fall-out: sum over the wall face points of Wf_q J_F x the accumulated
    // outward water flux, J_F = |K| / 2^d x 2 / h_z
    if (S::RAIN && A.fallout) {
        const int nh = S::D == 3 ? A.M.n[0] * A.M.n[1] : A.M.n[0];
        const size_t npt = (size_t)2 * nh * S::NFP1;
        const double jf = A.M.jac * A.M.two_over_h[S::VERT];
        for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npt;
             p += (size_t)gridDim.x * blockDim.x) {
            const int q = (int)(p % S::NFP1);
            double wq = jf * (double)A.ref.w[q % S::P1];
            if (S::D == 3) wq *= (double)A.ref.w[q / S::P1];
            acc[8] += wq * A.fallout[p];
        }
    }
#pragma unroll
    for (int r = 0; r < kNRed; ++r) sh[r][threadIdx.x] = acc[r];
    __syncthreads();
    for (int off = kRedThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
#pragma unroll
            for (int r = 0; r < kNRed; ++r) {
                const double o = sh[r][threadIdx.x + off];
                sh[r][threadIdx.x] = (r == 5 || r == 6) ? fmax(sh[r][threadIdx.x], o)
                                                        : sh[r][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < kNRed; ++r) partials[(size_t)blockIdx.x * kNRed + r] = sh[r][0];
    }
}

// Taylor-table entries of rho_vs (dg_math.cuh): at T_i = 150 K + i/128 K,
// c_0 = rho_vs(T_i) from the float64 closed form; phi = (a-1) ln T - b/T has
// the Taylor coefficients p_k = (-1)^(k+1) ((a-1)/(k T_i^k) + b/T_i^(k+1)),
// and exp gives c_n = (1/n) sum_{k=1..n} k p_k c_{n-k}.
static __global__ void k_fill_rvs_table(double *tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kTabN) {
        const double T = kTabT0 + (double)i / kTabInvStep;
        const double it = 1.0 / T;
        double p[6], c[6];
        double itk = 1.0, sgn = 1.0;
        for (int k = 1; k <= 5; ++k) {
            itk *= it;
            p[k] = sgn * ((kEsA - 1.0) * itk / k + kEsB * itk * it);
            sgn = -sgn;
        }
        c[0] = rho_vs(T, it);
        for (int n = 1; n <= 5; ++n) {
            double acc = 0.0;
            for (int k = 1; k <= n; ++k) acc += k * p[k] * c[n - k];
            c[n] = acc / n;
        }
        double *e = tab + (size_t)kTabStride * i;
        for (int n = 0; n < 6; ++n) e[n] = c[n];
        e[6] = 2.0 * c[2];
        e[7] = 3.0 * c[3];
    }
}

}  // namespace dgm
