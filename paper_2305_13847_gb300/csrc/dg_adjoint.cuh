// Adjoint (vector-Jacobian product) of the DG right-hand side, float64.
//
// For a state U and an adjoint vector w (both in the ABI layout) the kernels
// compute ubar = (dR/dU)^T w, R the right-hand side of Eq. (3.2)/(3.3):
//   k_adj_local   per element: transposed volume contraction, the nodal
//                 flux and source Jacobians, the Lax-Friedrichs face-flux
//                 Jacobians on both sides of every face point, and the
//                 transposed interpolation of the own-side trace adjoints;
//                 the neighbour-side trace adjoints go to a buffer;
//   k_adj_gather  per node: gathers the neighbours' contributions to its
//                 traces, then the split Eq. (2.8) is differentiated by the
//                 implicit-function theorem on the active branch, giving
//                 the adjoint of U; out = alpha out + beta w + gamma ubar.
// The pointwise Jacobians (flux, wave-speed bound, sources, v_r) are taken
// in forward mode with dual numbers through the same templated code the
// forward kernels run, so the adjoint linearises exactly the computed
// operator.  Non-smooth points take the active branch: max in Lambda, the
// saturation min in the split, max(rho_c, 0) and max(rho_r, 0); fractional
// powers of rain below kRainFloorLin are differentiated at the floor.
#pragma once

#include "dg_device.cuh"

namespace dgm {

// ---------------------------------------------------------------------------
// Dual numbers (value, derivative) for forward-mode differentiation
// ---------------------------------------------------------------------------
struct Dual {
    double v, d;
    __device__ __forceinline__ Dual() : v(0.0), d(0.0) {}
    __device__ __forceinline__ Dual(double x) : v(x), d(0.0) {}
    __device__ __forceinline__ Dual(double x, double y) : v(x), d(y) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { return a = a + b; }
__device__ __forceinline__ Dual &operator-=(Dual &a, Dual b) { return a = a - b; }
__device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ __forceinline__ bool operator!=(Dual a, Dual b) { return a.v != b.v; }
__device__ __forceinline__ Dual fma(Dual a, Dual b, Dual c) {
    return Dual(::fma(a.v, b.v, c.v), a.d * b.v + a.v * b.d + c.d);
}

// v_r(rho_r, rho_m) and its partial derivatives (the fractional power of
// rho_r differentiated at max(rho_r, floor), kRainFloorLin: the powers p < 1
// of the warm-rain closure have unbounded derivatives as rho_r -> 0+, and the
// rain that the DG discretisation leaks into cloud-free elements would
// otherwise dominate the linearisation)
struct RainVel {
    double v, d_rm, d_rr;
};
__device__ __forceinline__ RainVel rain_velocity_partials(double rr, double rm, const MeshData &M) {
    RainVel o = {0.0, 0.0, 0.0};
    const bool lit = !gt0(M.rho_w);
    const double rw = lit ? rm + rr : M.rho_w;
    if (!gt0(rr) || !gt0(rw)) return o;
    // y = rho_r^(1/8) = x^2 with x = rho_r^(1/16) = rho_r q^15, q = rho_r^(-1/16);
    // dy/drho_r = y / (8 rho_r), taken at max(rho_r, floor)
    const double q = inv_root16(rr);
    const double q2 = q * q, q4 = q2 * q2, q8 = q4 * q4;
    const double x = rr * (q8 * q4 * q2 * q);
    const double y = x * x;
    const double dy = rr > M.rain_floor ? 0.125 * y * recip(rr) : M.rain_d8;
    const double z = inv_root8(rw);                       // rho_w^(-1/8)
    const double dz = lit ? -0.125 * z * recip(rw) : 0.0; // d z / d rho_w, rho_w = rho_m + rho_r
    o.v = M.kvr * y * z;
    o.d_rr = M.kvr * (dy * z + y * dz);
    o.d_rm = M.kvr * (y * dz);
    return o;
}
// ---------------------------------------------------------------------------
struct AdjArgs {
    MeshData M;
    RefData<double> ref;
    const double *U;        // state (ABI layout)
    const double *derived;  // T, rho_v, p' (, G, v_r) of U
    const double *trace;    // traces of U, [2D][NTR][ne][NFP1]
    const double *bnode, *bface;  // base tables
    const double *rvs_tab;  // rho_vs Taylor table (dg_math.cuh)
    const double *w;        // adjoint input (ABI layout)
    double *ubar_part;      // [NTR][nodes]: adjoints of U (NF) and of T, rho_v, p'
    double *tadj;           // [2D][NTR][ne][NFP1]: neighbour trace adjoints
    double *out;            // [NF][nodes]
    double alpha, beta, gamma;
};

// Reverse-mode derivatives of the pointwise flux, by hand: the adjoints of
// the primitive quantities of make_prim accumulate in PrimBar (flux_dir_vjp,
// wave_speed_vjp) and prim_to_inputs carries them back to the inputs
// x = (U', T, rho_v, p').  One reverse sweep replaces one forward
// dual-number pass per input.
template <int D>
struct PrimBar {
    double rd, rm, rr, rho, E, p, T, rv, vr;
    double m[D], u[D];
};

template <int D>
__device__ __forceinline__ void zero_bar(PrimBar<D> &B) {
    B.rd = B.rm = B.rr = B.rho = B.E = B.p = B.T = B.rv = B.vr = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) B.m[i] = B.u[i] = 0.0;
}

// B += W where c holds (a select per quantity, no branch)
template <int D>
__device__ __forceinline__ void add_bar_if(PrimBar<D> &B, const PrimBar<D> &W, bool c) {
    B.rd += c ? W.rd : 0.0;
    B.rm += c ? W.rm : 0.0;
    B.rr += c ? W.rr : 0.0;
    B.rho += c ? W.rho : 0.0;
    B.E += c ? W.E : 0.0;
    B.p += c ? W.p : 0.0;
    B.T += c ? W.T : 0.0;
    B.rv += c ? W.rv : 0.0;
    B.vr += c ? W.vr : 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        B.m[i] += c ? W.m[i] : 0.0;
        B.u[i] += c ? W.u[i] : 0.0;
    }
}

// sign, with the derivative of |x| taken as 0 at exactly 0 (the velocity is
// exactly 0 in a resting initial state; central differences see 0 there)
__device__ __forceinline__ double sgn0(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// Fb . dF_j/dP for the flux of flux_dir (same formulas):
//   F_j = rho_d u_j, rho_m u_j, rho_r (u_j - v_r d_jz), m_i u_j - rho_r v_r u_i d_jz + p' d_ij,
//         (E + p) u_j - (c_l (T - T_ref) + |u|^2/2) rho_r v_r d_jz
template <class S>
__device__ __forceinline__ void flux_dir_vjp(const Prim<S::D, S::RAIN, double> &P, int j,
                                             const double *Fb, PrimBar<S::D> &B) {
    const bool vert = (j == S::VERT);
    const double uj = P.u[j];
    double ubj = Fb[0] * P.rd + Fb[1] * P.rm + Fb[S::IE] * (P.E + P.p);
    B.rd += Fb[0] * uj;
    B.rm += Fb[1] * uj;
    if (S::RAIN) {
        ubj += Fb[2] * P.rr;
        B.rr += Fb[2] * uj;
    }
#pragma unroll
    for (int i = 0; i < S::D; ++i) {
        ubj += Fb[S::IM + i] * P.m[i];
        B.m[i] += Fb[S::IM + i] * uj;
    }
    B.p += Fb[S::IM + j] + Fb[S::IE] * uj;     // p' d_ij and (E + p) u_j (p = p_bar + p')
    B.E += Fb[S::IE] * uj;
    if (S::RAIN && vert) {
        const double rvr = P.rr * P.vr;
        double ke = 0.0;
#pragma unroll
        for (int i = 0; i < S::D; ++i) ke += P.u[i] * P.u[i];
        double rvrb = -Fb[2] - Fb[S::IE] * (kCl * (P.T - kTref) + 0.5 * ke);
#pragma unroll
        for (int i = 0; i < S::D; ++i) {
            rvrb -= Fb[S::IM + i] * P.u[i];
            B.u[i] -= (Fb[S::IM + i] + Fb[S::IE] * P.u[i]) * rvr;
        }
        B.T -= Fb[S::IE] * kCl * rvr;
        B.rr += rvrb * P.vr;
        B.vr += rvrb * P.rr;
    }
    B.u[j] += ubj;
}

// lb . dLambda_side/dP for wave_speed: |u_J| + c_m (+ |v_r| on faces normal
// to e_z), c_m = sqrt(num / (c_v rho)), num = (c_v + R) p, so that
// dc = c/2 (d(c_v + R)/(c_v + R) + dp/p - dc_v/c_v - drho/rho)
template <class S, int J>
__device__ __forceinline__ void wave_speed_vjp(const Prim<S::D, S::RAIN, double> &P, double lb,
                                               PrimBar<S::D> &B) {
    B.u[J] += lb * sgn0(P.u[J]);
    if (S::RAIN && J == S::VERT) B.vr += lb * sgn0(P.vr);
    const double cv = kCvd * P.rd + kCvv * P.rv + kCl * (P.rm - P.rv + P.rr);
    const double R = kRd * P.rd + kRv * P.rv;
    const double num = (cv + R) * P.p;
    const double nd = num * (cv * P.rho);
    if (!(nd > 0.0)) return;
    const double h = 0.5 * lb * num * rsqrt_nr(nd);       // c/2 times lb
    const double a = h / (cv + R);
    const double cvb = a - h / cv;
    B.p += h / P.p;
    B.rho -= h / P.rho;
    B.rd += cvb * kCvd + a * kRd;
    B.rv += cvb * (kCvv - kCl) + a * kRv;
    B.rm += cvb * kCl;
    if (S::RAIN) B.rr += cvb * kCl;
}

// back through make_prim (rho_d = rho_d_bar + x_0, ..., u = m / rho,
// p = p_bar + p') and v_r(rho_r, rho_m) to the inputs x
template <class S>
__device__ __forceinline__ void prim_to_inputs(const Prim<S::D, S::RAIN, double> &P, PrimBar<S::D> &B,
                                               const RainVel &rvel, double *xb) {
    if (S::RAIN) {
        B.rr += B.vr * rvel.d_rr;
        B.rm += B.vr * rvel.d_rm;
    }
    double irb = 0.0;
#pragma unroll
    for (int i = 0; i < S::D; ++i) {
        B.m[i] += B.u[i] * P.irho;
        irb += B.u[i] * P.m[i];
    }
    B.rho -= irb * P.irho * P.irho;
    xb[0] += B.rd + B.rho;
    xb[1] += B.rm + B.rho;
    if (S::RAIN) xb[2] += B.rr + B.rho;
#pragma unroll
    for (int i = 0; i < S::D; ++i) xb[S::IM + i] += B.m[i];
    xb[S::IE] += B.E;
    xb[S::NF] += B.T;
    xb[S::NF + 1] += B.rv;
    xb[S::NF + 2] += B.p;
}

// Nodal flux: xbar += sum_j sum_f Fbar[j][f] dF_jf / dx
template <class S>
__device__ __forceinline__ void flux_vjp(const double *x, double brd, double brm, double bE,
                                         double bp, const double (*Fbar)[S::NF], const MeshData &M,
                                         double *xbar) {
    RainVel rvel = {0.0, 0.0, 0.0};
    if (S::RAIN) rvel = rain_velocity_partials(x[2], brm + x[1], M);
    Prim<S::D, S::RAIN, double> P;
    make_prim<S, double>(P, x, brd, brm, bE, bp, x[S::NF], x[S::NF + 1], x[S::NF + 2]);
    if (S::RAIN) P.vr = rvel.v;
    PrimBar<S::D> B;
    zero_bar<S::D>(B);
#pragma unroll
    for (int j = 0; j < S::D; ++j) flux_dir_vjp<S>(P, j, Fbar[j], B);
    prim_to_inputs<S>(P, B, rvel, xbar);
}

// Sources G (Eq. (2.4), gravity) as functions of x = (U, T, rho_v, p'):
// forward-mode Jacobian-vector products dotted with the adjoint wv.
template <class S>
__device__ __forceinline__ void source_vjp(const double *x, double brd, double brm,
                                           const double *wv, const MeshData &M,
                                           const double *__restrict__ tab, double *xbar) {
    const double g = M.g;
    // gravity: G_{m_vert} = -g (rho_d' + rho_m' + rho_r'), G_E = -g m_vert
    const double wm = wv[S::IM + S::VERT];
    xbar[0] -= g * wm;
    xbar[1] -= g * wm;
    if (S::RAIN) xbar[2] -= g * wm;
    xbar[S::IM + S::VERT] -= g * wv[S::IE];
    if (!S::RAIN) return;
    // microphysics: G_rm = S_ev - S_au - S_ac, G_rr = -G_rm; inputs rho_m', rho_r', T, rho_v
    const double wg = wv[1] - wv[2];
    const int ins[4] = {1, 2, S::NF, S::NF + 1};
    const double rm0 = brm + x[1];
    const bool sat = rm0 - x[S::NF + 1] > 0.0;
    // the pieces that depend on one input only, evaluated once with their
    // derivatives: rho_vs(T) (table) and x_r = rho_r^(1/16)
    double drvs;
    const double rvs = rho_vs_tab(x[S::NF], tab, drvs);
    const Dual rvs1(rvs, drvs);
    // x_r = rho_r^(1/16) = rho_r q^15, q = rho_r^(-1/16); dx_r/drho_r = x_r / (16 rho_r)
    // at max(rho_r, floor)
    const bool rpos = gt0(x[2]);
    Dual xr1(0.0);
    if (rpos) {
        const double q = inv_root16(x[2]);
        const double q2 = q * q, q4 = q2 * q2, q8 = q4 * q4;
        const double xr = x[2] * (q8 * q4 * q2 * q);
        xr1 = Dual(xr, x[2] > M.rain_floor ? 0.0625 * xr * recip(x[2]) : M.rain_d16);
    }
    for (int c = 0; c < 4; ++c) {
        const int k = ins[c];
        const Dual rm = Dual(brm) + Dual(x[1], k == 1 ? 1.0 : 0.0);
        const Dual T = Dual(x[S::NF], k == S::NF ? 1.0 : 0.0);
        const Dual rv = Dual(x[S::NF + 1], k == S::NF + 1 ? 1.0 : 0.0);
        const Dual rc = rm - rv;
        Dual deficit = Dual(rvs1.v, k == S::NF ? rvs1.d : 0.0) - rv;
        if (sat) deficit.v = 0.0;            // the forward value is exactly 0 at saturation
        const Dual xr = Dual(xr1.v, k == 2 ? xr1.d : 0.0);
        const Dual x2 = xr * xr, x3 = x2 * xr, x4 = x2 * x2, x8 = x4 * x4, x14 = x8 * x4 * x2;
        const Dual s_ev = (Dual(kSevA) - Dual(kSevB) * (T - Dual(kTref))) *
                          (Dual(1.0) + Dual(kSevC) * x3) * deficit * x8;
        const Dual s_au = rc.v > 0.0 ? Dual(kSau) * rc : Dual(0.0);
        const Dual s_ac = Dual(kSac) * rc * x14;
        xbar[k] += wg * (s_ev - s_au - s_ac).d;
    }
    (void)brd;
}

// Lax-Friedrichs face flux: adjoints of both traces at one face point.
template <class S, int J>
__device__ __forceinline__ void face_vjp(const AdjArgs &A, const double *s_w, double *s_ta, int el2,
                                         int face, int q, int e2) {
    constexpr int STR = S::EPB * S::NP;
    const MeshData &M = A.M;
    const int ne = M.ne;
    const int s = (face & 1) ? 1 : -1;
    double tm[S::NTR], tp[S::NTR];
#pragma unroll
    for (int fld = 0; fld < S::NTR; ++fld)
        tm[fld] = has_trace<S>(fld, J) ? A.trace[(((size_t)face * S::NTR + fld) * ne + e2) * S::NFP1 + q]
                                       : 0.0;
    const int nb = neighbour<S::D>(M, e2, J, s);
    if (nb >= 0) {
        const int fo = 2 * J + (s > 0 ? 0 : 1);
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            tp[fld] = has_trace<S>(fld, J) ? A.trace[(((size_t)fo * S::NTR + fld) * ne + nb) * S::NFP1 + q]
                                           : 0.0;
    } else {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) tp[fld] = tm[fld];
        tp[S::IM + J] = -tm[S::IM + J];
    }
    double brd, brm, bE, bp;
    const int iz = vert_index<S::D>(M, e2);
    if (J == S::VERT) {
        load_base<S, double>(A.bface, M.nzlev_face, iz + (s > 0 ? 1 : 0), brd, brm, bE, bp);
    } else {
        load_base<S, double>(A.bnode, M.nzlev_node, iz * S::P1 + face_q_vert<S::D, S::P1>(J, q), brd,
                             brm, bE, bp);
    }
    // adjoint of Fhat: R_a -= (2/h_J) l_a(s)/w_a Fhat(q) along the line through q
    const double *lift = (face & 1) ? A.ref.liftp : A.ref.liftm;
    double fhb[S::NF];
#pragma unroll
    for (int f = 0; f < S::NF; ++f) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < S::P1; ++i)
            acc = ::fma(lift[i], s_w[f * STR + el2 * S::NP + line_node<S::D, S::P1>(J, q, i)], acc);
        fhb[f] = -M.two_over_h[J] * acc;
    }
    // values: which side's wave speed is the max (forward: lam = lm > lp ? lm : lp)
    Prim<S::D, S::RAIN, double> Pm, Pp;
    make_prim<S, double>(Pm, tm, brd, brm, bE, bp, tm[S::NF], tm[S::NF + 1], tm[S::NF + 2]);
    make_prim<S, double>(Pp, tp, brd, brm, bE, bp, tp[S::NF], tp[S::NF + 1], tp[S::NF + 2]);
    if (S::RAIN) {
        Pm.vr = rain_velocity(Pm.rr, Pm.rm, M);
        Pp.vr = rain_velocity(Pp.rr, Pp.rm, M);
    }
    const double lmv = wave_speed<S, J, double>(Pm), lpv = wave_speed<S, J, double>(Pp);
    const bool m_active = lmv > lpv;
    const double lam = m_active ? lmv : lpv;
    const double hs = 0.5 * s;
    double tmb[S::NTR], tpb[S::NTR];
    // d Fhat / d(side) = hs dF_J/d(side) + [active] (dLambda/d(side)) (tm - tp)/2
    //                    + jsign lam/2 on the field itself
    double Fb[S::NF], lb = 0.0;
#pragma unroll
    for (int f = 0; f < S::NF; ++f) {
        Fb[f] = hs * fhb[f];
        lb = ::fma(fhb[f], 0.5 * (tm[f] - tp[f]), lb);
    }
    RainVel rv_m = {0.0, 0.0, 0.0}, rv_p = {0.0, 0.0, 0.0};
    if (S::RAIN && J == S::VERT) {
        rv_m = rain_velocity_partials(Pm.rr, Pm.rm, M);
        rv_p = rain_velocity_partials(Pp.rr, Pp.rm, M);
        Pm.vr = rv_m.v;
        Pp.vr = rv_p.v;
    }
    PrimBar<S::D> Bm, Bp, Bw;
    zero_bar<S::D>(Bm);
    zero_bar<S::D>(Bp);
    zero_bar<S::D>(Bw);
    flux_dir_vjp<S>(Pm, J, Fb, Bm);
    flux_dir_vjp<S>(Pp, J, Fb, Bp);
    // the wave speed of the active side, once per lane (the side is chosen
    // per lane by selects, so the warp runs this without divergence)
    {
        const Prim<S::D, S::RAIN, double> Pa = m_active ? Pm : Pp;
        wave_speed_vjp<S, J>(Pa, lb, Bw);
    }
    add_bar_if<S::D>(Bm, Bw, m_active);
    add_bar_if<S::D>(Bp, Bw, !m_active);
#pragma unroll
    for (int k = 0; k < S::NTR; ++k) tmb[k] = tpb[k] = 0.0;
    prim_to_inputs<S>(Pm, Bm, rv_m, tmb);
    prim_to_inputs<S>(Pp, Bp, rv_p, tpb);
    // the jump term: d[[U]]/dU^- = 1, d[[U]]/dU^+ = -1
#pragma unroll
    for (int f = 0; f < S::NF; ++f) {
        tmb[f] = ::fma(0.5 * lam, fhb[f], tmb[f]);
        tpb[f] = ::fma(-0.5 * lam, fhb[f], tpb[f]);
    }
    if (nb >= 0) {
        // the + side is the neighbour's trace on its face (J, -s)
        const int fo = 2 * J + (s > 0 ? 0 : 1);
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld)
            A.tadj[(((size_t)fo * S::NTR + fld) * ne + nb) * S::NFP1 + q] = tpb[fld];
    } else {
        // wall ghost: tp = tm with m_J negated
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) tmb[fld] += (fld == S::IM + J) ? -tpb[fld] : tpb[fld];
    }
    double *o = s_ta + ((size_t)(el2 * S::NFACE + face) * S::NTR) * S::NFP1 + q;
#pragma unroll
    for (int fld = 0; fld < S::NTR; ++fld) o[fld * S::NFP1] = tmb[fld];
}

template <class S>
constexpr size_t adj_smem_bytes() {
    return sizeof(double) * ((size_t)S::NF * S::EPB * S::NP + (size_t)S::EPB * S::NFACE * S::NTR * S::NFP1);
}

template <class S>
__global__ void __launch_bounds__(S::NT) k_adj_local(AdjArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int STR = S::EPB * S::NP;
    double *s_w = reinterpret_cast<double *>(smem_raw);        // [NF][STR]
    double *s_ta = s_w + S::NF * STR;                          // [EPB][NFACE][NTR][NFP1]
    const MeshData &M = A.M;
    const int ne = M.ne;
    const size_t nodes = (size_t)ne * S::NP;
    const int t = threadIdx.x;
    const int el = t / S::NP, a = t - el * S::NP;
    const int e = blockIdx.x * S::EPB + el;
    const bool valid = (t < STR) && (e < ne);
    double x[S::NTR], xbar[S::NTR];
    double brd = 0.0, brm = 0.0, bE = 0.0, bp = 0.0;
    if (valid) {
        const size_t gi = (size_t)e * S::NP + a;
#pragma unroll
        for (int f = 0; f < S::NF; ++f) {
            x[f] = A.U[f * nodes + gi];
            s_w[f * STR + t] = A.w[f * nodes + gi];
        }
        x[S::NF] = A.derived[gi];
        x[S::NF + 1] = A.derived[nodes + gi];
        x[S::NF + 2] = A.derived[2 * nodes + gi];
        const int lev = vert_index<S::D>(M, e) * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        load_base<S, double>(A.bnode, M.nzlev_node, lev, brd, brm, bE, bp);
#pragma unroll
        for (int k = 0; k < S::NTR; ++k) xbar[k] = 0.0;
    }
    __syncthreads();
    if (valid) {
        // volume: R_a += (2/h_j) sum_i dhat[a_j][i] F_j(i)  =>  Fbar_j(i) = (2/h_j) sum_a dhat[a_j][i] w(a)
        double Fbar[S::D][S::NF];
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            const int aj = digit<S::D, S::P1>(a, j);
            const int st = stride_of<S::P1>(j);
            const int b0 = el * S::NP + a - aj * st;
#pragma unroll
            for (int f = 0; f < S::NF; ++f) {
                double acc = 0.0;
#pragma unroll
                for (int i = 0; i < S::P1; ++i)
                    acc = ::fma(A.ref.dhat[i][aj], s_w[f * STR + b0 + i * st], acc);
                Fbar[j][f] = M.two_over_h[j] * acc;
            }
        }
        flux_vjp<S>(x, brd, brm, bE, bp, Fbar, M, xbar);
        double wv[S::NF];
#pragma unroll
        for (int f = 0; f < S::NF; ++f) wv[f] = s_w[f * STR + t];
        source_vjp<S>(x, brd, brm, wv, M, A.rvs_tab, xbar);
    }
    // face points in direction-major order (direction, element, side,
    // point), so that the lanes of a warp mostly share the face direction
    // and each direction-specialised body runs with full warps
    constexpr int PER_J = S::EPB * 2 * S::NFP1;
    for (int item = t; item < S::EPB * S::NFACE * S::NFP1; item += S::NT) {
        const int jd = item / PER_J;
        const int r = item - jd * PER_J;
        const int el2 = r / (2 * S::NFP1);
        const int r2 = r - el2 * (2 * S::NFP1);
        const int side = r2 / S::NFP1;
        const int q = r2 - side * S::NFP1;
        const int face = 2 * jd + side;
        const int e2 = blockIdx.x * S::EPB + el2;
        if (e2 >= ne) continue;
        switch (jd) {
            case 0: face_vjp<S, 0>(A, s_w, s_ta, el2, face, q, e2); break;
            case 1: face_vjp<S, 1>(A, s_w, s_ta, el2, face, q, e2); break;
            default: face_vjp<S, (S::D == 3 ? 2 : 1)>(A, s_w, s_ta, el2, face, q, e2); break;
        }
    }
    __syncthreads();
    if (valid) {
        // own-side trace adjoints back to the nodes: trace = sum_i l_i(s) v(line node i)
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            const int aj = digit<S::D, S::P1>(a, j);
            const int q = face_q<S::D, S::P1>(a, j);
            const double cm = A.ref.lm[aj], cp = A.ref.lp[aj];
            const double *tmn = s_ta + ((size_t)(el * S::NFACE + 2 * j) * S::NTR) * S::NFP1 + q;
            const double *tpl = s_ta + ((size_t)(el * S::NFACE + 2 * j + 1) * S::NTR) * S::NFP1 + q;
#pragma unroll
            for (int fld = 0; fld < S::NTR; ++fld)
                xbar[fld] += cm * tmn[fld * S::NFP1] + cp * tpl[fld * S::NFP1];
        }
        const size_t gi = (size_t)e * S::NP + a;
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) A.ubar_part[fld * nodes + gi] = xbar[fld];
    }
}

// Split Eq. (2.8) differentiated at one node: given the adjoints of T, rho_v
// and p' = (rho_d R_d + rho_v R_v) T - p_bar, add the adjoints of the totals
// and of rho e, then of U.  Unsaturated: T = T_ref + (rho e - rho_m L')/C_u,
// rho_v = rho_m.  Saturated: H(T, x) = 0 gives dT = -(dH/dx dx)/H'(T) and
// rho_v = rho_vs(T).
template <class S>
__device__ __forceinline__ void split_vjp(const double *u, double brd, double brm, double bE,
                                          double T, double rv, double Tb, double rvb, double ppb,
                                          const double *__restrict__ tab, double *ub) {
    const double rd = brd + u[0], rm = brm + u[1], rr = S::RAIN ? u[2] : 0.0;
    const double rho = rd + rm + rr;
    double msq = 0.0;
#pragma unroll
    for (int j = 0; j < S::D; ++j) msq += u[S::IM + j] * u[S::IM + j];
    // p'
    double rdb = ppb * kRd * T, rmb = 0.0, rrb = 0.0;
    Tb += ppb * (rd * kRd + rv * kRv);
    rvb += ppb * kRv * T;
    double reb;
    const bool sat = rm - rv > 0.0;
    if (!sat) {
        // rho_v = rho_m; T = T_ref + (re - rm L') / C_u
        rmb += rvb;
        const double cu = kCvd * rd + kCvv * rm + kCl * rr;
        const double dT = (T - kTref);
        reb = Tb * recip(cu);
        rmb += reb * (-kLprime - kCvv * dT);
        rdb += reb * (-kCvd * dT);
        rrb += reb * (-kCl * dT);
    } else {
        double drvs;
        const double rvs = rho_vs_tab(T, tab, drvs);
        Tb += rvb * drvs;                              // rho_v = rho_vs(T)
        const double heat = kCvd * rd + kCvv * rvs + kCl * (rm - rvs + rr);
        const double dH = heat + ((kCvv - kCl) * (T - kTref) + kLprime) * drvs;
        const double lam = Tb * recip(dH);             // dT = -(H_x dx) / H'
        const double dT = (T - kTref);
        rdb -= lam * kCvd * dT;
        rmb -= lam * kCl * dT;
        rrb -= lam * kCl * dT;
        reb = lam;                                     // H_re = -1
    }
    // re = E - |m|^2 / (2 rho)
    const double irho = recip(rho);
    const double rhob = 0.5 * reb * msq * irho * irho;
    ub[0] += rdb + rhob;
    ub[1] += rmb + rhob;
    if (S::RAIN) ub[2] += rrb + rhob;
#pragma unroll
    for (int j = 0; j < S::D; ++j) ub[S::IM + j] -= reb * u[S::IM + j] * irho;
    ub[S::IE] += reb;
    (void)bE;
}

template <class S>
__global__ void k_adj_gather(AdjArgs A) {
    const MeshData &M = A.M;
    const int ne = M.ne;
    const size_t nodes = (size_t)ne * S::NP;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < nodes;
         gi += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(gi / S::NP), a = (int)(gi - (size_t)e * S::NP);
        double xb[S::NTR];
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) xb[fld] = A.ubar_part[fld * nodes + gi];
        // neighbours' contributions to this element's traces
#pragma unroll
        for (int j = 0; j < S::D; ++j) {
            const int aj = digit<S::D, S::P1>(a, j);
            const int q = face_q<S::D, S::P1>(a, j);
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
                const int s = sd ? 1 : -1;
                if (neighbour<S::D>(M, e, j, s) < 0) continue;
                const int face = 2 * j + sd;
                const double c = sd ? A.ref.lp[aj] : A.ref.lm[aj];
#pragma unroll
                for (int fld = 0; fld < S::NTR; ++fld)
                    xb[fld] += c * A.tadj[(((size_t)face * S::NTR + fld) * ne + e) * S::NFP1 + q];
            }
        }
        double u[S::NF];
#pragma unroll
        for (int f = 0; f < S::NF; ++f) u[f] = A.U[f * nodes + gi];
        const int lev = vert_index<S::D>(M, e) * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        double brd, brm, bE, bp;
        load_base<S, double>(A.bnode, M.nzlev_node, lev, brd, brm, bE, bp);
        split_vjp<S>(u, brd, brm, bE, A.derived[gi], A.derived[nodes + gi], xb[S::NF], xb[S::NF + 1],
                     xb[S::NF + 2], A.rvs_tab, xb);
#pragma unroll
        for (int f = 0; f < S::NF; ++f) {
            const size_t o = f * nodes + gi;
            double v = A.gamma * xb[f];
            if (A.beta != 0.0) v += A.beta * A.w[o];
            if (A.alpha != 0.0) v += A.alpha * A.out[o];
            A.out[o] = v;
        }
    }
}

// Cloud-water functional J = sum_nodes W_a |K|/2^d rho_c and its gradient
// dJ/dU (rho_c = rho_m - rho_v from the split at the nodes).
template <class S>
__global__ void __launch_bounds__(kRedThreads) k_cloud(AdjArgs A, double *partials) {
    __shared__ double sh[kRedThreads];
    const MeshData &M = A.M;
    const size_t nodes = (size_t)M.ne * S::NP;
    double acc = 0.0;
    for (size_t gi = (size_t)blockIdx.x * blockDim.x + threadIdx.x; gi < nodes;
         gi += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(gi / S::NP), a = (int)(gi - (size_t)e * S::NP);
        double W = M.jac;
#pragma unroll
        for (int j = 0; j < S::D; ++j) W *= A.ref.w[digit<S::D, S::P1>(a, j)];
        double u[S::NF], ub[S::NF];
#pragma unroll
        for (int f = 0; f < S::NF; ++f) {
            u[f] = A.U[f * nodes + gi];
            ub[f] = 0.0;
        }
        const int lev = vert_index<S::D>(M, e) * S::P1 + digit<S::D, S::P1>(a, S::VERT);
        double brd, brm, bE, bp;
        load_base<S, double>(A.bnode, M.nzlev_node, lev, brd, brm, bE, bp);
        const double T = A.derived[gi], rv = A.derived[nodes + gi];
        acc += W * (brm + u[1] - rv);
        ub[1] += W;                                       // d rho_c / d rho_m'
        split_vjp<S>(u, brd, brm, bE, T, rv, 0.0, -W, 0.0, A.rvs_tab, ub);
#pragma unroll
        for (int f = 0; f < S::NF; ++f) A.out[f * nodes + gi] = ub[f];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kRedThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

}  // namespace dgm
