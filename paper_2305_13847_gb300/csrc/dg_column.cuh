// Column march: one SSPRK stage (or the right-hand side) of the float32 forms
// with the face data kept on chip.
//
// A CTA owns a brick of BX x BY element columns (3-D; a row of BX columns in
// 2-D) and marches up through the vertical layers.  At layer L it holds the
// node values of layers L and L+1 in shared memory, so that
//   * the face between L and L+1 (normal to e_z) is evaluated there, once,
//     and its flux serves as the top face of L and the bottom face of L+1;
//   * the horizontal faces between elements of the brick are evaluated from
//     shared memory, once each;
//   * only the faces on the brick's sides need the neighbouring brick's
//     traces, which go through HBM: the stage writes the side traces of the
//     state it produces, the next stage reads them.
// A face on a brick side is evaluated by both bricks from the same two traces
// with the same arithmetic (lf_flux), so both get the same flux bitwise and
// the conservation of the face-pass schedule holds.  Per node the stage then
// reads and writes the state and the derived fields and a trace share of the
// brick sides only, instead of every face trace and face flux.
//
// The arithmetic per node and face point is that of the other two schedules
// (stage_block's nodal flux, sum-factorised volume term, lift and stage
// update; lf_flux on faces; split_and_store), so the right-hand side is
// bitwise the face pass's.
#pragma once

#include "dg_device.cuh"

namespace dgm {

template <class S>
struct ColShape {
    // 3-D: 2 x 2 columns for k >= 3 (256, 500, 864 nodes per layer), 3 x 3 for
    // k = 2, 4 x 8 for k = 1; 2-D: a row of about 256 nodes
    static constexpr int BX = S::D == 3 ? (S::K >= 3 ? 2 : (S::K == 2 ? 3 : 4))
                                        : ((256 / S::NP) > 0 ? 256 / S::NP : 1);
    static constexpr int BY = S::D == 3 ? (S::K >= 3 ? 2 : (S::K == 2 ? 3 : 8)) : 1;
    static constexpr int TE = BX * BY;               // elements of one layer of the brick
    static constexpr int STR = TE * S::NP;           // nodes of one layer of the brick
    static constexpr int NT = ((STR + 31) / 32) * 32;
    static constexpr int NXF = (BX + 1) * BY;        // faces normal to e_0 in a layer of the brick
    static constexpr int NYF = S::D == 3 ? BX * (BY + 1) : 0;   // normal to e_1 (3-D)
    static constexpr int NHF = NXF + NYF;            // horizontal faces
    static constexpr int FB = S::NF * S::NFP1;       // flux values of one face
    // node rows of a layer in shared memory: the NTR traced values (U, T,
    // rho_v, p'), then with rain the microphysics source and v_r
    static constexpr int NROW = S::NTR + (S::RAIN ? 2 : 0);
    // CTAs per SM the register budget is sized for (64 registers at 4 x 256)
    static constexpr int MINB = (1024 / NT) > 0 ? 1024 / NT : 1;
};

template <class S, typename Real>
constexpr size_t column_smem_bytes() {
    using C = ColShape<S>;
    return sizeof(Real) * ((size_t)S::D * S::NF * C::STR + 2 * (size_t)C::NROW * C::STR +
                           2 * (size_t)C::TE * C::FB + (size_t)C::NHF * C::FB);
}

// Where the element on one side of a horizontal face of the brick lies:
// kind 0 a wall (no element), 1 an element of this brick (loc = its local
// index), 2 an element of another brick (glob = its column).  c[] are the
// side's column coordinates relative to the mesh (may lie outside it).
struct ColSide {
    int kind, loc, glob;
};

template <class S>
__device__ __forceinline__ ColSide col_side(const MeshData &M, int cx0, int cy0, int x, int y) {
    using C = ColShape<S>;
    ColSide r;
    r.kind = 0;
    r.loc = -1;
    r.glob = -1;
    if (x < 0 || x >= M.n[0]) {
        if (!M.periodic[0]) return r;
        x = x < 0 ? x + M.n[0] : x - M.n[0];
    }
    if (S::D == 3 && (y < 0 || y >= M.n[1])) {
        if (!M.periodic[1]) return r;
        y = y < 0 ? y + M.n[1] : y - M.n[1];
    }
    if (S::D == 2) y = 0;
    const int bx = x - cx0, by = y - cy0;
    if (bx >= 0 && bx < C::BX && by >= 0 && by < C::BY) {
        r.kind = 1;
        r.loc = bx + C::BX * by;
    } else {
        r.kind = 2;
    }
    r.glob = x + M.n[0] * y;
    return r;
}

// traces of the NTR fields of local element el at face point q of face (J, s)
// from the node values in s_tr [NTR][STR] (the interpolation chain of
// write_line / interp_face, so bitwise the traces the other schedules store)
template <class S, typename Real, int J, int STR>
__device__ __forceinline__ void col_trace_smem(const RefData<Real> &ref, const Real *s_tr, int el, int s,
                                               int q, Real *tr) {
    const Real *ls = s > 0 ? ref.lp : ref.lm;
#pragma unroll
    for (int fld = 0; fld < S::NTR; ++fld)
        tr[fld] = has_trace<S>(fld, J) ? interp_face<S, Real>(s_tr + fld * STR + el * S::NP, ls, J, q)
                                       : Real(0);
}

// one horizontal face point (J < VERT) of the brick layer: G along +e_J
template <class S, typename Real, int J>
__device__ __forceinline__ void col_hface(const KArgs<Real> &A, const Real *s_tr, Real *s_fh, int f, int q,
                                          int cx0, int cy0, int iz, int lo_x, int lo_y, int hi_x,
                                          int hi_y) {
    using C = ColShape<S>;
    const MeshData &M = A.M;
    const int ne = M.ne;
    const int ncol = S::D == 3 ? M.n[0] * M.n[1] : M.n[0];
    const ColSide lo = col_side<S>(M, cx0, cy0, lo_x, lo_y);
    const ColSide hi = col_side<S>(M, cx0, cy0, hi_x, hi_y);
    // needed only where an element of this brick lifts it
    if (lo.kind != 1 && hi.kind != 1) return;
    Real tl[S::NTR], th[S::NTR];
    const ColSide sides[2] = {lo, hi};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        Real *tr = side == 0 ? tl : th;
        const ColSide &sd = sides[side];
        if (sd.kind == 1) {
            // the low element's high face, the high element's low face
            col_trace_smem<S, Real, J, C::STR>(A.ref, s_tr, sd.loc, side == 0 ? 1 : -1, q, tr);
        } else if (sd.kind == 2) {
            const int e = sd.glob + ncol * iz;
            const int face = 2 * J + (side == 0 ? 1 : 0);
#pragma unroll
            for (int fld = 0; fld < S::NTR; ++fld)
                tr[fld] = has_trace<S>(fld, J)
                              ? A.trace_in[(((size_t)face * S::NTR + fld) * ne + e) * S::NFP1 + q]
                              : Real(0);
        }
    }
    // slip wall: the ghost copies the other side with m.n mirrored
    if (lo.kind == 0) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) tl[fld] = th[fld];
        tl[S::IM + J] = -th[S::IM + J];
    }
    if (hi.kind == 0) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) th[fld] = tl[fld];
        th[S::IM + J] = -tl[S::IM + J];
    }
    Real brd, brm, bE, bp;
    load_base<S, Real>(A.bnode, M.nzlev_node, iz * S::P1 + face_q_vert<S::D, S::P1>(J, q), brd, brm, bE,
                       bp);
    Real G[S::NF];
    lf_flux<S, Real, J>(tl, th, brd, brm, bE, bp, M, G);
    Real *out = s_fh + (size_t)f * C::FB + q;
#pragma unroll
    for (int fld = 0; fld < S::NF; ++fld) out[fld * S::NFP1] = G[fld];
}

// the vertical face at the top of element el of layer iz (its bottom if
// bottom = true, only for iz = 0): G along +e_z into gz [NF][NFP1]
template <class S, typename Real>
__device__ __forceinline__ void col_vface(const KArgs<Real> &A, const Real *s_lo, const Real *s_hi,
                                          Real *gz, int el, int q, int iz, bool bottom, int col) {
    using C = ColShape<S>;
    constexpr int J = S::VERT;
    const MeshData &M = A.M;
    const int nz = M.n[J];
    Real tl[S::NTR], th[S::NTR];
    const bool wall_lo = bottom, wall_hi = !bottom && iz == nz - 1;
    if (!wall_lo) col_trace_smem<S, Real, J, C::STR>(A.ref, s_lo, el, 1, q, tl);
    if (!wall_hi) col_trace_smem<S, Real, J, C::STR>(A.ref, bottom ? s_lo : s_hi, el, -1, q, th);
    if (wall_lo) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) tl[fld] = th[fld];
        tl[S::IM + J] = -th[S::IM + J];
    }
    if (wall_hi) {
#pragma unroll
        for (int fld = 0; fld < S::NTR; ++fld) th[fld] = tl[fld];
        th[S::IM + J] = -tl[S::IM + J];
    }
    const int lev = bottom ? 0 : iz + 1;
    Real brd, brm, bE, bp;
    load_base<S, Real>(A.bface, M.nzlev_face, lev, brd, brm, bE, bp);
    Real G[S::NF];
    lf_flux<S, Real, J>(tl, th, brd, brm, bE, bp, M, G);
#pragma unroll
    for (int fld = 0; fld < S::NF; ++fld) gz[fld * S::NFP1 + q] = G[fld];
    if (S::RAIN && (wall_lo || wall_hi) && A.fallout) {
        // outward normal -e_z at the bottom wall, +e_z at the top
        const double gw = to_f64(G[1]) + to_f64(G[2]);
        add_fallout<S, Real>(A, wall_hi, col, q, wall_lo ? -gw : gw);
    }
}

template <class S, typename Real, int MODE>
__global__ void __launch_bounds__(ColShape<S>::NT, ColShape<S>::MINB) k_column(KArgs<Real> A) {
    using C = ColShape<S>;
    constexpr int STR = C::STR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *s_fl = reinterpret_cast<Real *>(smem_raw);      // [D][NF][STR] nodal fluxes
    Real *s_trb = s_fl + S::D * S::NF * STR;              // [2][NROW][STR] node values, layer parity
    Real *s_gz = s_trb + 2 * C::NROW * STR;               // [2][TE][NF][NFP1] vertical faces, layer parity
    Real *s_fh = s_gz + 2 * C::TE * C::FB;                // [NHF][NF][NFP1] horizontal faces
    const MeshData &M = A.M;
    const RefData<Real> &ref = A.ref;
    const size_t nodes = (size_t)M.ne * S::NP;
    const int nz = M.n[S::VERT];
    const int ncol = S::D == 3 ? M.n[0] * M.n[1] : M.n[0];
    const int nxb = (M.n[0] + C::BX - 1) / C::BX;
    const int cx0 = (blockIdx.x % nxb) * C::BX;
    const int cy0 = S::D == 3 ? (blockIdx.x / nxb) * C::BY : 0;
    const int t = threadIdx.x;
    const int el = t / S::NP, a = t - el * S::NP;
    const int bx = el % C::BX, by = el / C::BX;
    const bool valid = t < STR && cx0 + bx < M.n[0] && (S::D == 2 || cy0 + by < M.n[1]);
    const int col = (cx0 + bx) + (S::D == 3 ? M.n[0] * (cy0 + by) : 0);
    const int av = digit<S::D, S::P1>(a, S::VERT);

    // this node's values of one layer (U, T, rho_v, p', G_rm, v_r) from the
    // state and derived fields to row t of s_tr
    auto load = [&](int iz, Real *v) {
        const size_t gi = (size_t)(col + ncol * iz) * S::NP + a;
#pragma unroll
        for (int f = 0; f < S::NF; ++f) v[f] = A.Uin[f * nodes + gi];
#pragma unroll
        for (int d = 0; d < (S::RAIN ? 5 : 3); ++d) v[S::NF + d] = A.derived[d * nodes + gi];
    };
    auto put = [&](Real *s_tr, const Real *v) {
#pragma unroll
        for (int r = 0; r < C::NROW; ++r) s_tr[r * STR + t] = v[r];
    };

    // prologue: layer 0 and the bottom wall's flux
    if (valid) {
        Real v[C::NROW];
        load(0, v);
        put(s_trb, v);
    }
    __syncthreads();
    for (int item = t; item < C::TE * S::NFP1; item += C::NT) {
        const int e2 = item / S::NFP1, q = item - e2 * S::NFP1;
        const int x = cx0 + e2 % C::BX, y = cy0 + e2 / C::BX;
        if (x >= M.n[0] || (S::D == 3 && y >= M.n[1])) continue;
        col_vface<S, Real>(A, s_trb, s_trb, s_gz + (size_t)e2 * C::FB, e2, q, 0, true,
                           x + (S::D == 3 ? M.n[0] * y : 0));
    }

    for (int iz = 0; iz < nz; ++iz) {
        Real *s_trc = s_trb + (iz & 1) * C::NROW * STR;         // layer iz (state U_s)
        Real *s_trn = s_trb + ((iz + 1) & 1) * C::NROW * STR;   // layer iz + 1
        const Real *s_gzb = s_gz + (iz & 1) * C::TE * C::FB;    // bottom faces of iz
        Real *s_gzt = s_gz + ((iz + 1) & 1) * C::TE * C::FB;    // top faces of iz
        const bool more = iz + 1 < nz;
        // the next layer's node values: loads issued now, stored after the
        // nodal fluxes
        Real nv[C::NROW];
        if (valid && more) load(iz + 1, nv);

        // ---- nodal fluxes (stage_block's phase 1)
        if (valid) {
            Real u[S::NF];
#pragma unroll
            for (int f = 0; f < S::NF; ++f) u[f] = s_trc[f * STR + t];
            const int lev = iz * S::P1 + av;
            Real brd, brm, bE, bp;
            load_base<S, Real>(A.bnode, M.nzlev_node, lev, brd, brm, bE, bp);
            Prim<S::D, S::RAIN, Real> P;
            make_prim<S, Real>(P, u, brd, brm, bE, bp, s_trc[S::NF * STR + t],
                               s_trc[(S::NF + 1) * STR + t], s_trc[(S::NF + 2) * STR + t]);
            if (S::RAIN) P.vr = s_trc[(S::NTR + 1) * STR + t];
#pragma unroll
            for (int j = 0; j < S::D; ++j) {
                Real F[S::NF];
                flux_dir<S, Real>(P, j, F);
#pragma unroll
                for (int f = 0; f < S::NF; ++f) s_fl[(j * S::NF + f) * STR + t] = F[f];
            }
            if (more) put(s_trn, nv);
        }
        __syncthreads();

        // ---- faces of the layer: horizontal faces of the brick, and the
        // vertical faces between this layer and the next (or the top wall)
        for (int item = t; item < (C::NHF + C::TE) * S::NFP1; item += C::NT) {
            const int f = item / S::NFP1, q = item - f * S::NFP1;
            if (f < C::NXF) {
                const int ry = f / (C::BX + 1), px = f - ry * (C::BX + 1);
                col_hface<S, Real, 0>(A, s_trc, s_fh, f, q, cx0, cy0, iz, cx0 + px - 1, cy0 + ry,
                                      cx0 + px, cy0 + ry);
            } else if (f < C::NHF) {
                if (S::D == 3) {
                    const int g2 = f - C::NXF;
                    const int py = g2 / C::BX, rx = g2 - py * C::BX;
                    col_hface<S, Real, (S::D == 3 ? 1 : 0)>(A, s_trc, s_fh, f, q, cx0, cy0, iz, cx0 + rx,
                                                           cy0 + py - 1, cx0 + rx, cy0 + py);
                }
            } else {
                const int e2 = f - C::NHF;
                const int x = cx0 + e2 % C::BX, y = cy0 + e2 / C::BX;
                if (x < M.n[0] && (S::D == 2 || y < M.n[1]))
                    col_vface<S, Real>(A, s_trc, s_trn, s_gzt + (size_t)e2 * C::FB, e2, q, iz, false,
                                       x + (S::D == 3 ? M.n[0] * y : 0));
            }
        }
        __syncthreads();

        // ---- sources, volume term, lift and stage update (stage_block's
        // phases 1, 2a and 3 in the same order of operations)
        if (valid) {
            Real u[S::NF], R[S::NF];
#pragma unroll
            for (int f = 0; f < S::NF; ++f) {
                u[f] = s_trc[f * STR + t];
                R[f] = Real(0);
            }
            if (S::RAIN) {
                const Real dgm = s_trc[S::NTR * STR + t];
                R[1] = dgm;
                R[2] = -dgm;
            }
            const Real g = mconst<Real>(M.g, M.g_f);
            R[S::IM + S::VERT] = -g * (u[0] + u[1] + (S::RAIN ? u[2] : Real(0)));
            R[S::IE] = -g * u[S::IM + S::VERT];
#pragma unroll
            for (int j = 0; j < S::D; ++j) {
                const int aj = digit<S::D, S::P1>(a, j);
                const int st = stride_of<S::P1>(j);
                const int b0 = el * S::NP + a - aj * st;
#pragma unroll
                for (int f = 0; f < S::NF; ++f) {
                    const Real *fl = s_fl + (j * S::NF + f) * STR + b0;
                    Real acc = R[f];
#pragma unroll
                    for (int i = 0; i < S::P1; ++i) acc = fma(A.ref.dhat_s[j][aj][i], fl[i * st], acc);
                    R[f] = acc;
                }
            }
            // lift, face-pass convention: every face holds G along +e_j
#pragma unroll
            for (int j = 0; j < S::D; ++j) {
                const int aj = digit<S::D, S::P1>(a, j);
                const int q = face_q<S::D, S::P1>(a, j);
                const Real *fm, *fp;
                if (j == S::VERT) {
                    fm = s_gzb + (size_t)el * C::FB;
                    fp = s_gzt + (size_t)el * C::FB;
                } else if (j == 0) {
                    const int lo = by * (C::BX + 1) + bx;
                    fm = s_fh + (size_t)lo * C::FB;
                    fp = s_fh + (size_t)(lo + 1) * C::FB;
                } else {
                    const int lo = C::NXF + by * C::BX + bx;
                    fm = s_fh + (size_t)lo * C::FB;
                    fp = s_fh + (size_t)(lo + C::BX) * C::FB;
                }
                fm += q;
                fp += q;
                const Real cm = A.ref.liftm_s[j][aj], cp = A.ref.liftp_s[j][aj];
#pragma unroll
                for (int f = 0; f < S::NF; ++f)
                    R[f] = fma(cm, fm[f * S::NFP1], fma(-cp, fp[f * S::NFP1], R[f]));
            }
            const size_t gi = (size_t)(col + ncol * iz) * S::NP + a;
            if (MODE == MODE_RHS) {
#pragma unroll
                for (int f = 0; f < S::NF; ++f) A.Uout[f * nodes + gi] = R[f];
            } else {
                Real unew[S::NF];
#pragma unroll
                for (int f = 0; f < S::NF; ++f) {
                    // one explicit fma: every stage kernel rounds the update alike;
                    // beta u is u itself when beta = 1 (three stages in four)
                    Real v = fma(A.gdt, R[f], is_one(A.beta) ? u[f] : A.beta * u[f]);
                    if (nonzero(A.alpha)) v = fma(A.alpha, A.Un[f * nodes + gi], v);
                    unew[f] = v;
                }
                if (A.sponge) {
                    const Real dl = A.sponge[iz * S::P1 + av];
                    if (dl != Real(0)) {
                        const Real om = Real(1) - dl;
                        Real removed = dl * unew[1];
                        if (S::RAIN) removed = add_rn(removed, dl * unew[2]);
                        unew[0] = unew[0] + removed;
#pragma unroll
                        for (int f = 1; f < S::NF; ++f) unew[f] = om * unew[f];
                    }
                }
#pragma unroll
                for (int f = 0; f < S::NF; ++f) A.Uout[f * nodes + gi] = unew[f];
                const Real Tprev = s_trc[S::NF * STR + t];
                split_and_store<S, Real, false, STR>(A, unew, col + ncol * iz, a, iz, s_trc, t,
                                                     nullptr, Tprev);
            }
        }
        if (MODE == MODE_STAGE) {
            __syncthreads();
            // side traces of the new state for the neighbouring bricks' next stage
            for (int item = t; item < C::TE * 2 * (S::D - 1) * S::NFP1; item += C::NT) {
                const int e2 = item / (2 * (S::D - 1) * S::NFP1);
                const int r = item - e2 * (2 * (S::D - 1) * S::NFP1);
                const int face = r / S::NFP1, q = r - face * S::NFP1;
                const int j = face >> 1, s = (face & 1) ? 1 : -1;
                const int x = cx0 + e2 % C::BX, y = cy0 + e2 / C::BX;
                if (x >= M.n[0] || (S::D == 3 && y >= M.n[1])) continue;
                const ColSide nb = col_side<S>(M, cx0, cy0, x + (j == 0 ? s : 0), y + (j == 1 ? s : 0));
                if (nb.kind != 2) continue;
                const int e = x + (S::D == 3 ? M.n[0] * y : 0) + ncol * iz;
                Real tr[S::NTR];
                if (j == 0)
                    col_trace_smem<S, Real, 0, STR>(ref, s_trc, e2, s, q, tr);
                else
                    col_trace_smem<S, Real, (S::D == 3 ? 1 : 0), STR>(ref, s_trc, e2, s, q, tr);
#pragma unroll
                for (int fld = 0; fld < S::NTR; ++fld)
                    if (has_trace<S>(fld, j))
                        A.trace_out[(((size_t)face * S::NTR + fld) * M.ne + e) * S::NFP1 + q] = tr[fld];
            }
        }
        __syncthreads();
    }
}

}  // namespace dgm
