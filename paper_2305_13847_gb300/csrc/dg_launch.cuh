// Host-side launchers of the device kernels, one table per (D, K, rain,
// storage type).  Instantiated in dg_inst_*.cu so that the configurations
// compile in parallel.
#pragma once

#include "dg_device.cuh"

namespace dgm {

template <typename Real>
struct Launchers {
    int nf, np, nfp1, nd, ntr, epb, nt;
    size_t prep_smem, stage_smem;
    cudaError_t (*prepare)(const KArgs<Real> &, cudaStream_t);
    // pf: the stage kernel takes its face fluxes from the face pass
    cudaError_t (*stage)(const KArgs<Real> &, int mode, bool pf, cudaStream_t);
    cudaError_t (*face)(const KArgs<Real> &, cudaStream_t);
    cudaError_t (*split)(const KArgs<Real> &, double *, double *, double *, double *, cudaStream_t);
    cudaError_t (*init_bubble)(const KArgs<Real> &, const BubbleArgs &, cudaStream_t);
    cudaError_t (*reduce)(const KArgs<Real> &, double *partials, int nblocks, cudaStream_t);
};

constexpr int kGridStrideBlocks = 152 * 8;

inline int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > (size_t)kGridStrideBlocks) b = kGridStrideBlocks;
    return (int)(b > 0 ? b : 1);
}

template <class S, typename Real>
struct Impl {
    static constexpr size_t prep_smem = sizeof(Real) * (size_t)S::NTR * S::EPB * S::NP;
    static constexpr size_t stage_smem = stage_smem_bytes<S, Real, false>();
    static constexpr size_t stage_smem_pf = stage_smem_bytes<S, Real, true>();

    static int blocks(const KArgs<Real> &A) { return (A.M.ne + S::EPB - 1) / S::EPB; }

    static cudaError_t prepare(const KArgs<Real> &A, cudaStream_t st) {
        static bool attr = false;
        if (!attr) {
            cudaError_t err = cudaFuncSetAttribute(k_prepare<S, Real>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)prep_smem);
            if (err != cudaSuccess) return err;
            attr = true;
        }
        k_prepare<S, Real><<<blocks(A), S::NT, prep_smem, st>>>(A);
        return cudaGetLastError();
    }

    template <int MODE, bool PF>
    static cudaError_t launch_stage(const KArgs<Real> &A, cudaStream_t st) {
        static bool attr = false;
        if (!attr) {
            cudaError_t err = cudaFuncSetAttribute(k_stage<S, Real, MODE, PF>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(PF ? stage_smem_pf : stage_smem));
            if (err != cudaSuccess) return err;
            attr = true;
        }
        k_stage<S, Real, MODE, PF><<<blocks(A), S::NT, PF ? stage_smem_pf : stage_smem, st>>>(A);
        return cudaGetLastError();
    }

    static cudaError_t stage(const KArgs<Real> &A, int mode, bool pf, cudaStream_t st) {
        if (mode == MODE_RHS)
            return pf ? launch_stage<MODE_RHS, true>(A, st) : launch_stage<MODE_RHS, false>(A, st);
        return pf ? launch_stage<MODE_STAGE, true>(A, st) : launch_stage<MODE_STAGE, false>(A, st);
    }

    static cudaError_t face(const KArgs<Real> &A, cudaStream_t st) {
        const int nb = A.M.fblk[0] + A.M.fblk[1] + A.M.fblk[2];
        k_face<S, Real><<<nb, kFaceThreads, 0, st>>>(A);
        return cudaGetLastError();
    }

    static cudaError_t split(const KArgs<Real> &A, double *T, double *rv, double *rc, double *pp,
                             cudaStream_t st) {
        const size_t nodes = (size_t)A.M.ne * S::NP;
        k_split<S, Real><<<grid_for(nodes, 256), 256, 0, st>>>(A, T, rv, rc, pp);
        return cudaGetLastError();
    }

    static cudaError_t init_bubble(const KArgs<Real> &A, const BubbleArgs &B, cudaStream_t st) {
        const size_t nodes = (size_t)A.M.ne * S::NP;
        k_init_bubble<S, Real><<<grid_for(nodes, 256), 256, 0, st>>>(A, B);
        return cudaGetLastError();
    }

    static cudaError_t reduce(const KArgs<Real> &A, double *partials, int nblocks, cudaStream_t st) {
        k_reduce_partial<S, Real><<<nblocks, kRedThreads, 0, st>>>(A, partials);
        return cudaGetLastError();
    }

    static Launchers<Real> table() {
        Launchers<Real> L;
        L.nf = S::NF;
        L.np = S::NP;
        L.nfp1 = S::NFP1;
        L.nd = S::ND;
        L.ntr = S::NTR;
        L.epb = S::EPB;
        L.nt = S::NT;
        L.prep_smem = prep_smem;
        L.stage_smem = stage_smem;
        L.prepare = &prepare;
        L.stage = &stage;
        L.face = &face;
        L.split = &split;
        L.init_bubble = &init_bubble;
        L.reduce = &reduce;
        return L;
    }
};

// Tables defined in the instantiation units; NULL for an unsupported order.
const Launchers<double> *launchers_d2_f64(int K, int rain);
const Launchers<double> *launchers_d3_f64(int K, int rain);
const Launchers<float> *launchers_d2_f32(int K, int rain);
const Launchers<float> *launchers_d3_f32(int K, int rain);

}  // namespace dgm

#define DGM_DEFINE_LAUNCHERS(NAME, DIM, REAL)                                          \
    namespace dgm {                                                                    \
    const Launchers<REAL> *NAME(int K, int rain) {                                     \
        static const Launchers<REAL> t[5][2] = {                                       \
            {Impl<Shape<DIM, 1, false>, REAL>::table(), Impl<Shape<DIM, 1, true>, REAL>::table()}, \
            {Impl<Shape<DIM, 2, false>, REAL>::table(), Impl<Shape<DIM, 2, true>, REAL>::table()}, \
            {Impl<Shape<DIM, 3, false>, REAL>::table(), Impl<Shape<DIM, 3, true>, REAL>::table()}, \
            {Impl<Shape<DIM, 4, false>, REAL>::table(), Impl<Shape<DIM, 4, true>, REAL>::table()}, \
            {Impl<Shape<DIM, 5, false>, REAL>::table(), Impl<Shape<DIM, 5, true>, REAL>::table()}, \
        };                                                                             \
        if (K < 1 || K > 5) return nullptr;                                            \
        return &t[K - 1][rain ? 1 : 0];                                                \
    }                                                                                  \
    }

// ---------------------------------------------------------------------------
// Adjoint launchers (float64 only), instantiated in dg_adj_*.cu
// ---------------------------------------------------------------------------
#include "dg_adjoint.cuh"

namespace dgm {

struct AdjLaunchers {
    int ntr;
    cudaError_t (*local)(const AdjArgs &, cudaStream_t);
    cudaError_t (*gather)(const AdjArgs &, cudaStream_t);
    cudaError_t (*cloud)(const AdjArgs &, double *partials, int nblocks, cudaStream_t);
};

template <class S>
struct AdjImpl {
    static constexpr size_t smem = adj_smem_bytes<S>();
    static cudaError_t local(const AdjArgs &A, cudaStream_t st) {
        static bool attr = false;
        if (!attr) {
            cudaError_t err = cudaFuncSetAttribute(k_adj_local<S>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            attr = true;
        }
        k_adj_local<S><<<(A.M.ne + S::EPB - 1) / S::EPB, S::NT, smem, st>>>(A);
        return cudaGetLastError();
    }
    static cudaError_t gather(const AdjArgs &A, cudaStream_t st) {
        const size_t nodes = (size_t)A.M.ne * S::NP;
        k_adj_gather<S><<<grid_for(nodes, 256), 256, 0, st>>>(A);
        return cudaGetLastError();
    }
    static cudaError_t cloud(const AdjArgs &A, double *partials, int nblocks, cudaStream_t st) {
        k_cloud<S><<<nblocks, kRedThreads, 0, st>>>(A, partials);
        return cudaGetLastError();
    }
    static AdjLaunchers table() {
        AdjLaunchers L;
        L.ntr = S::NTR;
        L.local = &local;
        L.gather = &gather;
        L.cloud = &cloud;
        return L;
    }
};

const AdjLaunchers *adj_launchers_d2(int K, int rain);
const AdjLaunchers *adj_launchers_d3(int K, int rain);

}  // namespace dgm

#define DGM_DEFINE_ADJ_LAUNCHERS(NAME, DIM)                                             \
    namespace dgm {                                                                    \
    const AdjLaunchers *NAME(int K, int rain) {                                        \
        static const AdjLaunchers t[5][2] = {                                          \
            {AdjImpl<Shape<DIM, 1, false>>::table(), AdjImpl<Shape<DIM, 1, true>>::table()}, \
            {AdjImpl<Shape<DIM, 2, false>>::table(), AdjImpl<Shape<DIM, 2, true>>::table()}, \
            {AdjImpl<Shape<DIM, 3, false>>::table(), AdjImpl<Shape<DIM, 3, true>>::table()}, \
            {AdjImpl<Shape<DIM, 4, false>>::table(), AdjImpl<Shape<DIM, 4, true>>::table()}, \
            {AdjImpl<Shape<DIM, 5, false>>::table(), AdjImpl<Shape<DIM, 5, true>>::table()}, \
        };                                                                             \
        if (K < 1 || K > 5) return nullptr;                                            \
        return &t[K - 1][rain ? 1 : 0];                                                \
    }                                                                                  \
    }
