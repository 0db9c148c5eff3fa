// Host-side launchers of the device kernels, one table per (D, K, rain,
// storage type).  Instantiated in dg_inst_*.cu so that the configurations
// compile in parallel.
#pragma once

#include <type_traits>

#include "dg_column.cuh"
#include "dg_device.cuh"

namespace dgm {

template <typename Real>
struct Launchers {
    int nf, np, nfp1, nd, ntr, epb, nt;
    size_t prep_smem, stage_smem;
    // diff: with the artificial diffusion of Eq. (3.7) (face pass only)
    cudaError_t (*prepare)(const KArgs<Real> &, bool diff, cudaStream_t);
    // pf: the stage kernel takes its face fluxes from the face pass
    cudaError_t (*stage)(const KArgs<Real> &, int mode, bool pf, bool diff, cudaStream_t);
    cudaError_t (*face)(const KArgs<Real> &, bool diff, cudaStream_t);
    cudaError_t (*alpha_vertex)(const KArgs<Real> &, cudaStream_t);
    cudaError_t (*split)(const KArgs<Real> &, double *, double *, double *, double *, cudaStream_t);
    cudaError_t (*init_bubble)(const KArgs<Real> &, const BubbleArgs &, cudaStream_t);
    cudaError_t (*reduce)(const KArgs<Real> &, double *partials, int nblocks, cudaStream_t);
    // column march (float32 forms only; null for float64): a stage or the
    // right-hand side with the face fluxes evaluated on chip
    cudaError_t (*column)(const KArgs<Real> &, int mode, cudaStream_t);
};

constexpr int kGridStrideBlocks = 152 * 8;

inline int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > (size_t)kGridStrideBlocks) b = kGridStrideBlocks;
    return (int)(b > 0 ? b : 1);
}

template <class S, typename Real>
struct Impl {
    static constexpr size_t prep_smem = sizeof(Real) * ((size_t)S::NTR * S::EPB * S::NP + 2 * S::EPB);
    static constexpr size_t stage_smem = stage_smem_bytes<S, Real, false>();
    static constexpr size_t stage_smem_pf = stage_smem_bytes<S, Real, true>();
    static constexpr size_t stage_smem_diff = stage_smem_bytes<S, Real, true, true>();

    static int blocks(const KArgs<Real> &A) { return (A.M.ne + S::EPB - 1) / S::EPB; }

    template <bool DIFF>
    static cudaError_t launch_prepare(const KArgs<Real> &A, cudaStream_t st) {
        static bool attr = false;
        if (!attr) {
            cudaError_t err = cudaFuncSetAttribute(k_prepare<S, Real, DIFF>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)prep_smem);
            if (err != cudaSuccess) return err;
            attr = true;
        }
        k_prepare<S, Real, DIFF><<<A.ntiles > 0 ? A.ntiles : blocks(A), S::NT, prep_smem, st>>>(A);
        return cudaGetLastError();
    }

    static cudaError_t prepare(const KArgs<Real> &A, bool diff, cudaStream_t st) {
        return diff ? launch_prepare<true>(A, st) : launch_prepare<false>(A, st);
    }

    // the stage kernel of one schedule: float32 face-pass tiles of 64, 128
    // or 256 threads take the variant with the 48-register budget
    template <int MODE, bool PF, bool DIFF>
    static constexpr auto stage_kernel() {
        if constexpr (std::is_same<Real, float>::value && PF && !DIFF &&
                      (S::NT == 64 || S::NT == 128 || S::NT == 256))
            return &k_stage_f32pf<S, MODE>;
        else
            return &k_stage<S, Real, MODE, PF, DIFF>;
    }

    template <int MODE, bool PF, bool DIFF>
    static cudaError_t launch_stage(const KArgs<Real> &A, cudaStream_t st) {
        constexpr size_t smem = DIFF ? stage_smem_diff : (PF ? stage_smem_pf : stage_smem);
        const auto kern = stage_kernel<MODE, PF, DIFF>();
        static bool attr = false;
        if (!attr) {
            cudaError_t err =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            attr = true;
        }
        kern<<<A.ntiles > 0 ? A.ntiles : blocks(A), S::NT, smem, st>>>(A);
        return cudaGetLastError();
    }

    static cudaError_t stage(const KArgs<Real> &A, int mode, bool pf, bool diff, cudaStream_t st) {
        if (diff) {
            if (!pf) return cudaErrorInvalidValue;
            return mode == MODE_RHS ? launch_stage<MODE_RHS, true, true>(A, st)
                                    : launch_stage<MODE_STAGE, true, true>(A, st);
        }
        if (mode == MODE_RHS)
            return pf ? launch_stage<MODE_RHS, true, false>(A, st)
                      : launch_stage<MODE_RHS, false, false>(A, st);
        return pf ? launch_stage<MODE_STAGE, true, false>(A, st)
                  : launch_stage<MODE_STAGE, false, false>(A, st);
    }

    static cudaError_t face(const KArgs<Real> &A, bool diff, cudaStream_t st) {
        const int nb = A.M.fblk[0] + A.M.fblk[1] + A.M.fblk[2];
        if (diff)
            k_face<S, Real, true><<<nb, kFaceThreads, 0, st>>>(A);
        else
            k_face<S, Real, false><<<nb, kFaceThreads, 0, st>>>(A);
        return cudaGetLastError();
    }

    static cudaError_t alpha_vertex(const KArgs<Real> &A, cudaStream_t st) {
        const size_t nvt = (size_t)A.M.nv[0] * A.M.nv[1] * (S::D == 3 ? A.M.nv[2] : 1);
        k_alpha_vertex<S::D, Real><<<grid_for(nvt, 256), 256, 0, st>>>(A.M, A.alphaK,
                                                                        const_cast<Real *>(A.alphaV));
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

    template <int MODE>
    static cudaError_t launch_column(const KArgs<Real> &A, cudaStream_t st) {
        using C = ColShape<S>;
        constexpr size_t smem = column_smem_bytes<S, Real>();
        static bool attr = false;
        if (!attr) {
            cudaError_t err = cudaFuncSetAttribute(k_column<S, Real, MODE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return err;
            attr = true;
        }
        const int nxb = (A.M.n[0] + C::BX - 1) / C::BX;
        const int nyb = S::D == 3 ? (A.M.n[1] + C::BY - 1) / C::BY : 1;
        k_column<S, Real, MODE><<<nxb * nyb, C::NT, smem, st>>>(A);
        return cudaGetLastError();
    }

    static cudaError_t column(const KArgs<Real> &A, int mode, cudaStream_t st) {
        return mode == MODE_RHS ? launch_column<MODE_RHS>(A, st) : launch_column<MODE_STAGE>(A, st);
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
        L.alpha_vertex = &alpha_vertex;
        L.split = &split;
        L.init_bubble = &init_bubble;
        L.reduce = &reduce;
        if constexpr (std::is_same<Real, float>::value)
            L.column = &column;
        else
            L.column = nullptr;
        return L;
    }
};

// Tables defined in the instantiation units; NULL for an unsupported order.
const Launchers<double> *launchers_d2_f64(int K, int rain);
const Launchers<double> *launchers_d3_f64(int K, int rain);
const Launchers<float> *launchers_d2_f32(int K, int rain);
const Launchers<float> *launchers_d3_f32(int K, int rain);
// float64 reference tables with the coefficients scaled by 2/h_j (dg_api.cu)
RefData<double> scaled_ref64(int order, const double two_over_h[3]);
// float64 with float-float contractions (DG_FP64_FFC)
const Launchers<double> *launchers_d2_f64ff(int K, int rain);
const Launchers<double> *launchers_d3_f64ff(int K, int rain);

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

#define DGM_FF_SHAPE(DIM, K, RAIN) Shape<DIM, K, RAIN, (DIM == 3 ? 128 : 256), true>
#define DGM_DEFINE_LAUNCHERS_FF(NAME, DIM)                                             \
    namespace dgm {                                                                    \
    const Launchers<double> *NAME(int K, int rain) {                                   \
        static const Launchers<double> t[5][2] = {                                     \
            {Impl<DGM_FF_SHAPE(DIM, 1, false), double>::table(),                       \
             Impl<DGM_FF_SHAPE(DIM, 1, true), double>::table()},                       \
            {Impl<DGM_FF_SHAPE(DIM, 2, false), double>::table(),                       \
             Impl<DGM_FF_SHAPE(DIM, 2, true), double>::table()},                       \
            {Impl<DGM_FF_SHAPE(DIM, 3, false), double>::table(),                       \
             Impl<DGM_FF_SHAPE(DIM, 3, true), double>::table()},                       \
            {Impl<DGM_FF_SHAPE(DIM, 4, false), double>::table(),                       \
             Impl<DGM_FF_SHAPE(DIM, 4, true), double>::table()},                       \
            {Impl<DGM_FF_SHAPE(DIM, 5, false), double>::table(),                       \
             Impl<DGM_FF_SHAPE(DIM, 5, true), double>::table()},                       \
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
