// Private: the context structure shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "dg_launch.cuh"
#include "dgmoist.h"

using namespace dgm;

struct dg_ctx {
    dg_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    int fp32 = 0;
    const Launchers<double> *L64 = nullptr;
    const Launchers<float> *L32 = nullptr;
    int nf = 0, np = 0, nfp1 = 0, nd = 0, ntr = 0, epb = 0;
    long long ne = 0, nodes = 0;
    size_t rsz = 8;
    MeshData M;
    RefData<double> ref64;
    RefData<float> ref32;
    void *U[2] = {nullptr, nullptr};   // U^n, work state
    void *derived = nullptr;
    void *trace[2] = {nullptr, nullptr};
    double *bnode_d = nullptr, *bface_d = nullptr;
    void *bnode_r = nullptr, *bface_r = nullptr;
    unsigned long long *flags = nullptr;
    double *fallout = nullptr;   // rain: accumulated outward water flux per wall face point
    size_t fallout_len = 0;
    double *partials = nullptr;
    double *rvs_tab = nullptr;
    float *bsplit = nullptr;     // DG_FP32_PERT: base-state split tables
    bool face_pass = false;      // faces in k_face (DG_FACES_PASS) instead of in the stage kernel
    bool column = false;         // DG_FACES_COLUMN: the column-march stage kernel (float32 forms)
    void *fbuf = nullptr;        // face pass: fluxes per face point
    int *ftab = nullptr;         // face pass: index in fbuf of each element's 2D faces [ne][2D]
    // artificial diffusion and sponge layer (dg_set_stabilisation)
    dg_stabilisation stab{};
    bool diff = false;           // gamma > 0
    bool in_ensemble = false;    // stepped by dg_ensemble_step (no stabilisation there)
    void *alphaK = nullptr, *alphaV = nullptr;
    void *dtrace[2] = {nullptr, nullptr};
    void *sponge = nullptr;      // delta_R at the node levels, storage type
    // adjoint scratch (allocated on first use): stage states, adjoint vectors,
    // partial node adjoints, neighbour trace adjoints
    const AdjLaunchers *LA = nullptr;
    void *adjX[3] = {nullptr, nullptr, nullptr};
    double *adjL[3] = {nullptr, nullptr, nullptr};
    double *ubar_part = nullptr, *tadj = nullptr;
    int nred = 0;
    std::vector<double> z_node, z_face;
    // host uploads (dg_set_state): the copies of one chunk go to up_stream
    // while the stream splits the chunk before (created on first use)
    cudaStream_t up_stream = nullptr;
    cudaEvent_t up_ev[9] = {};
    bool base_set = false, state_set = false, derived_valid = false;
    int parity = 0;  // trace buffer holding the traces of U^n
    size_t device_bytes = 0;
};


namespace dgm {
// Launch helpers of dg_api.cu used by other units.
int ctx_prepare(dg_ctx *c, const void *U, int tb);
}
