// dg_rhs_noalloc: the right-hand side of dg_rhs without any device allocation.
//
// Some callers cannot call cudaMalloc: a host program whose memory pool owns
// every byte of the device (a stray allocation would fragment the pool or
// escape its accounting), a latency-critical loop that cannot pay for the
// implicit device synchronisation an allocation may cause, or a process that
// fixes its device-memory budget at start-up.  This entry point serves them:
// the caller passes the inputs and the output, and the scratch the kernels
// need (a saturation-density table, failure counters, derived fields, face
// traces) lives in one file-scope __device__ array of fixed size,
// DG_STATIC_SCRATCH_BYTES, that every GPU which loads the library holds until
// the process exits.  dg_rhs_noalloc_status reads (and clears) the failure
// counters that the calls accumulate there.
//
// The paper has no counterpart: this is packaging; the arithmetic is that of
// the kernels dg_rhs launches (k_prepare, then k_stage in MODE_RHS), with the
// face fluxes evaluated inside the stage kernel (the inline face schedule),
// so the result agrees with dg_rhs to rounding.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "dg_launch.cuh"
#include "dgmoist.h"

using namespace dgm;

namespace {

// The scratch array.  In host code its name is only a stand-in for the
// device symbol, never a device address: its address on each device is
// looked up once with cudaGetSymbolAddress (below) and passed to the kernels.
static __device__ __align__(256) unsigned char g_static_scratch[DG_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

size_t round_up(size_t b) { return (b + 255) & ~(size_t)255; }

// fixed part of the scratch: the rho_vs Taylor table, then the two failure
// counters (Newton iterations at their cap, non-physical nodes); the
// mesh-dependent part (derived fields, one face-trace buffer) follows
constexpr size_t kTableBytes = ((sizeof(double) * kTabStride * kTabN) + 255) & ~(size_t)255;
constexpr size_t kFlagBytes = 256;
constexpr size_t kFixedBytes = kTableBytes + kFlagBytes;

// Address of the scratch array on the current device.  The first call on a
// device (with that device current) looks it up with cudaGetSymbolAddress,
// fills the table and zeroes the counters on the legacy default stream and
// waits for that work; later calls reuse the address.  cudaDeviceReset
// unloads the module and invalidates the cached address, so the entry points
// must not be used on a device after it has been reset.
int scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DG_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return DG_ECUDA;
        }
        unsigned char *base = static_cast<unsigned char *>(p);
        k_fill_rvs_table<<<(kTabN + 255) / 256, 256, 0, 0>>>(reinterpret_cast<double *>(base));
        if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
        if (cudaMemsetAsync(base + kTableBytes, 0, kFlagBytes, 0) != cudaSuccess) return DG_ECUDA;
        if (cudaStreamSynchronize(0) != cudaSuccess) return DG_ECUDA;
        g_scratch_ptr[dev] = base;
    }
    *out = g_scratch_ptr[dev];
    return DG_OK;
}

}  // namespace

extern "C" int dg_rhs_noalloc(const dg_config *cfg, const double *base_node, const double *base_face,
                              const void *U, void *dUdt, void *cuda_stream) {
    if (!cfg || !base_node || !base_face || !U || !dUdt || U == dUdt) return DG_EINVAL;
    const dg_config &g = *cfg;
    if (g.dim != 2 && g.dim != 3) return DG_EINVAL;
    if (g.order < 1 || g.order > 5 || (g.rain != 0 && g.rain != 1)) return DG_EINVAL;
    if (g.precision != DG_FP64) return DG_EINVAL;
    if (g.faces == DG_FACES_PASS) return DG_EINVAL;     // the face pass needs a flux buffer
    // each n[j] bounded before the product, which then fits the int32
    // indexing of the kernels exactly as dg_init_mesh requires
    long long ne = 1;
    for (int j = 0; j < g.dim; ++j) {
        if (g.n[j] < 1 || g.n[j] > (1 << 20) || !(g.L[j] > 0.0) || !std::isfinite(g.L[j]))
            return DG_EINVAL;
        ne *= g.n[j];
        if (ne > 2147483647LL) return DG_EINVAL;
    }
    if (!std::isfinite(g.g)) return DG_EINVAL;
    const Launchers<double> *L =
        g.dim == 2 ? launchers_d2_f64(g.order, g.rain) : launchers_d3_f64(g.order, g.rain);
    if (!L) return DG_EINVAL;
    if (ne * L->np * (long long)(L->nf + 3) * 2 > 2147483647LL) return DG_EINVAL;

    // scratch: the fixed part (table, counters), derived fields, one trace buffer
    const size_t nodes = (size_t)ne * L->np;
    const size_t derived_bytes = round_up(sizeof(double) * L->nd * nodes);
    const size_t trace_bytes = round_up(sizeof(double) * 2 * g.dim * L->ntr * (size_t)ne * L->nfp1);
    if (kFixedBytes + derived_bytes + trace_bytes > (size_t)DG_STATIC_SCRATCH_BYTES) return DG_EINVAL;

    unsigned char *scratch = nullptr;
    int st = scratch_on_current_device(&scratch);
    if (st != DG_OK) return st;

    KArgs<double> A;
    std::memset(&A, 0, sizeof(A));
    MeshData &M = A.M;
    const int p1 = g.order + 1;
    for (int j = 0; j < 3; ++j) {
        M.n[j] = j < g.dim ? g.n[j] : 1;
        M.h[j] = j < g.dim ? g.L[j] / g.n[j] : 1.0;
        M.two_over_h[j] = 2.0 / M.h[j];
        M.periodic[j] = (j < g.dim - 1) ? ((g.periodic_mask >> j) & 1) : 0;
    }
    M.ne = (int)ne;
    M.nzlev_node = g.n[g.dim - 1] * p1;
    M.nzlev_face = g.n[g.dim - 1] + 1;
    M.g = g.g;
    M.rho_w = g.rho_w;
    M.kvr = 130.0 * std::tgamma(4.5) / 6.0 * std::pow(M_PI * 8.0e6, -0.125);
    M.jac = 1.0;
    for (int j = 0; j < g.dim; ++j) M.jac *= M.h[j] / 2.0;
    M.newton_cap = kMaxNewton;
    // the reference tables of dg_init_mesh (scaled by 2/h_j of this mesh)
    A.ref = scaled_ref64(g.order, M.two_over_h);

    A.rvs_tab = reinterpret_cast<const double *>(scratch);
    A.flags = reinterpret_cast<unsigned long long *>(scratch + kTableBytes);
    A.derived = reinterpret_cast<double *>(scratch + kFixedBytes);
    double *trace = reinterpret_cast<double *>(scratch + kFixedBytes + derived_bytes);
    A.bnode = base_node;
    A.bface = base_face;
    A.bnode_d = base_node;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // derived fields and traces are written in full by k_prepare before
    // anything reads them; the counters keep accumulating until
    // dg_rhs_noalloc_status reads and clears them
    A.Uin = static_cast<const double *>(U);
    A.trace_out = trace;
    if (L->prepare(A, false, stream) != cudaSuccess) return DG_ECUDA;
    A.Un = A.Uin;
    A.Uout = static_cast<double *>(dUdt);
    A.trace_in = trace;
    A.trace_out = nullptr;
    A.alpha = 0.0;
    A.beta = 1.0;
    A.gdt = 1.0;
    if (L->stage(A, MODE_RHS, false, false, stream) != cudaSuccess) return DG_ECUDA;
    return DG_OK;
}

extern "C" int dg_rhs_noalloc_status(long long counts[2], void *cuda_stream) {
    unsigned char *scratch = nullptr;
    int st = scratch_on_current_device(&scratch);
    if (st != DG_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned long long h[2] = {0, 0};
    unsigned long long *flags = reinterpret_cast<unsigned long long *>(scratch + kTableBytes);
    if (cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return DG_ECUDA;
    if (cudaMemsetAsync(flags, 0, sizeof(h), stream) != cudaSuccess) return DG_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return DG_ECUDA;
    if (counts) {
        counts[0] = (long long)h[0];
        counts[1] = (long long)h[1];
    }
    if (h[1]) return DG_ENONPHYS;
    if (h[0]) return DG_ENOCONV;
    return DG_OK;
}
